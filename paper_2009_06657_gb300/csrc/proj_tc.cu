// Tensor-core (tcgen05) projection of the row pairs for the FP32 state:
//   [V_new,0 V_new,1] = [V_0 V_1] D      (N/2 x 2c) x (2c x 2k), complex
// the projection V <- V' U_r of the truncation (Theorem 1, Sec. II.B) applied
// without forming V' (D folds the Kraus matrices and the kept eigenvectors).
//
// Real form: with Z the pair rows as interleaved (re, im) floats (4c values)
// and D_r the 4c x 4k real matrix of D ([[Re, Im], [-Im, Re]] per entry), the
// output row is Z D_r. One CTA computes 256 pair rows as two M = 128 MMA tiles
// that share each staged chunk of D_r (two accumulators, 512 tensor-memory
// columns). The K dimension (4c real input columns) is staged 16 at a time in
// a three-deep ring:
//   * warp 8 streams D_r^T chunks (pre-split into TF32 high part + FP32
//     remainder and pre-laid-out in the K-major core-matrix layout by
//     k_proj_prep) with one bulk async copy per chunk (cp.async.bulk, completion
//     on an mbarrier), as soon as the MMAs that used the slot have finished;
//   * warps 0-7 keep the pair rows of the next three chunks in flight in
//     registers while the current one is split and stored, so global latency
//     overlaps the MMAs;
//   * warps 0-7 arrive on the slot's "full" mbarrier once the chunk is stored;
//   * warp 9 waits for both, issues the 3xTF32 MMAs (hi*hi + hi*lo + lo*hi,
//     M = 128, N = 4k, K = 8) for both tiles and commits them to the slot's
//     "free" mbarrier, which the row and D_r producers wait on before reuse.
// The epilogue reads each accumulator with tcgen05.ld, transposes 32 x 32
// blocks through shared memory and writes whole 128-byte row segments of
// rows x0 and x0 | 2^q. Every wait is bounded and sets the status word.
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace lret {

namespace {

using namespace tc;

constexpr int PT_AW = 256;            // row-staging / epilogue threads (warps 0-7)
constexpr int PT_THREADS = PT_AW + 64;  // + warp 8: D_r streaming, warp 9: MMA issue
constexpr int PT_TILE = 128;
constexpr int PT_ROWS = 2 * PT_TILE;  // pair rows per CTA
constexpr int PT_KC = 16;             // real input columns per chunk
constexpr int PT_MAXN = 256;
constexpr int PT_NS = 3;              // ring depth
constexpr uint32_t PT_LBO = 128;
constexpr uint32_t PT_SBO = (PT_KC / 4) * 128;
constexpr int PT_A_FLOATS = PT_ROWS * PT_KC;   // one of hi / lo
constexpr int PT_B_FLOATS = PT_MAXN * PT_KC;   // one of hi / lo
constexpr int PT_STAGE_FLOATS = 2 * PT_A_FLOATS + 2 * PT_B_FLOATS;
constexpr int PT_SMEM = PT_NS * PT_STAGE_FLOATS * 4 + 1024;
constexpr int PT_EP_LD = 36;          // floats per row of the epilogue transpose tile
constexpr int PF = 3;                 // chunks of pair rows in flight in registers

__device__ __forceinline__ int core_off(int row, int kl) {  // floats, K-major core-matrix layout
  return ((row >> 3) * (PT_KC / 4) + (kl >> 2)) * 32 + (row & 7) * 4 + (kl & 3);
}

// barrier of the row-staging warps only (warp 8 keeps streaming)
__device__ __forceinline__ void bar_rows() { asm volatile("barrier.sync 1, %0;" ::"n"(PT_AW) : "memory"); }

// D (2c x 2k complex, row-major) -> per chunk kc: [hi | lo] of D_r^T (N = 4k rows x 16)
__device__ __forceinline__ void proj_prep_body(const double2* __restrict__ D, int c, int k, float* __restrict__ B,
                                               int e) {
  const int N = 4 * k, K = 4 * c;
  if (e >= N * K) return;
  const int n = e / K, kk = e % K;  // B[n][kk] = D_r[kk][n]
  const int I = kk >> 1, J = n >> 1;
  const double2 d = D[(int64_t)I * (2 * k) + J];
  double val;
  if ((kk & 1) == 0) val = (n & 1) ? d.y : d.x;  // re_in -> re_out: Dr, re_in -> im_out: Di
  else val = (n & 1) ? d.x : -d.y;                // im_in -> re_out: -Di, im_in -> im_out: Dr
  const float f = (float)val;
  const float h = tf32_hi(f);
  const int kc = kk / PT_KC, kl = kk % PT_KC;
  float* chunk = B + (int64_t)kc * 2 * (N * PT_KC);
  chunk[core_off(n, kl)] = h;
  chunk[N * PT_KC + core_off(n, kl)] = f - h;
}

__global__ void k_proj_prep(const double2* __restrict__ D, int c, int k, float* __restrict__ B) {
  proj_prep_body(D, c, k, B, blockIdx.x * blockDim.x + threadIdx.x);
}

// one task per blockIdx.y (tasks without the tensor-core projection return at once)
__global__ void k_proj_prep_batch(const TruncTask* __restrict__ tasks) {
  const TruncTask& tk = tasks[blockIdx.y];
  if (!tk.tcp) return;
  proj_prep_body(tk.D, tk.c, tk.k, tk.B, blockIdx.x * blockDim.x + threadIdx.x);
}


// the four float4 of pair-row data this thread stages for chunk ch
__device__ __forceinline__ void load_rows(const float2* __restrict__ V, int ld, int c, int pairbit, int64_t N2,
                                          int64_t m0, int ch, int warp, int lane, float4 (&ra)[4]) {
  const int kg = lane >> 3;
  const int n0 = ch * PT_KC;
  const int b = n0 >= 2 * c;  // the whole chunk lies in one half (2c is a multiple of 16)
  const int cc = ((n0 - b * 2 * c) >> 1) + kg * 2;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = (warp * 4 + i) * 8 + (lane & 7);
    const int64_t x = m0 + row;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (x < N2) {
      const uint64_t xp = insert_zero((uint64_t)x, pairbit) | ((uint64_t)b << pairbit);
      v = __ldg((const float4*)(V + xp * (uint64_t)ld + cc));
    }
    ra[i] = v;
  }
}

// Pair rows tile * 256 .. + 255.
// ssq (nullable): ssq[tile] receives the squared norm of everything this block wrote
// (FP32 per thread, FP64 across the threads in a fixed order).
__device__ __forceinline__ void proj_tc_body(const float2* __restrict__ V, int ld, int c, int k, int pairbit,
                                             int64_t N2, const float* __restrict__ B, float2* __restrict__ W,
                                             int* __restrict__ status, int tile, double* __restrict__ ssq) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* stage = (float*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar_mma[PT_NS], mbar_b[PT_NS], mfull[PT_NS];
  __shared__ __align__(8) uint64_t mdrain;  // every MMA issued by this CTA has completed
  __shared__ int s_fail;
  __shared__ double s_sq[PT_AW / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = 4 * c, N = 4 * k;
  const int nchunks = K / PT_KC;
  const int64_t m0 = (int64_t)tile * PT_ROWS;
  const uint32_t b_bytes = (uint32_t)(2 * N * PT_KC * 4);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < PT_NS; ++s) {
      mbar_init(smem_u32(&mbar_mma[s]), 1);
      mbar_init(smem_u32(&mbar_b[s]), 1);
      mbar_init(smem_u32(&mfull[s]), PT_AW);
    }
    mbar_init(smem_u32(&mdrain), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == PT_AW / 32) {
    // ---- D_r streaming: chunk ch into slot ch % 3 once MMAs of ch - 3 are done
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int s = ch % PT_NS;
        if (ch >= PT_NS) ok = mbar_wait(smem_u32(&mbar_mma[s]), (uint32_t)(((ch - PT_NS) / PT_NS) & 1));
        if (!ok) break;
        float* bdst = stage + s * PT_STAGE_FLOATS + 2 * PT_A_FLOATS;
        bulk_load(smem_u32(bdst), B + (int64_t)ch * 2 * N * PT_KC, b_bytes, smem_u32(&mbar_b[s]));
        issued = ch + 1;
      }
      // no copy may still be landing when the CTA leaves
      for (int ch = issued - PT_NS > 0 ? issued - PT_NS : 0; ch < issued; ++ch)
        if (!mbar_wait(smem_u32(&mbar_b[ch % PT_NS]), (uint32_t)((ch / PT_NS) & 1))) ok = false;
      if (!ok) s_fail = 1;
    }
  } else if (warp == PT_AW / 32 + 1) {
    // ---- MMA issue: chunk ch once its rows are staged and its D_r chunk landed
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int s = ch % PT_NS;
        ok = mbar_wait(smem_u32(&mfull[s]), (uint32_t)((ch / PT_NS) & 1)) &&
             mbar_wait(smem_u32(&mbar_b[s]), (uint32_t)((ch / PT_NS) & 1));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        float* a_hi = stage + s * PT_STAGE_FLOATS;
        float* a_lo = a_hi + PT_A_FLOATS;
        float* b_hi = a_lo + PT_A_FLOATS;
        float* b_lo = b_hi + N * PT_KC;
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
        const uint32_t id = idesc_tf32(N);
#pragma unroll
        for (int ks = 0; ks < PT_KC / 8; ++ks) {
          const uint32_t o = (uint32_t)ks * 2 * PT_LBO;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const uint32_t ot = o + (uint32_t)t * (PT_TILE / 8) * PT_SBO;
            const uint32_t d = tmem + (uint32_t)t * 256u;
            const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
            mma_tf32(d, sdesc(ah + ot, PT_LBO, PT_SBO), sdesc(bh + o, PT_LBO, PT_SBO), id, first);
            mma_tf32(d, sdesc(ah + ot, PT_LBO, PT_SBO), sdesc(bl + o, PT_LBO, PT_SBO), id, 1u);
            mma_tf32(d, sdesc(al + ot, PT_LBO, PT_SBO), sdesc(bh + o, PT_LBO, PT_SBO), id, 1u);
          }
        }
        commit(smem_u32(&mbar_mma[s]));
        issued = ch + 1;
      }
      // whether or not a wait gave up, no MMA may still write tensor memory when
      // it is freed: one more commit tracks all of them (bounded wait)
      if (issued > 0) {
        commit(smem_u32(&mdrain));
        if (!mbar_wait(smem_u32(&mdrain), 0u)) ok = false;
      }
      if (!ok) s_fail = 1;
    }
  } else {
    // ---- pair rows: split into TF32 high part + remainder; three register sets
    // keep the rows of chunks ch + 1 .. ch + 3 in flight while chunk ch is split
    // and stored
    bool ok = true;
    float4 ra[4], rb[4], rc[4];
    auto step = [&](int ch, float4 (&rv)[4]) {
      const int s = ch % PT_NS;
      float* a_hi = stage + s * PT_STAGE_FLOATS;
      float* a_lo = a_hi + PT_A_FLOATS;
      if (ch >= PT_NS && ok) ok = mbar_wait(smem_u32(&mbar_mma[s]), (uint32_t)(((ch - PT_NS) / PT_NS) & 1));
      if (!ok) return;
      const int kg = lane >> 3;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = (warp * 4 + i) * 8 + (lane & 7);
        const float4 v = rv[i];
        const float h0 = tf32_hi(v.x), h1 = tf32_hi(v.y), h2 = tf32_hi(v.z), h3 = tf32_hi(v.w);
        const int off = core_off(row, kg * 4);
        *(float4*)(a_hi + off) = make_float4(h0, h1, h2, h3);
        *(float4*)(a_lo + off) = make_float4(v.x - h0, v.y - h1, v.z - h2, v.w - h3);
      }
      if (ch + PF < nchunks) load_rows(V, ld, c, pairbit, N2, m0, ch + PF, warp, lane, rv);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&mfull[s])) : "memory");
    };
    if (nchunks > 0) load_rows(V, ld, c, pairbit, N2, m0, 0, warp, lane, ra);
    if (nchunks > 1) load_rows(V, ld, c, pairbit, N2, m0, 1, warp, lane, rb);
    if (nchunks > 2) load_rows(V, ld, c, pairbit, N2, m0, 2, warp, lane, rc);
    for (int ch = 0; ch < nchunks && ok; ch += PF) {
      step(ch, ra);
      if (ch + 1 < nchunks) step(ch + 1, rb);
      if (ch + 2 < nchunks) step(ch + 2, rc);
    }
    if (nchunks > 0 && ok) {
      const int ch = nchunks - 1;
      ok = mbar_wait(smem_u32(&mbar_mma[ch % PT_NS]), (uint32_t)((ch / PT_NS) & 1));
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) s_fail = 1;
    bar_rows();
    if (__shfl_sync(0xffffffffu, s_fail, 0) == 0) {  // warp-uniform: tcgen05.ld is warp-collective
      // ---- epilogue: warp w reads tile w / 4, tensor-memory lanes 32 (w % 4) .. + 31
      const int t = warp >> 2, wq = warp & 3;
      float* ep = stage + warp * (32 * PT_EP_LD);  // the ring is idle now
      const int64_t rbase = m0 + t * PT_TILE + wq * 32;
      float sq = 0.f;
      for (int cb = 0; cb < N; cb += 32) {
        float v[32];
        tmem_ld32(tmem + (uint32_t)t * 256u + ((uint32_t)(wq * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *(float4*)(ep + lane * PT_EP_LD + 4 * j) = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        __syncwarp();
        const int piece = lane & 7;
        const int Jp = cb / 2 + 2 * piece;  // first of the piece's two complex output columns
        if (Jp < 2 * k) {
          const int b = Jp >= k;
          const int col = Jp - b * k;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int rl = i * 4 + (lane >> 3);
            const int64_t x = rbase + rl;
            if (x < N2) {
              const uint64_t xp = insert_zero((uint64_t)x, pairbit) | ((uint64_t)b << pairbit);
              const float4 o = *(const float4*)(ep + rl * PT_EP_LD + 4 * piece);
              *(float4*)(W + xp * (uint64_t)ld + col) = o;
              sq += o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
            }
          }
        }
        __syncwarp();
      }
      if (ssq) {
        double d = (double)sq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) s_sq[warp] = d;
      }
    }
    if (ssq) {
      bar_rows();
      if (tid == 0) {
        double t = 0.0;
        if (!s_fail)
          for (int w = 0; w < PT_AW / 32; ++w) t += s_sq[w];
        ssq[tile] = t;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && s_fail) atomicExch(status, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

__global__ void __launch_bounds__(PT_THREADS, 1)
    k_proj_pair_tc(const float2* __restrict__ V, int ld, int c, int k, int pairbit, int64_t N2,
                   const float* __restrict__ B, float2* __restrict__ W, int* __restrict__ status,
                   double* __restrict__ ssq) {
  proj_tc_body(V, ld, c, k, pairbit, N2, B, W, status, blockIdx.x, ssq);
}


// task of block b: the last task whose first block is <= b
__device__ __forceinline__ int pt_task_of_block(const int* __restrict__ bstart, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(PT_THREADS, 1)
    k_proj_pair_tc_batch(const TruncTask* __restrict__ tasks, const int* __restrict__ bstart, int ntasks) {
  const int t = pt_task_of_block(bstart, ntasks, blockIdx.x);
  const TruncTask& tk = tasks[t];
  proj_tc_body((const float2*)tk.V, tk.ld, tk.c, tk.k, tk.q, tk.N2, tk.B, (float2*)tk.W, tk.status,
               blockIdx.x - bstart[t], tk.tcs + 2);
}

// one block per task: the per-block squared norms summed in a fixed order, the new scale
__global__ void __launch_bounds__(256) k_trace_scale_batch(const TruncTask* __restrict__ tasks) {
  const TruncTask& tk = tasks[blockIdx.x];
  if (!tk.tcp) return;
  __shared__ double red[256];
  const int nparts = (int)((tk.N2 + PT_ROWS - 1) / PT_ROWS);
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) v += tk.tcs[2 + i];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tr = 1.0 - tk.acc[0], n2 = red[0];
    tk.tcs[1] = (n2 > 0.0 && tr > 0.0) ? sqrt(tr / n2) : 1.0;
  }
}

}  // namespace

cudaError_t prepare_proj_tc_batch() {
  return cudaFuncSetAttribute(k_proj_pair_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM);
}

cudaError_t launch_proj_pair_tc_batch(const TruncTask* tasks, const int* bstart, int nblocks, int ntasks,
                                      int max_nk, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  k_proj_prep_batch<<<dim3((max_nk + 255) / 256, ntasks), 256, 0, s>>>(tasks);
  k_proj_pair_tc_batch<<<nblocks, PT_THREADS, PT_SMEM, s>>>(tasks, bstart, ntasks);
  k_trace_scale_batch<<<ntasks, 256, 0, s>>>(tasks);
  note_launches(3);
  return cudaGetLastError();
}

bool proj_pair_tc_supported(int c, int k, int64_t N2) {
  return c % 8 == 0 && 4 * c <= 256 && k % 4 == 0 && k >= 4 && 4 * k <= PT_MAXN && N2 >= 4096;
}


int proj_pair_tc_blocks(int64_t N2) { return (int)((N2 + PT_ROWS - 1) / PT_ROWS); }

size_t proj_pair_tc_scratch_bytes(int c, int k) { return (size_t)2 * (4 * c) * (4 * k) * sizeof(float); }

cudaError_t launch_proj_pair_tc(const void* V, int ld, int c, int k, int pairbit, int64_t N2, const double2* D,
                                float* Bscratch, void* W, int* status, double* ssq, cudaStream_t s) {
  static std::atomic<uint64_t> attr_done{0};
  {
    cudaError_t e = set_dyn_smem_once(k_proj_pair_tc, PT_SMEM, attr_done);
    if (e != cudaSuccess) return e;
  }
  const int nel = (4 * k) * (4 * c);
  k_proj_prep<<<(nel + 255) / 256, 256, 0, s>>>(D, c, k, Bscratch);
  note_launches(1);
  const int blocks = (int)((N2 + PT_ROWS - 1) / PT_ROWS);
  k_proj_pair_tc<<<blocks, PT_THREADS, PT_SMEM, s>>>((const float2*)V, ld, c, k, pairbit, N2, Bscratch,
                                                      (float2*)W, status, ssq);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lret
