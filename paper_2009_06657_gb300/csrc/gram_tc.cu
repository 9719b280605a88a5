// Tensor-core (tcgen05) Gram of the row pairs for the FP32 state:
//   S = Z^dag Z,  Z = [V_0 V_1]  (N/2 x 2c complex; V_b = rows of V with bit q = b)
// which the truncation of Sec. II.B needs (the Gram of the implicit V' is
// assembled from S). In the real view Y (N/2 x 4c floats, interleaved re/im),
// S comes from the real Gram R = Y^T Y:
//   Re S_ij = R[2i][2j] + R[2i+1][2j+1],  Im S_ij = R[2i][2j+1] - R[2i+1][2j].
//
// One CTA (8 warps) per split of the rows. Rows are staged 32 at a time into
// shared memory in the K-major, no-swizzle core-matrix layout (8 rows x 16 B per
// core matrix; 128 B between core matrices along K, 1024 B between 8-row groups),
// each FP32 value split into a TF32 high part and an FP32 remainder; one thread
// issues tcgen05.mma kind::tf32 (hi*hi + hi*lo + lo*hi, the 3xTF32 product) into
// FP32 accumulators in tensor memory. Warps 0-7 stage chunks (the loads of the
// next two chunks stay in flight in registers while the current one is stored)
// into a three-deep ring and arrive on the slot's "full" mbarrier; warp 8 waits
// on it, issues the chunk's MMAs and commits them to the slot's "free"
// mbarrier, on which the staging warps wait before reusing the slot. Every wait
// is bounded and sets a status word instead of hanging. The accumulators hold the upper triangle of R by 128-row blocks: block 0
// (rows 0..127) x all columns, block 1 (rows 128..255) x columns 128..255. The
// epilogue reads them with tcgen05.ld, folds 2x2 real blocks into complex S
// entries and writes this split's FP32 partial; the split partials are summed in
// FP64 in a fixed order by the same reduction as the SIMT path (deterministic).
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace lret {

namespace {

using namespace tc;

constexpr int TC_SW = 256;              // row-staging threads (warps 0-7); warps 0-3 also run the epilogue
constexpr int TC_THREADS = TC_SW + 32;  // + warp 8: issues the MMAs
constexpr int TC_KC = 32;                       // rows per staged chunk
constexpr int TC_MAXR = 256;                    // real columns (4c) at most
constexpr int TC_NS = 3;                        // ring depth
constexpr int TC_PART_FLOATS = TC_MAXR * TC_KC; // one hi or lo operand chunk
constexpr int TC_STAGE_FLOATS = 2 * TC_PART_FLOATS;
constexpr uint32_t TC_LBO = 128;                // bytes between core matrices along K
constexpr uint32_t TC_SBO = (TC_KC / 4) * 128;  // bytes between 8-row groups
constexpr int TC_SMEM = TC_NS * TC_STAGE_FLOATS * 4 + 1024;
constexpr int TC_UPW = 8;                       // (4-row group, 32-column strip) units per warp

// the 32 values (8 units x 4 rows) this thread stages for the chunk at row x0
__device__ __forceinline__ void gram_load(const float2* __restrict__ V, int ld, int c, int pairbit, int64_t x0,
                                          int64_t x_end, int NR, int strips, int units, int warp, int lane,
                                          float (&val)[TC_UPW][4]) {
  const int ub = warp * TC_UPW;
#pragma unroll
  for (int uu = 0; uu < TC_UPW; ++uu) {
    const int u = ub + uu;
    const int kg = u / strips, strip = u % strips;
    const int n = strip * 32 + lane;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t x = x0 + kg * 4 + i;
      float v = 0.f;
      if (u < units && n < NR && x < x_end) {
        const int b = n >= 2 * c;             // which row of the pair
        const int cc = (n - b * 2 * c) >> 1;  // complex column
        const uint64_t xp = insert_zero((uint64_t)x, pairbit) | ((uint64_t)b << pairbit);
        v = __ldg((const float*)(V + xp * (uint64_t)ld + cc) + (n & 1));
      }
      val[uu][i] = v;
    }
  }
}

// One split of the rows: row pairs split * rows_per_split .. + rows_per_split - 1,
// its FP32 partial of S into P (2c x 2c).
__device__ __forceinline__ void gram_tc_body(const float2* __restrict__ V, int ld, int c, int pairbit, int64_t N2,
                                             int64_t rows_per_split, int split, float2* __restrict__ P,
                                             int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand area
  float* stage = (float*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[TC_NS];   // slot free again: the MMAs that read it are done
  __shared__ __align__(8) uint64_t mfull[TC_NS];  // slot staged by all TC_SW threads
  __shared__ __align__(8) uint64_t mdrain;        // every MMA issued by this CTA has completed
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NR = 4 * c;               // real columns
  const int nacc = NR > 128 ? 2 : 1;  // 128-row accumulator blocks
  const int rows_pad = NR < 128 ? 128 : NR;
  const int64_t x_begin = (int64_t)split * rows_per_split;
  int64_t x_end = x_begin + rows_per_split;
  if (x_end > N2) x_end = N2;
  const int nchunks = x_begin < x_end ? (int)((x_end - x_begin + TC_KC - 1) / TC_KC) : 0;
  const int strips = (NR + 31) / 32;
  const int units = (TC_KC / 4) * strips;  // <= 64 = 8 warps x TC_UPW

  // zero the ring once: padding rows (NR..rows_pad) must read as zero
  for (int i = tid; i < TC_NS * TC_STAGE_FLOATS; i += TC_THREADS) stage[i] = 0.f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < TC_NS; ++s) {
      mbar_init(smem_u32(&mbar[s]), 1);
      mbar_init(smem_u32(&mfull[s]), TC_SW);
    }
    mbar_init(smem_u32(&mdrain), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t acc_col[2] = {0u, 256u};  // accumulator 0: columns 0..255, 1: 256..383
  bool ok = true;

  if (warp == TC_SW / 32) {
    // ---- MMA issue: chunk ch once all staging threads have stored it
    if (lane == 0) {
      int issued = 0;
      for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int s = ch % TC_NS;
        ok = mbar_wait(smem_u32(&mfull[s]), (uint32_t)((ch / TC_NS) & 1));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        float* hi = stage + s * TC_STAGE_FLOATS;
        float* lo = hi + TC_PART_FLOATS;
        const uint32_t base_hi = smem_u32(hi), base_lo = smem_u32(lo);
#pragma unroll
        for (int ks = 0; ks < TC_KC / 8; ++ks) {
          for (int a = 0; a < nacc; ++a) {
            const uint32_t aoff = (uint32_t)(a * 16) * TC_SBO + (uint32_t)ks * 2 * TC_LBO;
            const uint32_t boff = (uint32_t)(a * 16) * TC_SBO + (uint32_t)ks * 2 * TC_LBO;
            const int ncols = a == 0 ? NR : NR - 128;
            const uint32_t id = idesc_tf32(ncols < 16 ? 16 : ncols);
            const uint32_t d = tmem + acc_col[a];
            const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
            mma_tf32(d, sdesc(base_hi + aoff, TC_LBO, TC_SBO), sdesc(base_hi + boff, TC_LBO, TC_SBO), id, first);
            mma_tf32(d, sdesc(base_hi + aoff, TC_LBO, TC_SBO), sdesc(base_lo + boff, TC_LBO, TC_SBO), id, 1u);
            mma_tf32(d, sdesc(base_lo + aoff, TC_LBO, TC_SBO), sdesc(base_hi + boff, TC_LBO, TC_SBO), id, 1u);
          }
        }
        commit(smem_u32(&mbar[s]));
        issued = ch + 1;
      }
      // whether or not a wait gave up, no MMA may still write tensor memory when
      // it is freed: one more commit tracks all of them (bounded wait)
      if (issued > 0) {
        commit(smem_u32(&mdrain));
        if (!mbar_wait(smem_u32(&mdrain), 0u)) ok = false;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  } else {
    // ---- row staging: two register sets keep the loads of chunks ch + 1 and
    // ch + 2 in flight while chunk ch is split and stored; slot ch % 3 is reused
    // once the MMAs of chunk ch - 3 have completed
    float va[TC_UPW][4], vb[TC_UPW][4];
    auto load = [&](int ch, float (&val)[TC_UPW][4]) {
      gram_load(V, ld, c, pairbit, x_begin + (int64_t)ch * TC_KC, x_end, NR, strips, units, warp, lane, val);
    };
    auto step = [&](int ch, float (&val)[TC_UPW][4]) {
      const int s = ch % TC_NS;
      float* hi = stage + s * TC_STAGE_FLOATS;
      float* lo = hi + TC_PART_FLOATS;
      if (ch >= TC_NS && ok) ok = mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((ch - TC_NS) / TC_NS) & 1));
      if (!ok) return;
      const int ub = warp * TC_UPW;
#pragma unroll
      for (int uu = 0; uu < TC_UPW; ++uu) {
        const int u = ub + uu;
        const int kg = u / strips, strip = u % strips;
        const int n = strip * 32 + lane;
        if (u < units && n < rows_pad) {
          float h4[4], l4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            h4[i] = tf32_hi(val[uu][i]);
            l4[i] = val[uu][i] - h4[i];
          }
          const int off = ((n >> 3) * (TC_KC / 4) + kg) * 32 + (n & 7) * 4;  // floats
          *(float4*)(hi + off) = make_float4(h4[0], h4[1], h4[2], h4[3]);
          *(float4*)(lo + off) = make_float4(l4[0], l4[1], l4[2], l4[3]);
        }
      }
      if (ch + 2 < nchunks) load(ch + 2, val);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&mfull[s])) : "memory");
    };
    if (nchunks > 0) load(0, va);
    if (nchunks > 1) load(1, vb);
    for (int ch = 0; ch < nchunks && ok; ch += 2) {
      step(ch, va);
      if (ch + 1 < nchunks) step(ch + 1, vb);
    }
    // the last commit covers every MMA issued before it
    if (nchunks > 0 && ok) {
      const int ch = nchunks - 1;
      ok = mbar_wait(smem_u32(&mbar[ch % TC_NS]), (uint32_t)((ch / TC_NS) & 1));
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  ok = __syncthreads_and(ok) != 0;  // block-uniform: tcgen05.ld below is warp-collective
  if (!ok && tid == 0) atomicExch(status, 1);

  // epilogue: real row r = 128 a + 32 warp + lane; fold into complex S rows, in
  // FP32 (FP64 arithmetic runs at 1/62 of the FP32 rate here); the split
  // partials are summed in FP64
  const int C2 = 2 * c;  // complex columns of S
  for (int a = 0; a < nacc && warp < 4; ++a) {
    const int r = a * 128 + warp * 32 + lane;
    const int col0 = a == 0 ? 0 : 128;
    const int ncols = a == 0 ? NR : NR - 128;
    for (int cb = 0; cb < ncols; cb += 32) {
      float v[32];
      if (nchunks > 0 && ok) {
        tmem_ld32(tmem + acc_col[a] + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
      }
      // odd rows hand their values to the even row below them
      float w[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) w[j] = __shfl_xor_sync(0xffffffffu, v[j], 1);
      if ((r & 1) == 0 && r < NR) {
        const int i = r >> 1;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int j = (col0 + cb) / 2 + jj;
          if (j >= C2) break;
          // v: row 2i, w: row 2i+1; columns 2j, 2j+1 at positions 2jj, 2jj+1
          P[(int64_t)i * C2 + j] = make_float2(v[2 * jj] + w[2 * jj + 1], v[2 * jj + 1] - w[2 * jj]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gram_pair_tc(const float2* __restrict__ V, int ld, int c, int pairbit, int64_t N2, int64_t rows_per_split,
                   double2* __restrict__ partials, int* __restrict__ status) {
  gram_tc_body(V, ld, c, pairbit, N2, rows_per_split, blockIdx.x,
               reinterpret_cast<float2*>(partials) + (int64_t)blockIdx.x * (2 * c) * (2 * c), status);
}

// task of block b: the last task whose first block is <= b (tasks with no blocks are
// skipped because the next task starts at the same block)
__device__ __forceinline__ int tc_task_of_block(const int* __restrict__ bstart, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gram_pair_tc_batch(const TruncTask* __restrict__ tasks, const int* __restrict__ bstart, int ntasks) {
  const int t = tc_task_of_block(bstart, ntasks, blockIdx.x);
  const TruncTask& tk = tasks[t];
  const int split = blockIdx.x - bstart[t];
  const int c = tk.c;
  gram_tc_body((const float2*)tk.V, tk.ld, c, tk.q, tk.N2, tk.tc_rows, split,
               reinterpret_cast<float2*>(tk.partials) + (int64_t)split * (2 * c) * (2 * c), tk.status);
}

}  // namespace

cudaError_t prepare_gram_tc_batch() {
  return cudaFuncSetAttribute(k_gram_pair_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
}

cudaError_t launch_gram_pair_tc_batch(const TruncTask* tasks, const int* bstart, int nblocks, int ntasks,
                                      cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  k_gram_pair_tc_batch<<<nblocks, TC_THREADS, TC_SMEM, s>>>(tasks, bstart, ntasks);
  note_launches(1);
  return cudaGetLastError();
}

bool gram_pair_tc_supported(int c, int64_t N2) { return c % 8 == 0 && c >= 8 && 4 * c <= TC_MAXR && N2 >= 4096; }

cudaError_t launch_gram_pair_tc(const void* V, int ld, int c, int pairbit, int64_t N2, double2* partials,
                                int max_splits, double2* out, int* status, cudaStream_t s) {
  int splits = 152;
  if (splits > max_splits) splits = max_splits;
  int64_t rows = (N2 + splits - 1) / splits;
  rows = ((rows + TC_KC - 1) / TC_KC) * TC_KC;
  splits = (int)((N2 + rows - 1) / rows);
  static std::atomic<uint64_t> attr_done{0};
  {
    cudaError_t e = set_dyn_smem_once(k_gram_pair_tc, TC_SMEM, attr_done);
    if (e != cudaSuccess) return e;
  }
  k_gram_pair_tc<<<splits, TC_THREADS, TC_SMEM, s>>>((const float2*)V, ld, c, pairbit, N2, rows, partials, status);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce_herm_f32(reinterpret_cast<const float2*>(partials), splits, 2 * c, out, s);
}

}  // namespace lret
