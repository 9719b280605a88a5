// Tensor-core (tcgen05) projection of the row pairs for the FP32 state:
//   [V_new,0 V_new,1] = [V_0 V_1] D      (N/2 x 2c) x (2c x 2k), complex
// the projection V <- V' U_r of the truncation (Theorem 1, Sec. II.B) applied
// without forming V' (D folds the Kraus matrices and the kept eigenvectors).
//
// Real form: with Z the pair rows as interleaved (re, im) floats (4c values)
// and D_r the 4c x 4k real matrix of D ([[Re, Im], [-Im, Re]] per entry), the
// output row is Z D_r. One CTA computes 128 pair rows: the 4c-long rows are
// staged 32 real columns at a time (K-major core-matrix layout, TF32 high part
// + FP32 remainder), D_r^T is pre-split and pre-laid-out in global memory by a
// small kernel and copied per chunk, and one thread issues the 3xTF32 MMAs
// (M = 128, N = 4k, K = 8) into a tensor-memory accumulator; two buffers and
// two mbarriers overlap staging with the MMAs. The epilogue reads the FP32
// accumulator with tcgen05.ld and writes complex64 rows x0 and x0 | 2^q.
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace lret {

namespace {

using namespace tc;

constexpr int PT_THREADS = 256;
constexpr int PT_M = 128;   // pair rows per CTA
constexpr int PT_KC = 32;   // real input columns per chunk
constexpr int PT_MAXN = 256;
constexpr uint32_t PT_LBO = 128;
constexpr uint32_t PT_SBO = (PT_KC / 4) * 128;
constexpr int PT_A_FLOATS = PT_M * PT_KC;        // one of hi / lo
constexpr int PT_B_FLOATS = PT_MAXN * PT_KC;     // one of hi / lo
constexpr int PT_STAGE_FLOATS = 2 * PT_A_FLOATS + 2 * PT_B_FLOATS;
constexpr int PT_SMEM = 2 * PT_STAGE_FLOATS * 4 + 1024;

__device__ __forceinline__ int core_off(int row, int kl) {  // floats, K-major core-matrix layout
  return ((row >> 3) * (PT_KC / 4) + (kl >> 2)) * 32 + (row & 7) * 4 + (kl & 3);
}

// D (2c x 2k complex, row-major) -> per chunk kc: [hi | lo] of D_r^T (N = 4k rows x 32)
__global__ void k_proj_prep(const double2* __restrict__ D, int c, int k, float* __restrict__ B) {
  const int N = 4 * k, K = 4 * c;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
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

__global__ void __launch_bounds__(PT_THREADS, 1)
    k_proj_pair_tc(const float2* __restrict__ V, int ld, int c, int k, int pairbit, int64_t N2,
                   const float* __restrict__ B, float2* __restrict__ W, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* stage = (float*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = 4 * c, N = 4 * k;
  const int nchunks = K / PT_KC;
  const int64_t m0 = (int64_t)blockIdx.x * PT_M;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  bool ok = true;

  for (int ch = 0; ch < nchunks; ++ch) {
    const int s = ch & 1;
    float* a_hi = stage + s * PT_STAGE_FLOATS;
    float* a_lo = a_hi + PT_A_FLOATS;
    float* b_hi = a_lo + PT_A_FLOATS;
    float* b_lo = b_hi + PT_B_FLOATS;
    if (ch >= 2) {
      if (!mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((ch - 2) >> 1) & 1))) ok = false;
    }
    // A: 128 rows x 32 real columns; a float4 covers 4 consecutive real columns
    // (two complex values of one physical row). Each group of 8 lanes stores
    // one 128-byte core matrix (8 rows, same 4-column group): no bank conflicts.
    {
      const int rr = lane & 7, grp = lane >> 3;
      for (int u = warp; u < (PT_M / 8) * 2; u += PT_THREADS / 32) {
        const int g = u >> 1, kgb = (u & 1) * 4;  // row group, first of 4 column groups
        const int row = g * 8 + rr, kg = kgb + grp;
        const int64_t x = m0 + row;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < N2) {
          const int n = ch * PT_KC + kg * 4;  // first real column
          const int b = n >= 2 * c;
          const int cc = (n - b * 2 * c) >> 1;
          const uint64_t xp = insert_zero((uint64_t)x, pairbit) | ((uint64_t)b << pairbit);
          v = __ldg((const float4*)(V + xp * (uint64_t)ld + cc));
        }
        const float h0 = tf32_hi(v.x), h1 = tf32_hi(v.y), h2 = tf32_hi(v.z), h3 = tf32_hi(v.w);
        const int off = core_off(row, kg * 4);
        *(float4*)(a_hi + off) = make_float4(h0, h1, h2, h3);
        *(float4*)(a_lo + off) = make_float4(v.x - h0, v.y - h1, v.z - h2, v.w - h3);
      }
    }
    // B: prepared chunk (hi then lo), contiguous N x 32 floats each
    {
      const float4* src = (const float4*)(B + (int64_t)ch * 2 * (N * PT_KC));
      float4* dst_hi = (float4*)b_hi;
      float4* dst_lo = (float4*)b_lo;
      const int n4 = N * PT_KC / 4;
      for (int i = tid; i < n4; i += PT_THREADS) {
        dst_hi[i] = __ldg(src + i);
        dst_lo[i] = __ldg(src + n4 + i);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      const uint32_t id = idesc_tf32(N);
#pragma unroll
      for (int ks = 0; ks < PT_KC / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 2 * PT_LBO;
        const uint32_t first = (ch == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, sdesc(ah + o, PT_LBO, PT_SBO), sdesc(bh + o, PT_LBO, PT_SBO), id, first);
        mma_tf32(tmem, sdesc(ah + o, PT_LBO, PT_SBO), sdesc(bl + o, PT_LBO, PT_SBO), id, 1u);
        mma_tf32(tmem, sdesc(al + o, PT_LBO, PT_SBO), sdesc(bh + o, PT_LBO, PT_SBO), id, 1u);
      }
      commit(smem_u32(&mbar[s]));
    }
  }
  for (int ch = nchunks - 2; ch < nchunks; ++ch) {
    if (ch < 0) continue;
    if (!mbar_wait(smem_u32(&mbar[ch & 1]), (uint32_t)((ch >> 1) & 1))) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  ok = __syncthreads_and(ok) != 0;
  if (!ok && tid == 0) atomicExch(status, 1);

  // epilogue: warps 0-3, row = 32 warp + lane; real output columns in chunks of 32
  if (warp < 4 && ok) {
    const int row = warp * 32 + lane;
    const int64_t x = m0 + row;
    for (int cb = 0; cb < N; cb += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (x < N2) {
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int J = cb / 2 + jj;  // complex output column of the pair row
          if (J >= 2 * k) break;
          const int b = J >= k;
          const uint64_t xp = insert_zero((uint64_t)x, pairbit) | ((uint64_t)b << pairbit);
          W[xp * (uint64_t)ld + (J - b * k)] = make_float2(v[2 * jj], v[2 * jj + 1]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace

bool proj_pair_tc_supported(int c, int k, int64_t N2) {
  return c % 8 == 0 && 4 * c <= 256 && k % 4 == 0 && k >= 4 && 4 * k <= PT_MAXN && N2 >= 4096;
}

size_t proj_pair_tc_scratch_bytes(int c, int k) { return (size_t)2 * (4 * c) * (4 * k) * sizeof(float); }

cudaError_t launch_proj_pair_tc(const void* V, int ld, int c, int k, int pairbit, int64_t N2, const double2* D,
                                float* Bscratch, void* W, int* status, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_proj_pair_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, PT_SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int nel = (4 * k) * (4 * c);
  k_proj_prep<<<(nel + 255) / 256, 256, 0, s>>>(D, c, k, Bscratch);
  const int blocks = (int)((N2 + PT_M - 1) / PT_M);
  k_proj_pair_tc<<<blocks, PT_THREADS, PT_SMEM, s>>>((const float2*)V, ld, c, k, pairbit, N2, Bscratch,
                                                      (float2*)W, status);
  return cudaGetLastError();
}

}  // namespace lret
