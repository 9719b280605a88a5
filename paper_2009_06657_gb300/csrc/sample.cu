// Readouts that do not form rho, added to Prob(x) and <O> (Sec. II.D):
//
// * Measurement sampling: the counts of a computational-basis measurement are
//   drawn from Prob(x) = sum_v |V_xv|^2 (Eq. 9). Shot s is the smallest x with
//   CDF(x) > u_s * CDF(N - 1), CDF the running sum of Prob(x) in index order and
//   u_s the caller's uniform draw (inverse-transform sampling). Row values are
//   formed in the state's precision exactly as lr_probs forms them; the CDF is
//   an FP64 scan in a fixed order (blocks of SC_ROWS rows, then block offsets),
//   so a given state and u give the same shots on every run.
// * Von Neumann entropy (App. A): S = -sum_i mu_i log2 mu_i over the eigenvalues
//   mu of rho / Tr rho, which are those of V^dag V / Tr (Theorem 1); the effective
//   rank is 2^S. The spectrum comes from the FP64 eigensolvers; this file holds
//   the final sum.
#include "common.cuh"
#include "kernels.h"

namespace lret {

namespace {

constexpr int SC_THREADS = 256;
constexpr int SC_PER = SC_ROWS / SC_THREADS;  // rows per thread in a block scan

// FP64 scan of one value per thread over the block (fixed order): returns the
// exclusive prefix; *incl receives the inclusive one
__device__ double block_scan(double v, double* wsum, double* incl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double w = v;
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, w, o);
    if (lane >= o) w += t;
  }
  double ex = __shfl_up_sync(0xffffffffu, w, 1);  // exclusive within the warp
  if (lane == 0) ex = 0.0;
  if (lane == 31) wsum[warp] = w;
  __syncthreads();
  if (warp == 0) {
    double a = lane < nw ? wsum[lane] : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, a, o);
      if (lane >= o) a += t;
    }
    double b = __shfl_up_sync(0xffffffffu, a, 1);
    if (lane == 0) b = 0.0;
    if (lane < nw) wsum[lane] = b;  // exclusive warp offsets
  }
  __syncthreads();
  const double off = wsum[warp];
  __syncthreads();  // wsum is reused by the next call
  *incl = off + w;
  return off + ex;
}

// Prob(x) of block b's rows (warp per row, as k_probs) -> local inclusive scan in
// cdf, block total in bsum[b]
template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_prob_scan(const cx<T>* __restrict__ V, int64_t N, int c, int ld,
                                                          double* __restrict__ cdf, double* __restrict__ bsum) {
  __shared__ double rowp[SC_ROWS];
  __shared__ double wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t x0 = (int64_t)blockIdx.x * SC_ROWS;
  for (int rr = warp; rr < SC_ROWS; rr += SC_THREADS / 32) {
    const int64_t x = x0 + rr;
    T acc = 0;
    if (x < N)
      for (int j = lane; j < c; j += 32) {
        const cx<T> v = V[x * ld + j];
        acc += v.x * v.x + v.y * v.y;
      }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rowp[rr] = (double)acc;
  }
  __syncthreads();
  // thread t owns rows SC_PER t .. SC_PER t + SC_PER - 1
  double loc[SC_PER];
  double run = 0.0;
#pragma unroll
  for (int i = 0; i < SC_PER; ++i) {
    run += rowp[threadIdx.x * SC_PER + i];
    loc[i] = run;
  }
  double incl;
  const double excl = block_scan(run, wsum, &incl);
#pragma unroll
  for (int i = 0; i < SC_PER; ++i) {
    const int64_t x = x0 + threadIdx.x * SC_PER + i;
    if (x < N) cdf[x] = excl + loc[i];
  }
  if (threadIdx.x == SC_THREADS - 1) bsum[blockIdx.x] = incl;
}

// exclusive offsets of the block totals (one block of SC_THREADS threads; each
// thread a contiguous segment), and the grand total in boff[nb]
__global__ void __launch_bounds__(SC_THREADS) k_block_offsets(const double* __restrict__ bsum, int nb,
                                                              double* __restrict__ boff) {
  __shared__ double wsum[32];
  const int seg = (nb + SC_THREADS - 1) / SC_THREADS;
  const int b0 = threadIdx.x * seg;
  double run = 0.0;
  for (int b = b0; b < b0 + seg && b < nb; ++b) run += bsum[b];
  double incl;
  double acc = block_scan(run, wsum, &incl);
  for (int b = b0; b < b0 + seg && b < nb; ++b) {
    boff[b] = acc;
    acc += bsum[b];
  }
  if (threadIdx.x == SC_THREADS - 1) boff[nb] = incl;
}

__global__ void k_add_offsets(double* __restrict__ cdf, int64_t N, const double* __restrict__ boff) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (int64_t)gridDim.x * blockDim.x)
    cdf[x] += boff[x / SC_ROWS];
}

// shot s: smallest x with cdf[x] > u_s * total, clamped to N - 1
__global__ void k_search(const double* __restrict__ cdf, int64_t N, const double* __restrict__ total,
                         const double* __restrict__ u, int shots, int64_t* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= shots) return;
  const double t = u[s] * total[0];
  int64_t lo = 0, hi = N - 1;  // answer in [lo, hi]
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] > t) hi = mid;
    else lo = mid + 1;
  }
  out[s] = lo;
}

// S and 2^S from m eigenvalues (any order), fixed-order sums in one block
__global__ void __launch_bounds__(SC_THREADS) k_entropy(const double* __restrict__ lam, int m,
                                                        double* __restrict__ out) {
  __shared__ double red[32];
  __shared__ double s_tot;
  double mine = 0.0;
  for (int i = threadIdx.x; i < m; i += SC_THREADS) mine += lam[i] > 0.0 ? lam[i] : 0.0;
  const double tot = block_sum(mine, red);
  if (threadIdx.x == 0) s_tot = tot;
  __syncthreads();
  const double inv = s_tot > 0.0 ? 1.0 / s_tot : 0.0;
  double h = 0.0;
  for (int i = threadIdx.x; i < m; i += SC_THREADS) {
    const double mu = (lam[i] > 0.0 ? lam[i] : 0.0) * inv;
    if (mu > 0.0) h -= mu * log2(mu);
  }
  const double S = block_sum(h, red);
  if (threadIdx.x == 0) {
    out[0] = S;
    out[1] = exp2(S);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_sample(const void* V, int64_t N, int c, int ld, double* cdf, double* bsum, double* boff,
                          const double* u, int shots, int64_t* out, cudaStream_t s) {
  const int nb = (int)((N + SC_ROWS - 1) / SC_ROWS);
  k_prob_scan<T><<<nb, SC_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, cdf, bsum);
  note_launches(1);
  k_block_offsets<<<1, SC_THREADS, 0, s>>>(bsum, nb, boff);
  note_launches(1);
  int ab = (int)((N + 255) / 256);
  if (ab > 4096) ab = 4096;
  k_add_offsets<<<ab, 256, 0, s>>>(cdf, N, boff);
  note_launches(1);
  if (shots > 0) {
    k_search<<<(shots + 255) / 256, 256, 0, s>>>(cdf, N, boff + nb, u, shots, out);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_entropy(const double* lam, int m, double* out, cudaStream_t s) {
  k_entropy<<<1, SC_THREADS, 0, s>>>(lam, m, out);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_sample<float>(const void*, int64_t, int, int, double*, double*, double*,
                                          const double*, int, int64_t*, cudaStream_t);
template cudaError_t launch_sample<double>(const void*, int64_t, int, int, double*, double*, double*,
                                           const double*, int, int64_t*, cudaStream_t);

}  // namespace lret
