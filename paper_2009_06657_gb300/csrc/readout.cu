// Readouts without forming rho (Sec. II.D):
//   Prob(x) = sum_v |V_xv|^2                         (Eq. 9)
//   <Z_q> = sum_x Prob(x) (-1)^{x_q},  Tr rho = sum_x Prob(x)
//   <P> = Tr(V^dag P V) = sum_x sum_v conj(V[x ^ xm][v]) i^{#Y} (-1)^{pop(x & zm)} V[x][v]
// One warp per row: lanes stride over the row's columns (coalesced), a shuffle
// reduction gives the row value, and per-block partial sums are combined in a
// fixed order in FP64 (deterministic).
#include "common.cuh"
#include "kernels.h"

namespace lret {

constexpr int RO_THREADS = 256;
constexpr int RO_WARPS = RO_THREADS / 32;
constexpr int RO_MAX_BLOCKS = kReadoutMaxBlocks;

template <typename T>
__global__ void __launch_bounds__(RO_THREADS) k_probs(const cx<T>* __restrict__ V, int64_t N, int c, int ld,
                                                      T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = wid; x < N; x += nw) {
    T acc = 0;
    for (int j = lane; j < c; j += 32) {
      const cx<T> v = V[x * ld + j];
      acc += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[x] = acc;
  }
}

// lane l < n accumulates sum_x p(x) (1 - 2 x_l); lane n accumulates the trace.
template <typename T>
__global__ void __launch_bounds__(RO_THREADS) k_zexp(const cx<T>* __restrict__ V, int64_t N, int c, int ld,
                                                     int n, double* __restrict__ partials) {
  __shared__ double red[RO_WARPS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double mine = 0.0;
  for (int64_t x = wid; x < N; x += nw) {
    // row value in the state's precision, sums across rows in FP64
    T acc = 0;
    for (int j = lane; j < c; j += 32) {
      const cx<T> v = V[x * ld + j];
      acc += v.x * v.x + v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const double a = (double)acc;
    if (lane < n) mine += ((x >> lane) & 1) ? -a : a;
    else if (lane == n) mine += a;
  }
  red[warp][lane] = mine;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int w = 0; w < RO_WARPS; ++w) s += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * 32 + threadIdx.x] = s;
  }
}

// out[q] = sum_b partials[q * qstride + b * bstride] in block order
__global__ void k_colsum(const double* __restrict__ partials, int nblocks, int qstride, int bstride,
                         int count, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)q * qstride + (int64_t)b * bstride];
  out[q] = s;
}

template <typename T>
__global__ void __launch_bounds__(RO_THREADS) k_pauli_expect(const cx<T>* __restrict__ V, int64_t N, int c,
                                                             int ld, const uint64_t* __restrict__ xmv,
                                                             const uint64_t* __restrict__ zmv,
                                                             double* __restrict__ partials) {
  __shared__ double red[32];
  const int t = blockIdx.y;
  const uint64_t xm = xmv[t], zm = zmv[t];
  const int ny = __popcll(xm & zm) & 3;
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double mine = 0.0;
  for (int64_t x = wid; x < N; x += nw) {
    const uint64_t y = (uint64_t)x ^ xm;
    // row value in the state's precision, sums across rows in FP64
    T sr = 0, si = 0;
    for (int j = lane; j < c; j += 32) {
      const cx<T> a = V[y * ld + j], b = V[x * ld + j];
      // conj(a) * b
      sr += a.x * b.x + a.y * b.y;
      si += a.x * b.y - a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane != 0) continue;
    // Re(i^ny * S)
    double re;
    switch (ny) {
      case 0: re = sr; break;
      case 1: re = -si; break;
      case 2: re = -sr; break;
      default: re = si; break;
    }
    if (__popcll((uint64_t)x & zm) & 1) re = -re;
    mine += re;
  }
  const double tot = block_sum(mine, red);
  if (threadIdx.x == 0) partials[(int64_t)t * gridDim.x + blockIdx.x] = tot;
}

// The same sums for a group of PG terms per pass: a warp holds row x in registers
// (PJ entries per lane, c <= 32 PJ) and reads the partner row x ^ xmask of each
// term, so a pass over V serves PG terms (1 + PG row reads per row instead of 2 PG; PG = 4 keeps 64 registers).
// Each lane accumulates its entries' signed products over its rows with compensated
// FP32 sums (no per-row warp reduction); the phase i^#Y is applied once at the end
// and the lanes' sums are added in FP64 in a fixed order. The term masks sit in
// shared memory (broadcast reads) to keep registers for occupancy.
constexpr int PG = 4;
__device__ __forceinline__ void neu_add(float& s, float& comp, float v) {
  const float t = s + v;
  comp += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
  s = t;
}
__device__ __forceinline__ void neu_add(double& s, double& comp, double v) { s += v; }

template <typename T, int PJ>
__global__ void __launch_bounds__(RO_THREADS) k_pauli_expect_g(const cx<T>* __restrict__ V, int64_t N, int c,
                                                               int ld, int T_terms, const uint64_t* __restrict__ xmv,
                                                               const uint64_t* __restrict__ zmv,
                                                               double* __restrict__ partials) {
  __shared__ double red[32];
  __shared__ uint64_t s_xm[PG], s_zm[PG];
  const int t0 = blockIdx.y * PG;
  if (threadIdx.x < PG) {
    const int g = threadIdx.x;
    s_xm[g] = t0 + g < T_terms ? xmv[t0 + g] : 0;
    s_zm[g] = t0 + g < T_terms ? zmv[t0 + g] : 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  T sr[PG], si[PG], cr[PG], ci[PG];  // sum of sign * conj(a) b over this lane's entries, compensations
#pragma unroll
  for (int g = 0; g < PG; ++g) sr[g] = si[g] = cr[g] = ci[g] = 0;
  for (int64_t x = wid; x < N; x += nw) {
    cx<T> b[PJ];
#pragma unroll
    for (int k = 0; k < PJ; ++k) {
      const int j = lane + 32 * k;
      b[k] = j < c ? V[(uint64_t)x * ld + j] : mk<T>(0, 0);
    }
#pragma unroll
    for (int g = 0; g < PG; ++g) {
      const uint64_t y = (uint64_t)x ^ s_xm[g];
      const T sg = (__popcll((uint64_t)x & s_zm[g]) & 1) ? (T)-1 : (T)1;
      T pr = 0, pi = 0;
#pragma unroll
      for (int k = 0; k < PJ; ++k) {
        const int j = lane + 32 * k;
        if (j < c) {
          const cx<T> a = V[y * ld + j];  // conj(a) * b
          pr += a.x * b[k].x + a.y * b[k].y;
          pi += a.x * b[k].y - a.y * b[k].x;
        }
      }
      neu_add(sr[g], cr[g], sg * pr);
      neu_add(si[g], ci[g], sg * pi);
    }
  }
#pragma unroll
  for (int g = 0; g < PG; ++g) {
    // Re(i^ny * S)
    const int ny = __popcll(s_xm[g] & s_zm[g]) & 3;
    const double r = (double)sr[g] + (double)cr[g], i = (double)si[g] + (double)ci[g];
    const double re = ny == 0 ? r : ny == 1 ? -i : ny == 2 ? -r : i;
    const double tot = block_sum(re, red);
    if (threadIdx.x == 0 && t0 + g < T_terms) partials[(int64_t)(t0 + g) * gridDim.x + blockIdx.x] = tot;
  }
}

static int ro_blocks(int64_t N) {
  int64_t b = (N + RO_WARPS - 1) / RO_WARPS;
  if (b > RO_MAX_BLOCKS) b = RO_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t launch_probs(const void* V, int64_t N, int c, int ld, void* out, cudaStream_t s) {
  k_probs<T><<<ro_blocks(N), RO_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, (T*)out);
  note_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zexp(const void* V, int64_t N, int c, int ld, int n, double* partials, double* out,
                        cudaStream_t s) {
  const int nb = ro_blocks(N);
  k_zexp<T><<<nb, RO_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, n, partials);
  note_launches(1);
  k_colsum<<<1, 32, 0, s>>>(partials, nb, 1, 32, n + 1, out);
  note_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pauli_expect(const void* V, int64_t N, int c, int ld, int T_terms, const uint64_t* xm,
                                const uint64_t* zm, double* partials, double* out, cudaStream_t s) {
  if (T_terms <= 0) return cudaSuccess;
  const int nb = ro_blocks(N);
  if (c <= 256) {
    dim3 grid(nb, (T_terms + PG - 1) / PG);
    if (c <= 64)
      k_pauli_expect_g<T, 2><<<grid, RO_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, T_terms, xm, zm, partials);
    else if (c <= 128)
      k_pauli_expect_g<T, 4><<<grid, RO_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, T_terms, xm, zm, partials);
    else
      k_pauli_expect_g<T, 8><<<grid, RO_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, T_terms, xm, zm, partials);
  } else {
    dim3 grid(nb, T_terms);
    k_pauli_expect<T><<<grid, RO_THREADS, 0, s>>>((const cx<T>*)V, N, c, ld, xm, zm, partials);
  }
  note_launches(1);
  // out[t] = sum_b partials[t * nb + b]
  k_colsum<<<(T_terms + 127) / 128, 128, 0, s>>>(partials, nb, nb, 1, T_terms, out);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_probs<float>(const void*, int64_t, int, int, void*, cudaStream_t);
template cudaError_t launch_probs<double>(const void*, int64_t, int, int, void*, cudaStream_t);
template cudaError_t launch_zexp<float>(const void*, int64_t, int, int, int, double*, double*, cudaStream_t);
template cudaError_t launch_zexp<double>(const void*, int64_t, int, int, int, double*, double*, cudaStream_t);
template cudaError_t launch_pauli_expect<float>(const void*, int64_t, int, int, int, const uint64_t*,
                                                const uint64_t*, double*, double*, cudaStream_t);
template cudaError_t launch_pauli_expect<double>(const void*, int64_t, int, int, int, const uint64_t*,
                                                 const uint64_t*, double*, double*, cudaStream_t);

}  // namespace lret
