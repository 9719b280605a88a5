// Gate application fused with Kraus expansion (Eqs. 3 and 4), its adjoint,
// and the Pauli-sum apply used to seed the adjoint pass.
//
// V is a row-major slab: row x (basis state x, qubit q = bit q of x) holds c
// interleaved complex amplitudes at V[x*ld + j]. A one-qubit operator pairs
// rows x and x | 2^q; a two-qubit operator works on the four rows that differ
// only in its two bits. Consecutive threads take consecutive columns j of the
// same row group, so every load and store is a coalesced run of 8c (complex64)
// or 16c (complex128) bytes per row.
#include "common.cuh"
#include "kernels.h"

namespace lret {

template <int G>
__device__ __forceinline__ void group_rows(uint64_t grp, const int* bits, uint64_t* rows) {
  if (G == 2) {
    const uint64_t x0 = insert_zero(grp, bits[0]);
    rows[0] = x0;
    rows[1] = x0 | (1ull << bits[0]);
  } else {
    const int lo = bits[0] < bits[1] ? bits[0] : bits[1];
    const int hi = bits[0] < bits[1] ? bits[1] : bits[0];
    const uint64_t base = insert_zero(insert_zero(grp, lo), hi);
#pragma unroll
    for (int g = 0; g < 4; ++g)
      rows[g] = base | ((uint64_t)((g >> 1) & 1) << bits[0]) | ((uint64_t)(g & 1) << bits[1]);
  }
}

// W[x_a][alpha*c + j] = sum_g M[alpha][a][g] V[x_g][j]
template <typename T, int G>
__global__ void __launch_bounds__(256) k_expand(const cx<T>* __restrict__ V, cx<T>* __restrict__ W,
                                                int64_t total, int c, int ld, GroupOp op) {
  // operator matrices converted once per block (FP64 -> T conversion is slow per use)
  __shared__ cx<T> sM[4][G][G];
  const int K = op.K;
  for (int i = threadIdx.x; i < 4 * G * G; i += blockDim.x) {
    const int al = i / (G * G), a = (i / G) % G, g = i % G;
    sM[al][a][g] = from_d2<T>(op.M[al][a][g]);
  }
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t grp = (uint64_t)(e / c);
    const int j = (int)(e - (int64_t)grp * c);
    uint64_t rows[G];
    group_rows<G>(grp, op.bits, rows);
    cx<T> v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = V[rows[g] * (uint64_t)ld + j];
    for (int al = 0; al < K; ++al) {
#pragma unroll
      for (int a = 0; a < G; ++a) {
        cx<T> acc = mk<T>(0, 0);
#pragma unroll
        for (int g = 0; g < G; ++g) cfma(acc, sM[al][a][g], v[g]);
        W[rows[a] * (uint64_t)ld + (uint64_t)al * c + j] = acc;
      }
    }
  }
}

// Batched expansion: block b serves task t with bstart[t] <= b < bstart[t+1].
__device__ __forceinline__ int expand_task_of_block(const int* __restrict__ bstart, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, int G>
__device__ __forceinline__ void expand_batch_body(const ExpandTask& tk, int lb, int nlb) {
  __shared__ cx<T> sM[4][G][G];
  for (int i = threadIdx.x; i < tk.K * G * G; i += blockDim.x) {
    const int al = i / (G * G), a = (i / G) % G, g = i % G;
    sM[al][a][g] = from_d2<T>(tk.M[(al * G + a) * G + g]);
  }
  __syncthreads();
  const cx<T>* V = (const cx<T>*)tk.V;
  cx<T>* W = (cx<T>*)tk.W;
  const int c = tk.c, ld = tk.ld, K = tk.K;
  for (int64_t e = (int64_t)lb * blockDim.x + threadIdx.x; e < tk.total; e += (int64_t)nlb * blockDim.x) {
    const uint64_t grp = (uint64_t)(e / c);
    const int j = (int)(e - (int64_t)grp * c);
    uint64_t rows[G];
    group_rows<G>(grp, tk.bits, rows);
    cx<T> v[G];
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = V[rows[g] * (uint64_t)ld + j];
    for (int al = 0; al < K; ++al) {
#pragma unroll
      for (int a = 0; a < G; ++a) {
        cx<T> acc = mk<T>(0, 0);
#pragma unroll
        for (int g = 0; g < G; ++g) cfma(acc, sM[al][a][g], v[g]);
        W[rows[a] * (uint64_t)ld + (uint64_t)al * c + j] = acc;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_expand_batch(const ExpandTask* __restrict__ tasks,
                                                      const int* __restrict__ bstart, int ntasks) {
  const int t = expand_task_of_block(bstart, ntasks, blockIdx.x);
  const ExpandTask& tk = tasks[t];
  const int lb = blockIdx.x - bstart[t], nlb = bstart[t + 1] - bstart[t];
  if (tk.G == 2) expand_batch_body<T, 2>(tk, lb, nlb);
  else expand_batch_body<T, 4>(tk, lb, nlb);
}

int expand_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return b < 1 ? 1 : (int)b;
}

template <typename T>
cudaError_t launch_expand_batch(const ExpandTask* tasks, const int* bstart, int nblocks, int ntasks,
                                cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  k_expand_batch<T><<<nblocks, 256, 0, s>>>(tasks, bstart, ntasks);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t launch_expand_batch<float>(const ExpandTask*, const int*, int, int, cudaStream_t);
template cudaError_t launch_expand_batch<double>(const ExpandTask*, const int*, int, int, cudaStream_t);

static int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  const int64_t cap = 152 * 16;  // 16 resident 256-thread blocks per SM, grid-stride beyond
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t launch_expand(const void* V, void* W, int64_t N, int c, int ld, const GroupOp& op,
                          cudaStream_t s) {
  const int64_t total = (N / op.G) * (int64_t)c;
  if (total == 0) return cudaSuccess;
  const int blocks = grid_for(total, 256);
  if (op.G == 2)
    k_expand<T, 2><<<blocks, 256, 0, s>>>((const cx<T>*)V, (cx<T>*)W, total, c, ld, op);
  else
    k_expand<T, 4><<<blocks, 256, 0, s>>>((const cx<T>*)V, (cx<T>*)W, total, c, ld, op);
  note_launches(1);
  return cudaGetLastError();
}

// Adjoint: Vbar[x_g][j] = sum_{alpha,a} conj(M[alpha][a][g]) Wbar[x_a][alpha*c + j]
//          grad += 2 Re sum_{alpha,a} conj(Wbar[x_a][alpha*c+j]) * (sum_g dM[alpha][a][g] Vin[x_g][j])
template <typename T, int G>
__global__ void __launch_bounds__(256) k_expand_adj(const cx<T>* __restrict__ Wbar,
                                                    const cx<T>* __restrict__ Vin,
                                                    cx<T>* __restrict__ Vbar, int64_t total, int c,
                                                    int ld, GroupOp op, double* grad_partials) {
  __shared__ double red[32];
  __shared__ cx<T> sM[4][G][G], sdM[4][G][G];
  const int K = op.K;
  for (int i = threadIdx.x; i < 4 * G * G; i += blockDim.x) {
    const int al = i / (G * G), a = (i / G) % G, g = i % G;
    sM[al][a][g] = from_d2<T>(op.M[al][a][g]);
    sdM[al][a][g] = from_d2<T>(op.dM[al][a][g]);
  }
  __syncthreads();
  double gacc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t grp = (uint64_t)(e / c);
    const int j = (int)(e - (int64_t)grp * c);
    uint64_t rows[G];
    group_rows<G>(grp, op.bits, rows);
    cx<T> vin[G], out[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      out[g] = mk<T>(0, 0);
      vin[g] = op.has_grad ? Vin[rows[g] * (uint64_t)ld + j] : mk<T>(0, 0);
    }
    for (int al = 0; al < K; ++al) {
#pragma unroll
      for (int a = 0; a < G; ++a) {
        const cx<T> wb = Wbar[rows[a] * (uint64_t)ld + (uint64_t)al * c + j];
#pragma unroll
        for (int g = 0; g < G; ++g) cfmac(out[g], sM[al][a][g], wb);
        if (op.has_grad) {
          cx<T> dv = mk<T>(0, 0);
#pragma unroll
          for (int g = 0; g < G; ++g) cfma(dv, sdM[al][a][g], vin[g]);
          // Re(conj(wb) * dv)
          gacc += (double)wb.x * (double)dv.x + (double)wb.y * (double)dv.y;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) Vbar[rows[g] * (uint64_t)ld + j] = out[g];
  }
  if (op.has_grad) {
    const double tot = block_sum(2.0 * gacc, red);
    if (threadIdx.x == 0) grad_partials[blockIdx.x] = tot;
  }
}

template <typename T>
cudaError_t launch_expand_adj(const void* Wbar, const void* Vin, void* Vbar, int64_t N, int c, int ld,
                              const GroupOp& op, double* grad_partials, int* nblocks_out,
                              cudaStream_t s) {
  const int64_t total = (N / op.G) * (int64_t)c;
  const int blocks = grid_for(total, 256);
  *nblocks_out = blocks;
  if (op.G == 2)
    k_expand_adj<T, 2><<<blocks, 256, 0, s>>>((const cx<T>*)Wbar, (const cx<T>*)Vin, (cx<T>*)Vbar,
                                              total, c, ld, op, grad_partials);
  else
    k_expand_adj<T, 4><<<blocks, 256, 0, s>>>((const cx<T>*)Wbar, (const cx<T>*)Vin, (cx<T>*)Vbar,
                                              total, c, ld, op, grad_partials);
  note_launches(1);
  return cudaGetLastError();
}

// out[y][j] = sum_t coeff_t * (P_t V)[y][j], with P|x> = i^{#Y} (-1)^{pop(x & zm)} |x ^ xm>,
// so (P V)[y] = i^{#Y} (-1)^{pop((y ^ xm) & zm)} V[y ^ xm].
template <typename T>
__global__ void __launch_bounds__(256) k_pauli_apply(const cx<T>* __restrict__ V, cx<T>* __restrict__ out,
                                                     int64_t total, int c, int ld, int nterms,
                                                     const uint64_t* __restrict__ xm,
                                                     const uint64_t* __restrict__ zm,
                                                     const double* __restrict__ coeff) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t y = (uint64_t)(e / c);
    const int j = (int)(e - (int64_t)y * c);
    double ar = 0.0, ai = 0.0;
    for (int t = 0; t < nterms; ++t) {
      const uint64_t x = y ^ xm[t];
      const int ny = __popcll(xm[t] & zm[t]) & 3;
      const int sgn = __popcll(x & zm[t]) & 1;
      const cx<T> v = V[x * (uint64_t)ld + j];
      double vr = (double)v.x, vi = (double)v.y;
      // multiply by i^ny
      double pr, pi;
      switch (ny) {
        case 0: pr = vr; pi = vi; break;
        case 1: pr = -vi; pi = vr; break;
        case 2: pr = -vr; pi = -vi; break;
        default: pr = vi; pi = -vr; break;
      }
      const double cf = sgn ? -coeff[t] : coeff[t];
      ar += cf * pr;
      ai += cf * pi;
    }
    out[y * (uint64_t)ld + j] = mk<T>((T)ar, (T)ai);
  }
}

template <typename T>
cudaError_t launch_pauli_apply(const void* V, void* out, int64_t N, int c, int ld, int T_terms,
                               const uint64_t* xm, const uint64_t* zm, const double* coeff,
                               cudaStream_t s) {
  const int64_t total = N * (int64_t)c;
  const int blocks = grid_for(total, 256);
  k_pauli_apply<T><<<blocks, 256, 0, s>>>((const cx<T>*)V, (cx<T>*)out, total, c, ld, T_terms, xm, zm,
                                          coeff);
  note_launches(1);
  return cudaGetLastError();
}

__global__ void k_sum(const double* in, int count, double* out, int accumulate) {
  // one block of 256 threads: strided partial sums, then a fixed-order tree
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += in[i];
  const double tot = block_sum(v, red);
  if (threadIdx.x == 0) out[0] = accumulate ? out[0] + tot : tot;
}

cudaError_t launch_sum(const double* in, int count, double* out, int accumulate, cudaStream_t s) {
  k_sum<<<1, 256, 0, s>>>(in, count, out, accumulate);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_expand<float>(const void*, void*, int64_t, int, int, const GroupOp&, cudaStream_t);
template cudaError_t launch_expand<double>(const void*, void*, int64_t, int, int, const GroupOp&, cudaStream_t);
template cudaError_t launch_expand_adj<float>(const void*, const void*, void*, int64_t, int, int,
                                              const GroupOp&, double*, int*, cudaStream_t);
template cudaError_t launch_expand_adj<double>(const void*, const void*, void*, int64_t, int, int,
                                               const GroupOp&, double*, int*, cudaStream_t);
template cudaError_t launch_pauli_apply<float>(const void*, void*, int64_t, int, int, int, const uint64_t*,
                                               const uint64_t*, const double*, cudaStream_t);
template cudaError_t launch_pauli_apply<double>(const void*, void*, int64_t, int, int, int, const uint64_t*,
                                                const uint64_t*, const double*, cudaStream_t);

}  // namespace lret
