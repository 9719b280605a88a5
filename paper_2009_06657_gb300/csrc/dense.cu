// Dense k-qubit gates (k >= 3) and diagonal gates on V (Eq. 3, V <- G V with G
// acting on k of the n qubits), and their adjoints for the backward pass.
//
// Rows of V that differ only in the k target bits form a group of D = 2^k rows;
// the gate mixes the rows of each group. The matrix index of a row is
// sum_i b(q_i) 2^(k-1-i) (first listed qubit most significant), so row a of
// group g sits at x = base(g) + off[a], base(g) being g with zero bits inserted
// at the target positions and off[a] the target bits of a placed at their
// qubits. Columns are contiguous in a row, so consecutive threads (lanes) take
// consecutive columns and every row access is one coalesced run.
#include "common.cuh"
#include "kernels.h"

namespace lret {

__device__ __forceinline__ uint64_t dense_group_base(uint64_t g, const DenseOp& op) {
  // ascending positions: each insertion is at its final bit index
  for (int i = 0; i < op.k; ++i) g = insert_zero(g, op.pos[i]);
  return g;
}

// D = 8 or 16: one thread per (group, column); the D inputs stay in registers.
template <typename T, int D>
__global__ void __launch_bounds__(256) k_dense_small(const cx<T>* __restrict__ V, cx<T>* __restrict__ W,
                                                     int64_t total, int c, int ld, DenseOp op,
                                                     const cx<T>* __restrict__ U,
                                                     const uint32_t* __restrict__ off, int adjoint) {
  __shared__ cx<T> sU[D][D];
  __shared__ uint32_t soff[D];
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) {
    const int a = i / D, b = i % D;
    sU[a][b] = adjoint ? conjg(U[b * D + a]) : U[i];
  }
  for (int i = threadIdx.x; i < D; i += blockDim.x) soff[i] = off[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t g = (uint64_t)(e / c);
    const int j = (int)(e - (int64_t)g * c);
    const uint64_t base = dense_group_base(g, op);
    cx<T> v[D];
#pragma unroll
    for (int b = 0; b < D; ++b) v[b] = V[(base + soff[b]) * (uint64_t)ld + j];
#pragma unroll 1
    for (int a = 0; a < D; ++a) {  // not unrolled: the gate rows are read from shared memory
      cx<T> acc = mk<T>(0, 0);
#pragma unroll
      for (int b = 0; b < D; ++b) cfma(acc, sU[a][b], v[b]);
      W[(base + soff[a]) * (uint64_t)ld + j] = acc;
    }
  }
}

// D >= 32: a block computes a 32-row x 32-column output tile of one group,
// streaming 32 x 32 tiles of the gate and of the group's input rows through
// shared memory. Warp w owns output rows 4w..4w+3 of the tile, lane = column.
constexpr int DT = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_dense_tiled(const cx<T>* __restrict__ V, cx<T>* __restrict__ W,
                                                     int64_t groups, int c, int ld, DenseOp op,
                                                     const cx<T>* __restrict__ U,
                                                     const uint32_t* __restrict__ off, int adjoint) {
  __shared__ cx<T> sU[DT][DT + 1];
  __shared__ cx<T> sV[DT][DT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = 1 << op.k;
  const int atiles = D / DT;
  const int jtiles = (c + DT - 1) / DT;
  const int64_t ntiles = groups * atiles * jtiles;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int at = (int)(t % atiles);
    const int64_t rest = t / atiles;
    const int jt = (int)(rest % jtiles);
    const uint64_t g = (uint64_t)(rest / jtiles);
    const uint64_t base = dense_group_base(g, op);
    const int a0 = at * DT;
    const int j = jt * DT + lane;
    cx<T> acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = mk<T>(0, 0);
    for (int b0 = 0; b0 < D; b0 += DT) {
      for (int i = warp; i < DT; i += 8) {
        if (!adjoint) {
          sU[i][lane] = U[(size_t)(a0 + i) * D + b0 + lane];               // G[a0+i][b0+lane]
        } else {
          sU[lane][i] = conjg(U[(size_t)(b0 + i) * D + a0 + lane]);        // conj(G[b0+i][a0+lane])
        }
        sV[i][lane] = j < c ? V[(base + off[b0 + i]) * (uint64_t)ld + j] : mk<T>(0, 0);
      }
      __syncthreads();
#pragma unroll 8
      for (int bb = 0; bb < DT; ++bb) {
        const cx<T> v = sV[bb][lane];
#pragma unroll
        for (int i = 0; i < 4; ++i) cfma(acc[i], sU[warp * 4 + i][bb], v);
      }
      __syncthreads();
    }
    if (j < c) {
#pragma unroll
      for (int i = 0; i < 4; ++i) W[(base + off[a0 + warp * 4 + i]) * (uint64_t)ld + j] = acc[i];
    }
  }
}

// W[x][j] = d[i(x)] V[x][j] (or conj(d[i(x)]) for the adjoint). One warp per row;
// V == W is allowed (each element is read and written by one thread).
template <typename T>
__global__ void __launch_bounds__(256) k_diag(const cx<T>* V, cx<T>* W, int64_t N, int c, int ld, DiagOp op,
                                              const cx<T>* __restrict__ d, int conj) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = w0; x < N; x += nw) {
    uint32_t i = 0;
    for (int t = 0; t < op.k; ++t) i |= (uint32_t)((x >> op.q[t]) & 1) << (op.k - 1 - t);
    cx<T> f = d[i];
    if (conj) f = conjg(f);
    const cx<T>* src = V + (uint64_t)x * ld;
    cx<T>* dst = W + (uint64_t)x * ld;
    for (int j = lane; j < c; j += 32) dst[j] = cmul(f, src[j]);
  }
}

static int dense_grid(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  const int64_t cap = 152 * 8;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

template <typename T>
cudaError_t launch_dense(const void* V, void* W, int64_t N, int c, int ld, const DenseOp& op, const void* U,
                         const uint32_t* off, int adjoint, cudaStream_t s) {
  const int D = 1 << op.k;
  const int64_t groups = N / D;
  if (groups == 0 || c == 0) return cudaSuccess;
  if (D == 8) {
    const int64_t total = groups * c;
    k_dense_small<T, 8><<<dense_grid(total, 256), 256, 0, s>>>((const cx<T>*)V, (cx<T>*)W, total, c, ld, op,
                                                              (const cx<T>*)U, off, adjoint);
  } else if (D == 16) {
    const int64_t total = groups * c;
    k_dense_small<T, 16><<<dense_grid(total, 256), 256, 0, s>>>((const cx<T>*)V, (cx<T>*)W, total, c, ld, op,
                                                               (const cx<T>*)U, off, adjoint);
  } else {
    const int64_t tiles = groups * (D / DT) * ((c + DT - 1) / DT);
    int64_t blocks = tiles < 152 * 8 ? tiles : 152 * 8;
    k_dense_tiled<T><<<(int)blocks, 256, 0, s>>>((const cx<T>*)V, (cx<T>*)W, groups, c, ld, op,
                                                 (const cx<T>*)U, off, adjoint);
  }
  note_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag(const void* V, void* W, int64_t N, int c, int ld, const DiagOp& op, const void* d,
                        int conj, cudaStream_t s) {
  if (N == 0 || c == 0) return cudaSuccess;
  k_diag<T><<<dense_grid(N * 32, 256), 256, 0, s>>>((const cx<T>*)V, (cx<T>*)W, N, c, ld, op,
                                                     (const cx<T>*)d, conj);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_dense<float>(const void*, void*, int64_t, int, int, const DenseOp&, const void*,
                                         const uint32_t*, int, cudaStream_t);
template cudaError_t launch_dense<double>(const void*, void*, int64_t, int, int, const DenseOp&, const void*,
                                          const uint32_t*, int, cudaStream_t);
template cudaError_t launch_diag<float>(const void*, void*, int64_t, int, int, const DiagOp&, const void*, int,
                                        cudaStream_t);
template cudaError_t launch_diag<double>(const void*, void*, int64_t, int, int, const DiagOp&, const void*, int,
                                         cudaStream_t);

}  // namespace lret
