// Dense contractions of the truncation step (Sec. II.B, Theorem 1):
//   * Gram      G = X^dag X over the 2^n rows (split over row chunks; chunk
//                partials summed in FP64 in a fixed order -> deterministic);
//   * rowmat    Y = X M (project onto the kept eigenvectors, V <- V' U_r);
//   * the small FP64 matrices of the truncation adjoint.
// SIMT tiles: 64 x 64 complex outputs per 256-thread block, 4 x 4 per thread,
// operands staged through shared memory 16 rows/columns at a time.
#include "common.cuh"
#include "kernels.h"

namespace lret {

constexpr int TILE = 64;
constexpr int KSTEP = 16;

// FP32 products are accumulated in FP32 over FLUSH rows, then added into FP64
// registers, so the chunk sum carries FP64 rounding beyond 64-term runs.
template <typename T> struct Flush { static constexpr int rows = 64; };

// Pair mode (pairbit >= 0): the operand is Z = [V_0 V_1], the rows of V with
// bit `pairbit` clear and set side by side: logical row x of Z is the pair
// (x0, x0 | 2^pairbit) with x0 = x with a zero inserted at pairbit, and logical
// column i < 2*chalf is column i mod chalf of row x0 (i < chalf) or of its partner.
__device__ __forceinline__ int64_t pair_index(int64_t x, int i, int pairbit, int chalf, int ld) {
  const uint64_t x0 = insert_zero((uint64_t)x, pairbit);
  const int b = i >= chalf;
  return (int64_t)(x0 | ((uint64_t)b << pairbit)) * ld + (i - b * chalf);
}

template <typename T>
__device__ __forceinline__ void gram_body(const cx<T>* __restrict__ A, int lda, int ma,
                                          const cx<T>* __restrict__ B, int ldb, int mb, int64_t N,
                                          int64_t chunk, int tiles_j, int hermitian,
                                          double2* __restrict__ partials, int pairbit, int chalf, int bx,
                                          int by) {
  __shared__ cx<T> As[KSTEP][TILE];
  __shared__ cx<T> Bs[KSTEP][TILE];
  int ti, tj;
  if (hermitian) {
    // linear index over the upper triangle of tiles (ti <= tj)
    int lin = bx, row = 0, cnt = tiles_j;
    while (lin >= cnt) { lin -= cnt; ++row; --cnt; }
    ti = row; tj = row + lin;
  } else {
    ti = bx / tiles_j; tj = bx % tiles_j;
  }
  const int split = by;
  const int64_t x0 = (int64_t)split * chunk;
  int64_t x1 = x0 + chunk; if (x1 > N) x1 = N;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cx<T> acc[4][4];
  double2 dacc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = mk<T>(0, 0); dacc[a][b] = make_double2(0, 0); }
  int since_flush = 0;
  for (int64_t xb = x0; xb < x1; xb += KSTEP) {
    // stage KSTEP rows x TILE columns of each operand
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int idx = threadIdx.x + l * 256;
      const int rr = idx / TILE, cc = idx % TILE;
      const int64_t x = xb + rr;
      const int ia = ti * TILE + cc, ib = tj * TILE + cc;
      if (pairbit < 0) {
        As[rr][cc] = (x < x1 && ia < ma) ? A[x * lda + ia] : mk<T>(0, 0);
        Bs[rr][cc] = (x < x1 && ib < mb) ? B[x * ldb + ib] : mk<T>(0, 0);
      } else {
        As[rr][cc] = (x < x1 && ia < ma) ? A[pair_index(x, ia, pairbit, chalf, lda)] : mk<T>(0, 0);
        Bs[rr][cc] = (x < x1 && ib < mb) ? B[pair_index(x, ib, pairbit, chalf, ldb)] : mk<T>(0, 0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KSTEP; ++kk) {
      cx<T> av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfmac(acc[a][b], av[a], bv[b]);
    }
    __syncthreads();
    since_flush += KSTEP;
    if (since_flush >= Flush<T>::rows) {
      since_flush = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          dacc[a][b].x += (double)acc[a][b].x;
          dacc[a][b].y += (double)acc[a][b].y;
          acc[a][b] = mk<T>(0, 0);
        }
    }
  }
  double2* P = partials + (int64_t)split * ma * mb;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ti * TILE + ty + 16 * a, j = tj * TILE + tx + 16 * b;
      if (i < ma && j < mb)
        P[(int64_t)i * mb + j] = make_double2(dacc[a][b].x + (double)acc[a][b].x,
                                              dacc[a][b].y + (double)acc[a][b].y);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gram(const cx<T>* __restrict__ A, int lda, int ma,
                                              const cx<T>* __restrict__ B, int ldb, int mb, int64_t N,
                                              int64_t chunk, int tiles_j, int hermitian,
                                              double2* __restrict__ partials, int pairbit, int chalf) {
  gram_body<T>(A, lda, ma, B, ldb, mb, N, chunk, tiles_j, hermitian, partials, pairbit, chalf, blockIdx.x,
               blockIdx.y);
}

// sum over the splits of one entry, in a fixed order: eight independent FP64
// running sums. (FP32 partials are summed by k_gram_reduce_herm_f32x4 with
// compensated FP32 sums -- error about 2 eps of the sum of magnitudes, like an FP64
// sum of FP32 terms -- because FP64 arithmetic and conversions run at 1/62 of the
// FP32 rate here.)
__device__ __forceinline__ void split_sum(const double2* __restrict__ partials, int splits, int64_t total,
                                          int64_t e, double& sr, double& si) {
  double ar[8] = {0, 0, 0, 0, 0, 0, 0, 0}, ai[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int s = 0;
  for (; s + 8 <= splits; s += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double2 v = partials[(int64_t)(s + u) * total + e];
      ar[u] += v.x;
      ai[u] += v.y;
    }
  }
  for (int u = 0; s < splits; ++s, ++u) {
    const double2 v = partials[(int64_t)s * total + e];
    ar[u] += v.x;
    ai[u] += v.y;
  }
  sr = ((ar[0] + ar[1]) + (ar[2] + ar[3])) + ((ar[4] + ar[5]) + (ar[6] + ar[7]));
  si = ((ai[0] + ai[1]) + (ai[2] + ai[3])) + ((ai[4] + ai[5]) + (ai[6] + ai[7]));
}

__device__ __forceinline__ void neumaier(float& s, float& c, float x) {
  const float t = s + x;
  c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

// out[i][j] = sum_s partials[s][i][j]; Hermitian: fill the lower triangle from the
// upper one and make the diagonal exactly real.
template <typename P>
__global__ void k_gram_reduce(const P* __restrict__ partials, int splits, int ma, int mb, int hermitian,
                              double2* __restrict__ out) {
  const int64_t total = (int64_t)ma * mb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / mb), j = (int)(e % mb);
    if (hermitian && (i / TILE) > (j / TILE)) continue;  // tile not computed
    double sr, si;
    split_sum(partials, splits, total, e, sr, si);
    if (hermitian) {
      if (i == j) {
        out[e] = make_double2(sr, 0.0);
      } else if (i < j) {
        out[e] = make_double2(sr, si);
        out[(int64_t)j * mb + i] = make_double2(sr, -si);
      } else {
        // same tile row/col block, below the diagonal: the (j, i) element of this
        // tile is the one kept; this thread's value is its conjugate partner.
        // Skip: the i < j thread writes both.
      }
    } else {
      out[e] = make_double2(sr, si);
    }
  }
}

cudaError_t launch_gram_reduce_herm(const double2* partials, int splits, int m, double2* out, cudaStream_t s) {
  const int64_t total = (int64_t)m * m;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_gram_reduce<double2><<<blocks, 256, 0, s>>>(partials, splits, m, m, 1, out);
  note_launches(1);
  return cudaGetLastError();
}

// The Hermitian reduction of FP32 partials with four threads per element: thread
// sub of a group of four sums splits sub, sub + 4, ... (compensated), and the four
// (sum, compensation) pairs are added in a fixed order, so the result does not
// depend on scheduling. Four times the threads of one-thread-per-element, each with a
// quarter of the dependent loads.
__global__ void k_gram_reduce_herm_f32x4(const float2* __restrict__ partials, int splits, int m,
                                         double2* __restrict__ out) {
  const int64_t total = (int64_t)m * m;
  const int lane = threadIdx.x & 31, sub = lane & 3;
  // a warp takes 8 consecutive elements per iteration (warp-uniform loop: the
  // shuffles below need every lane)
  const int64_t wstep = (((int64_t)gridDim.x * blockDim.x) >> 5) * 8;
  for (int64_t gb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 8; gb < total; gb += wstep) {
    const int64_t g = gb + (lane >> 2);
    const int i = (int)(g / m), j = (int)(g % m);
    const bool keep = g < total && (i / TILE) <= (j / TILE) && i <= j;  // computed tile, upper triangle
    float s_r = 0.f, c_r = 0.f, s_i = 0.f, c_i = 0.f;
    if (keep) {
      int s = sub;
      for (; s + 12 < splits; s += 16) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = partials[(int64_t)(s + 4 * u) * total + g];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          neumaier(s_r, c_r, v[u].x);
          neumaier(s_i, c_i, v[u].y);
        }
      }
      for (; s < splits; s += 4) {
        const float2 v = partials[(int64_t)s * total + g];
        neumaier(s_r, c_r, v.x);
        neumaier(s_i, c_i, v.y);
      }
    }
    // (sum + compensation) of the four threads, in the order 0 + 1, 2 + 3, then both
    double r = (double)s_r + (double)c_r, im = (double)s_i + (double)c_i;
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    im += __shfl_xor_sync(0xffffffffu, im, 1);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    im += __shfl_xor_sync(0xffffffffu, im, 2);
    if (keep && sub == 0) {
      if (i == j) {
        out[g] = make_double2(r, 0.0);
      } else {
        out[g] = make_double2(r, im);
        out[(int64_t)j * m + i] = make_double2(r, -im);
      }
    }
  }
}

cudaError_t launch_gram_reduce_herm_f32(const float2* partials, int splits, int m, double2* out, cudaStream_t s) {
  const int64_t total = (int64_t)m * m;
  int blocks = (int)((4 * total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_gram_reduce_herm_f32x4<<<blocks, 256, 0, s>>>(partials, splits, m, out);
  note_launches(1);
  return cudaGetLastError();
}

int gram_splits(int64_t N, int ma, int mb) {
  const int ti = (ma + TILE - 1) / TILE, tj = (mb + TILE - 1) / TILE;
  const int tiles = ti * tj;
  int splits = (int)((4 * 152 + tiles - 1) / tiles);
  const int64_t max_by_rows = (N + 255) / 256;  // at least 256 rows per chunk
  if (splits > max_by_rows) splits = (int)max_by_rows;
  if (splits > 1024) splits = 1024;
  if (splits < 1) splits = 1;
  return splits;
}

template <typename T>
cudaError_t launch_gram(const void* A, int lda, int ma, const void* B, int ldb, int mb, int64_t N,
                        bool hermitian, double2* partials, int splits, double2* out, cudaStream_t s,
                        int pairbit, int chalf) {
  const int ti = (ma + TILE - 1) / TILE, tj = (mb + TILE - 1) / TILE;
  const int tiles = hermitian ? ti * (ti + 1) / 2 : ti * tj;
  int64_t chunk = (N + splits - 1) / splits;
  chunk = ((chunk + KSTEP - 1) / KSTEP) * KSTEP;
  dim3 grid(tiles, splits);
  k_gram<T><<<grid, 256, 0, s>>>((const cx<T>*)A, lda, ma, (const cx<T>*)B, ldb, mb, N, chunk, tj,
                                 hermitian ? 1 : 0, partials, pairbit, chalf);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)ma * mb;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_gram_reduce<double2><<<blocks, 256, 0, s>>>(partials, splits, ma, mb, hermitian ? 1 : 0, out);
  note_launches(1);
  return cudaGetLastError();
}

// Y[x][j] = sum_i A1[x][i] M1[i][j] + sum_i A2[x][i] M2[i][j]
// Pair mode (pairbit >= 0): rows are pairs as in k_gram, A1 has 2*chalf
// logical columns and Y has p = 2*phalf logical columns split the same way.
template <typename T>
__device__ __forceinline__ void rowmat_body(const cx<T>* __restrict__ A1, int lda1, int k1,
                                            const double2* __restrict__ M1, int ldm1,
                                            const cx<T>* __restrict__ A2, int lda2, int k2,
                                            const double2* __restrict__ M2, int ldm2,
                                            cx<T>* __restrict__ Y, int ldy, int p, int64_t N,
                                            int pairbit, int chalf, int phalf, int bx, int by) {
  __shared__ cx<T> As[TILE][KSTEP + 1];
  __shared__ cx<T> Ms[KSTEP][TILE];
  const int64_t xbase = (int64_t)bx * TILE;
  const int jbase = by * TILE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cx<T> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk<T>(0, 0);
  for (int src = 0; src < 2; ++src) {
    const cx<T>* A = src == 0 ? A1 : A2;
    const double2* M = src == 0 ? M1 : M2;
    const int lda = src == 0 ? lda1 : lda2, kk_n = src == 0 ? k1 : k2, ldm = src == 0 ? ldm1 : ldm2;
    if (A == nullptr || kk_n <= 0) continue;
    for (int ib = 0; ib < kk_n; ib += KSTEP) {
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int idx = threadIdx.x + l * 256;
        // A tile: TILE rows x KSTEP cols
        const int rr = idx / KSTEP, cc = idx % KSTEP;
        const int64_t x = xbase + rr;
        const int i = ib + cc;
        if (pairbit < 0)
          As[rr][cc] = (x < N && i < kk_n) ? A[x * lda + i] : mk<T>(0, 0);
        else
          As[rr][cc] = (x < N && i < kk_n) ? A[pair_index(x, i, pairbit, chalf, lda)] : mk<T>(0, 0);
        // M tile: KSTEP rows x TILE cols
        const int mr = idx / TILE, mc = idx % TILE;
        const int mi = ib + mr, mj = jbase + mc;
        Ms[mr][mc] = (mi < kk_n && mj < p) ? from_d2<T>(M[(int64_t)mi * ldm + mj]) : mk<T>(0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KSTEP; ++kk) {
        cx<T> av[4], mv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[ty + 16 * a][kk];
#pragma unroll
        for (int b = 0; b < 4; ++b) mv[b] = Ms[kk][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], mv[b]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t x = xbase + ty + 16 * a;
      const int j = jbase + tx + 16 * b;
      if (x < N && j < p) {
        if (pairbit < 0) Y[x * ldy + j] = acc[a][b];
        else Y[pair_index(x, j, pairbit, phalf, ldy)] = acc[a][b];
      }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rowmat(const cx<T>* __restrict__ A1, int lda1, int k1,
                                                const double2* __restrict__ M1, int ldm1,
                                                const cx<T>* __restrict__ A2, int lda2, int k2,
                                                const double2* __restrict__ M2, int ldm2,
                                                cx<T>* __restrict__ Y, int ldy, int p, int64_t N,
                                                int pairbit, int chalf, int phalf) {
  rowmat_body<T>(A1, lda1, k1, M1, ldm1, A2, lda2, k2, M2, ldm2, Y, ldy, p, N, pairbit, chalf, phalf, blockIdx.x,
                 blockIdx.y);
}

template <typename T>
cudaError_t launch_rowmat(const void* A1, int lda1, int k1, const double2* M1, int ldm1,
                          const void* A2, int lda2, int k2, const double2* M2, int ldm2,
                          void* Y, int ldy, int p, int64_t N, cudaStream_t s, int pairbit, int chalf,
                          int phalf) {
  if (N == 0 || p == 0) return cudaSuccess;
  dim3 grid((unsigned)((N + TILE - 1) / TILE), (unsigned)((p + TILE - 1) / TILE));
  k_rowmat<T><<<grid, 256, 0, s>>>((const cx<T>*)A1, lda1, k1, M1, ldm1, (const cx<T>*)A2, lda2, k2, M2,
                                   ldm2, (cx<T>*)Y, ldy, p, N, pairbit, chalf, phalf);
  note_launches(1);
  return cudaGetLastError();
}

// ---- structured truncation helpers (FP64, small) -----------------------------
// G'[al*c + i][be*c + j] = sum_{b,b'} Q[al][be][b][b'] S[b*c + i][b'*c + j]
__global__ void k_assemble_gram(const double2* __restrict__ S, int c, int K, PairQ q, double2* __restrict__ Gp) {
  const int m = K * c;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int row = e / m, col = e % m;
  const int al = row / c, i = row % c, be = col / c, j = col % c;
  const int ld = 2 * c;
  double2 acc = make_double2(0, 0);
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int bp = 0; bp < 2; ++bp)
      cfma(acc, q.Q[al][be][b][bp], S[(int64_t)(b * c + i) * ld + bp * c + j]);
  if (row == col) acc.y = 0.0;
  Gp[e] = acc;
}

// D[b*c + i][a*k + j] = sum_al M[al][a][b] U[al*c + i][j]   (U: m x m, leading dim m)
__global__ void k_build_proj(const double2* __restrict__ U, int c, int K, int k, PairQ q,
                             double2* __restrict__ D) {
  const int rows = 2 * c, cols = 2 * k, m = K * c;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int r = e / cols, cl = e % cols;
  const int b = r / c, i = r % c, a = cl / k, j = cl % k;
  double2 acc = make_double2(0, 0);
  for (int al = 0; al < K; ++al) cfma(acc, q.M[al][a][b], U[(int64_t)(al * c + i) * m + j]);
  D[e] = acc;
}

// C (M x N) = op(A) B with op(A) = A (M x K, row stride lda) or A^dag (A stored K x M).
// Small products of the deferred pair projection (M, N, K <= 512) in FP64 (the
// composed coefficients feed every later truncation on the qubit, so their rounding
// accumulates; FP32 products measurably loosened a 480-truncation run). ZT x ZT
// output tiles, K staged ZT * ZK at a time in shared memory and split over ZK thread
// groups whose partial sums are added in a fixed order.
constexpr int ZT = 8;  // 8 x 8 output tiles: a 128 x 128 product spreads over 256 blocks (all SMs)
constexpr int ZK = 4;  // K split four ways inside a block (four times the warps, a quarter of the chain)
template <typename TC>
__global__ void __launch_bounds__(ZT * ZT * ZK) k_zgemm_small(const double2* __restrict__ A, int lda, int adj,
                                                              const double2* __restrict__ B, int ldb,
                                                              double2* __restrict__ C, int ldc, int M, int N,
                                                              int K) {
  constexpr int KS = ZT * ZK;        // K slice staged per step
  __shared__ cx<TC> sA[ZT][KS + 1];  // sA[i][l] = op(A)[i0 + i][l0 + l]
  __shared__ cx<TC> sB[KS][ZT + 1];  // sB[l][j] = B[l0 + l][j0 + j]
  __shared__ cx<TC> red[ZK][ZT][ZT];
  const int tid = threadIdx.x;
  const int tx = tid % ZT, ty = (tid / ZT) % ZT, kg = tid / (ZT * ZT);
  const int i0 = blockIdx.y * ZT, j0 = blockIdx.x * ZT;
  cx<TC> acc = mk<TC>(0, 0);
  for (int l0 = 0; l0 < K; l0 += KS) {
    {
      const int i = tid / KS, l = tid % KS;  // op(A) tile: ZT rows x KS columns, one per thread
      const int gi = i0 + i, gl = l0 + l;
      double2 a = make_double2(0, 0);
      if (gi < M && gl < K) a = adj ? conjg(A[(int64_t)gl * lda + gi]) : A[(int64_t)gi * lda + gl];
      sA[i][l] = mk<TC>((TC)a.x, (TC)a.y);
      const int lb = tid / ZT, j = tid % ZT;  // B tile: KS rows x ZT columns, one per thread
      const int glb = l0 + lb, gj = j0 + j;
      double2 b = make_double2(0, 0);
      if (glb < K && gj < N) b = B[(int64_t)glb * ldb + gj];
      sB[lb][j] = mk<TC>((TC)b.x, (TC)b.y);
    }
    __syncthreads();
#pragma unroll
    for (int l = kg * ZT; l < kg * ZT + ZT; ++l) cfma(acc, sA[ty][l], sB[l][tx]);
    __syncthreads();
  }
  red[kg][ty][tx] = acc;
  __syncthreads();
  if (kg == 0) {
    cx<TC> r = red[0][ty][tx];
#pragma unroll
    for (int q = 1; q < ZK; ++q) r = cadd(r, red[q][ty][tx]);  // fixed order
    const int i = i0 + ty, j = j0 + tx;
    if (i < M && j < N) C[(int64_t)i * ldc + j] = make_double2((double)r.x, (double)r.y);
  }
}

cudaError_t launch_zgemm_small(const double2* A, int lda, int adj, const double2* B, int ldb, double2* C, int ldc,
                               int M, int N, int K, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((N + ZT - 1) / ZT, (M + ZT - 1) / ZT);
  k_zgemm_small<double><<<grid, ZT * ZT * ZK, 0, s>>>(A, lda, adj, B, ldb, C, ldc, M, N, K);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_assemble_gram(const double2* S, int c, int K, const PairQ& q, double2* Gp, cudaStream_t s) {
  const int m = K * c;
  k_assemble_gram<<<(m * m + 255) / 256, 256, 0, s>>>(S, c, K, q, Gp);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_build_proj(const double2* U, int c, int K, int k, const PairQ& q, double2* D, cudaStream_t s) {
  const int n = 4 * c * k;
  k_build_proj<<<(n + 255) / 256, 256, 0, s>>>(U, c, K, k, q, D);
  note_launches(1);
  return cudaGetLastError();
}

// ---- batched structured truncation (many circuits per launch) ---------------
// Each launch serves a list of tasks (one per circuit); blocks map to tasks
// through a prefix table of per-task block counts.
__device__ __forceinline__ int task_of_block(const int* __restrict__ bstart, int ntasks, int b) {
  int lo = 0, hi = ntasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_pair_gram_batch(const TruncTask* __restrict__ tasks,
                                                         const int* __restrict__ bstart, int ntasks) {
  const int t = task_of_block(bstart, ntasks, blockIdx.x);
  const TruncTask& tk = tasks[t];
  const int l = blockIdx.x - bstart[t];
  const int tiles = tk.tiles;
  const int c2 = 2 * tk.c;
  gram_body<T>((const cx<T>*)tk.V, tk.ld, c2, (const cx<T>*)tk.V, tk.ld, c2, tk.N2, tk.chunk,
               (c2 + TILE - 1) / TILE, 1, tk.partials, tk.q, tk.c, l % tiles, l / tiles);
}

// S = the pair Gram summed over splits, in split order (FP64 partials of the SIMT Gram, upper
// triangle by TILE blocks; or FP32 partials of the tensor-core Gram, upper triangle by 64-row
// blocks); only the blocks the Gram computed are written
__global__ void __launch_bounds__(256) k_split_sum_batch(const TruncTask* __restrict__ tasks) {
  const TruncTask& tk = tasks[blockIdx.y];
  const int c2 = 2 * tk.c;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c2 * c2) return;
  const int si = e / c2, sj = e % c2;
  const int blk = tk.tc ? 64 : TILE;
  if (si / blk > sj / blk) return;
  const int64_t stride = (int64_t)c2 * c2;
  double sr = 0.0, sim = 0.0;
  if (tk.tc) {
    const float2* pf = reinterpret_cast<const float2*>(tk.partials);
    for (int sp = 0; sp < tk.splits; ++sp) {
      const float2 v = pf[sp * stride + e];
      sr += (double)v.x; sim += (double)v.y;
    }
  } else {
    for (int sp = 0; sp < tk.splits; ++sp) {
      const double2 v = tk.partials[sp * stride + e];
      sr += v.x; sim += v.y;
    }
  }
  tk.S[e] = make_double2(sr, sim);
}

// G'[al c + i][be c + j] = sum_{b,b'} (M_al^dag M_be)_{bb'} S[b c + i][b' c + j]
__global__ void __launch_bounds__(256) k_reduce_assemble_batch(const TruncTask* __restrict__ tasks) {
  const TruncTask& tk = tasks[blockIdx.y];
  const int c = tk.c, K = tk.K, m = K * c, c2 = 2 * c;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int row = e / m, col = e % m;
  const int al = row / c, i = row % c, be = col / c, j = col % c;
  double2 acc = make_double2(0, 0);
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int bp = 0; bp < 2; ++bp) {
      const int si = b * c + i, sj = bp * c + j;
      const int blk = tk.tc ? 64 : TILE;
      const bool upper = (si / blk) <= (sj / blk);  // blocks computed by the Gram
      const int64_t idx = upper ? (int64_t)si * c2 + sj : (int64_t)sj * c2 + si;
      const double2 v = tk.S[idx];
      const double sr = v.x, sim = upper ? v.y : -v.y;
      double2 q = make_double2(0, 0);
#pragma unroll
      for (int a = 0; a < 2; ++a) cfmac(q, tk.M[al][a][b], tk.M[be][a][bp]);
      cfma(acc, q, make_double2(sr, sim));
    }
  if (row == col) acc.y = 0.0;
  if (tk.tcs) {  // the circuit's state is s V (trace anchoring of a tensor-core projection)
    const double s2 = tk.tcs[1] * tk.tcs[1];
    acc = make_double2(acc.x * s2, acc.y * s2);
  }
  tk.G[e] = acc;
}

// D[b c + i][a k + j] = sum_al M[al][a][b] U[al c + i][j]
__global__ void __launch_bounds__(256) k_build_proj_batch(const TruncTask* __restrict__ tasks) {
  const TruncTask& tk = tasks[blockIdx.y];
  const int c = tk.c, k = tk.k, K = tk.K, m = K * c;
  const int cols = 2 * k;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * c * cols) return;
  const int r = e / cols, cl = e % cols;
  const int b = r / c, i = r % c, a = cl / k, j = cl % k;
  double2 acc = make_double2(0, 0);
  for (int al = 0; al < K; ++al) cfma(acc, tk.M[al][a][b], tk.evecs[(int64_t)(al * c + i) * m + j]);
  if (tk.tcs) acc = make_double2(acc.x * tk.tcs[1], acc.y * tk.tcs[1]);  // and its projection s [V_0 V_1] D
  tk.D[e] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_pair_rowmat_batch(const TruncTask* __restrict__ tasks,
                                                           const int* __restrict__ bstart, int ntasks) {
  const int t = task_of_block(bstart, ntasks, blockIdx.x);
  const TruncTask& tk = tasks[t];
  const int l = blockIdx.x - bstart[t];
  const int coltiles = (2 * tk.k + TILE - 1) / TILE;
  rowmat_body<T>((const cx<T>*)tk.V, tk.ld, 2 * tk.c, tk.D, 2 * tk.k, nullptr, 0, 0, nullptr, 0, (cx<T>*)tk.W,
                 tk.ld, 2 * tk.k, tk.N2, tk.q, tk.c, tk.k, l / coltiles, l % coltiles);
}

__global__ void k_accum_batch(const TruncTask* __restrict__ tasks, int ntasks) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntasks) return;
  const TruncTask& tk = tasks[t];
  tk.acc[0] += tk.eo->dropped;
  tk.acc[1] = tk.eo->gap;
  if ((double)tk.eo->status > tk.acc[2]) tk.acc[2] = (double)tk.eo->status;
  tk.acc[3] += 1.0;
  if (tk.tcs) tk.tcs[1] = 1.0;  // the scale is folded into this projection (a tensor-core one sets a new one)
}

template <typename T>
cudaError_t launch_trunc_batch_gemms(const TruncTask* tasks, const int* gram_bstart, int gram_blocks,
                                     const int* proj_bstart, int proj_blocks, int ntasks, int max_m2,
                                     int max_d, int phase, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (phase == 0) {
    if (gram_blocks > 0) {
      k_pair_gram_batch<T><<<gram_blocks, 256, 0, s>>>(tasks, gram_bstart, ntasks);
      note_launches(1);
    }
    k_split_sum_batch<<<dim3((max_m2 + 255) / 256, ntasks), 256, 0, s>>>(tasks);  // max_m2 >= (2c)^2 too
    k_reduce_assemble_batch<<<dim3((max_m2 + 255) / 256, ntasks), 256, 0, s>>>(tasks);
    note_launches(2);
  } else {
    k_build_proj_batch<<<dim3((max_d + 255) / 256, ntasks), 256, 0, s>>>(tasks);
    note_launches(1);
    if (proj_blocks > 0) {
      k_pair_rowmat_batch<T><<<proj_blocks, 256, 0, s>>>(tasks, proj_bstart, ntasks);
      note_launches(1);
    }
    k_accum_batch<<<(ntasks + 127) / 128, 128, 0, s>>>(tasks, ntasks);
    note_launches(1);
  }
  return cudaGetLastError();
}

int trunc_tiles(int c) {
  const int t = (2 * c + TILE - 1) / TILE;
  return t * (t + 1) / 2;
}
int64_t trunc_chunk(int64_t N2, int splits) {
  int64_t chunk = (N2 + splits - 1) / splits;
  return ((chunk + KSTEP - 1) / KSTEP) * KSTEP;
}
int trunc_proj_blocks(int64_t N2, int k) {
  return (int)(((N2 + TILE - 1) / TILE) * ((2 * k + TILE - 1) / TILE));
}

template cudaError_t launch_trunc_batch_gemms<float>(const TruncTask*, const int*, int, const int*, int, int, int,
                                                     int, int, cudaStream_t);
template cudaError_t launch_trunc_batch_gemms<double>(const TruncTask*, const int*, int, const int*, int, int, int,
                                                      int, int, cudaStream_t);

// ---- truncation adjoint, small FP64 matrices (m <= 256) ----------------------
// FA[j][i] = F(lam_i - lam_{k+j}) * sum_l conj(U[l][k+j]) C[l][i]   (j < m-k, i < k)
__global__ void k_tadj_fa(const double2* __restrict__ C, const double2* __restrict__ U,
                          const double* __restrict__ lam, int m, int k, double2* __restrict__ FA) {
  const int d = m - k;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d * k) return;
  const int j = e / k, i = e % k;
  double2 acc = make_double2(0, 0);
  for (int l = 0; l < m; ++l) cfmac(acc, U[(int64_t)l * m + k + j], C[(int64_t)l * k + i]);
  const double l1 = fabs(lam[0]) > 0 ? fabs(lam[0]) : 1.0;
  const double delta = lam[i] - lam[k + j];
  const double eta = 1e-12 * l1;
  // A discarded eigenvalue within the FP64 eigensolve's resolution of zero (4 m u64
  // lambda_1) is a null direction of V' (V' u_j = 0 in exact arithmetic), and the pair's
  // term, carried by V' u_j, vanishes; left in, the rounding-level |V' u_j| ~ sqrt(lambda_j)
  // would be amplified by 1 / lambda_i for a small kept lambda_i.
  const bool null_j = fabs(lam[k + j]) <= 4.0 * m * 1.1102230246251565e-16 * l1;
  const double f = null_j ? 0.0 : delta / (delta * delta + eta * eta);  // 1/delta, regularised at ties
  FA[e] = make_double2(acc.x * f, acc.y * f);
}

// T1[a][i] = sum_j U[a][k+j] FA[j][i]   (a < m, i < k)
__global__ void k_tadj_t1(const double2* __restrict__ U, const double2* __restrict__ FA, int m, int k,
                          double2* __restrict__ T1) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int a = e / k, i = e % k;
  double2 acc = make_double2(0, 0);
  for (int j = 0; j < m - k; ++j) cfma(acc, U[(int64_t)a * m + k + j], FA[(int64_t)j * k + i]);
  T1[e] = acc;
}

// B[a][b] = sum_i T1[a][i] conj(U[b][i]);  Mcat[k + a][b] = B[a][b] + conj(B[b][a]);
// Mcat[i][b] = conj(U[b][i]) for i < k.
__global__ void k_tadj_mcat(const double2* __restrict__ T1, const double2* __restrict__ U, int m, int k,
                            double2* __restrict__ Mcat) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < k * m) {
    const int i = e / m, b = e % m;
    Mcat[e] = conjg(U[(int64_t)b * m + i]);
  }
  if (e >= m * m) return;
  const int a = e / m, b = e % m;
  double2 bab = make_double2(0, 0), bba = make_double2(0, 0);
  for (int i = 0; i < k; ++i) {
    cfma(bab, T1[(int64_t)a * k + i], conjg(U[(int64_t)b * m + i]));
    cfma(bba, T1[(int64_t)b * k + i], conjg(U[(int64_t)a * m + i]));
  }
  Mcat[(int64_t)(k + a) * m + b] = cadd(bab, conjg(bba));
}

cudaError_t launch_trunc_adj_small(const double2* C, const double2* U, const double* lam, int m, int k,
                                   double2* FA, double2* T1, double2* Mcat, cudaStream_t s) {
  const int d = m - k;
  if (d > 0) {
    k_tadj_fa<<<(d * k + 127) / 128, 128, 0, s>>>(C, U, lam, m, k, FA);
    note_launches(1);
    k_tadj_t1<<<(m * k + 127) / 128, 128, 0, s>>>(U, FA, m, k, T1);
    note_launches(1);
  } else {
    cudaMemsetAsync(T1, 0, sizeof(double2) * (size_t)m * k, s);
  }
  k_tadj_mcat<<<(m * m + 127) / 128, 128, 0, s>>>(T1, U, m, k, Mcat);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_gram<float>(const void*, int, int, const void*, int, int, int64_t, bool, double2*,
                                        int, double2*, cudaStream_t, int, int);
template cudaError_t launch_gram<double>(const void*, int, int, const void*, int, int, int64_t, bool, double2*,
                                         int, double2*, cudaStream_t, int, int);
template cudaError_t launch_rowmat<float>(const void*, int, int, const double2*, int, const void*, int, int,
                                          const double2*, int, void*, int, int, int64_t, cudaStream_t, int, int,
                                          int);
template cudaError_t launch_rowmat<double>(const void*, int, int, const double2*, int, const void*, int, int,
                                           const double2*, int, void*, int, int, int64_t, cudaStream_t, int, int,
                                           int);

}  // namespace lret
