// Hermitian eigensolver for the truncation step (Sec. II.B): the eigenpairs of
// rho' = V' V'^dag are obtained from the small Gram matrix G = V'^dag V'
// (Theorem 1, App. B). This kernel diagonalises G by two-sided cyclic Jacobi
// with the round-robin parallel ordering: each round pairs all m indices into
// m/2 disjoint (p, q) pairs, computes one complex rotation per pair, and
// applies J^dag A J as independent 2x2 block updates (A'_PQ = J_P^dag A_PQ J_Q),
// so a whole round is one data-parallel pass over A. Eigenvectors accumulate
// as Vec <- Vec J. One thread block; A and Vec live in shared memory when they
// fit and in a global scratch slab otherwise.
//
// Jacobi is chosen for accuracy: on positive semidefinite Gram matrices it
// resolves small eigenvalues to high relative accuracy, and those decide the
// cut. After convergence the kernel sorts eigenpairs descending, chooses the
// kept count k (fixed rank or the eps rule of Sec. II.B) and does the FP64
// kept/discarded accounting.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace lret {

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

constexpr int EIG_THREADS = 1024;
constexpr int EIG_MAX_SWEEPS = 40;
constexpr size_t EIG_SMEM_LIMIT = 200 * 1024;

template <typename T>
__device__ __forceinline__ T cabs_(cx<T> z) { return sqrt(z.x * z.x + z.y * z.y); }

__device__ __forceinline__ void pair_of(int k, int r, int mp, int* p, int* q) {
  // circle method: player 0 fixed, players 1..mp-1 rotate by one each round
  const int L = mp - 1;
  if (k == 0) {
    *p = 0;
    *q = (r % L) + 1;
  } else {
    *p = ((k + r) % L) + 1;
    *q = ((mp - 1 - k + r) % L) + 1;
  }
}

template <typename T>
__global__ void __launch_bounds__(EIG_THREADS) k_eigh_jacobi(const double2* __restrict__ G, int m,
                                                             cx<T>* gwork, int use_smem,
                                                             double* __restrict__ evals,
                                                             double2* __restrict__ evecs,
                                                             EigOut* __restrict__ out, int r, double eps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T rc[128];
  __shared__ cx<T> rsig[128];
  __shared__ short rp[128], rq[128];
  __shared__ int nrot;
  __shared__ double red[32];
  __shared__ int s_rank_dummy;
  cx<T>* A = use_smem ? (cx<T>*)smem_raw : gwork;
  cx<T>* Vec = A + (size_t)m * m;
  const int tid = threadIdx.x;
  const int mm = m * m;

  // load A = G, Vec = I; trace in FP64 from G
  double tr = 0.0;
  for (int e = tid; e < mm; e += blockDim.x) {
    const int i = e / m, j = e % m;
    A[e] = from_d2<T>(G[e]);
    Vec[e] = mk<T>(i == j ? (T)1 : (T)0, (T)0);
    if (i == j) tr += G[e].x;
  }
  const double trace = block_sum(tr, red);
  __shared__ double s_trace;
  if (tid == 0) s_trace = trace;
  __syncthreads();
  const T scale = (T)fabs(s_trace) > (T)0 ? (T)fabs(s_trace) : (T)1;
  const T tol_rel = (T)Eps<T>::v;
  const T tol_abs = (T)Eps<T>::v * (T)1e-2 * scale;

  const int mp = m + (m & 1);
  const int np = mp / 2;
  int sweep = 0;
  int converged = (m <= 1);
  for (; sweep < EIG_MAX_SWEEPS && !converged; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < mp - 1; ++rnd) {
      // rotation parameters, one thread per pair
      if (tid < np) {
        int p, q;
        pair_of(tid, rnd, mp, &p, &q);
        rp[tid] = (short)p;
        rq[tid] = (short)q;
        T c = (T)1;
        cx<T> sg = mk<T>(0, 0);
        if (p < m && q < m) {
          const T a = A[p * m + p].x, d = A[q * m + q].x;
          const cx<T> b = A[p * m + q];
          const T bb = cabs_<T>(b);
          if (bb > tol_rel * sqrt(fabs(a) * fabs(d)) && bb > tol_abs) {
            const T tau = (d - a) / (2 * bb);
            const T t = (tau >= 0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
            c = (T)1 / sqrt((T)1 + t * t);
            const T s = t * c;
            sg = mk<T>(s * b.x / bb, s * b.y / bb);  // s * e^{i phi}, e^{i phi} = b / |b|
            atomicAdd(&nrot, 1);
          }
        }
        rc[tid] = c;
        rsig[tid] = sg;
      }
      __syncthreads();
      // A <- J^dag A J as 2x2 block updates; Vec <- Vec J
      const int nblk = np * np;
      for (int e = tid; e < nblk; e += blockDim.x) {
        const int P = e / np, Q = e % np;
        const int p1 = rp[P], q1 = rq[P], p2 = rp[Q], q2 = rq[Q];
        const T c1 = rc[P], c2 = rc[Q];
        const cx<T> s1 = rsig[P], s2 = rsig[Q];
        const bool vq1 = q1 < m, vq2 = q2 < m, vp1 = p1 < m, vp2 = p2 < m;
        cx<T> b00 = (vp1 && vp2) ? A[p1 * m + p2] : mk<T>(0, 0);
        cx<T> b01 = (vp1 && vq2) ? A[p1 * m + q2] : mk<T>(0, 0);
        cx<T> b10 = (vq1 && vp2) ? A[q1 * m + p2] : mk<T>(0, 0);
        cx<T> b11 = (vq1 && vq2) ? A[q1 * m + q2] : mk<T>(0, 0);
        // X = B J_Q
        const cx<T> s2c = conjg(s2);
        cx<T> x00 = csub(cscale(b00, c2), cmul(s2c, b01));
        cx<T> x01 = cadd(cmul(s2, b00), cscale(b01, c2));
        cx<T> x10 = csub(cscale(b10, c2), cmul(s2c, b11));
        cx<T> x11 = cadd(cmul(s2, b10), cscale(b11, c2));
        // B' = J_P^dag X
        const cx<T> s1c = conjg(s1);
        cx<T> n00 = csub(cscale(x00, c1), cmul(s1, x10));
        cx<T> n01 = csub(cscale(x01, c1), cmul(s1, x11));
        cx<T> n10 = cadd(cmul(s1c, x00), cscale(x10, c1));
        cx<T> n11 = cadd(cmul(s1c, x01), cscale(x11, c1));
        if (P == Q) {  // diagonal block: exact zero off-diagonal, real diagonal
          n00.y = 0; n11.y = 0;
          if (s1.x != (T)0 || s1.y != (T)0) { n01 = mk<T>(0, 0); n10 = mk<T>(0, 0); }
        }
        if (vp1 && vp2) A[p1 * m + p2] = n00;
        if (vp1 && vq2) A[p1 * m + q2] = n01;
        if (vq1 && vp2) A[q1 * m + p2] = n10;
        if (vq1 && vq2) A[q1 * m + q2] = n11;
      }
      const int nvec = m * np;
      for (int e = tid; e < nvec; e += blockDim.x) {
        const int i = e / np, Q = e % np;
        const int p2 = rp[Q], q2 = rq[Q];
        if (p2 >= m || q2 >= m) continue;
        const T c2 = rc[Q];
        const cx<T> s2 = rsig[Q];
        if (s2.x == (T)0 && s2.y == (T)0) continue;
        const cx<T> vp = Vec[i * m + p2], vq = Vec[i * m + q2];
        Vec[i * m + p2] = csub(cscale(vp, c2), cmul(conjg(s2), vq));
        Vec[i * m + q2] = cadd(cmul(s2, vp), cscale(vq, c2));
      }
      __syncthreads();
    }
    converged = (nrot == 0);
    __syncthreads();
  }
  (void)s_rank_dummy;

  // a NaN diagonal (from a non-finite input) sorts last so ranks stay a permutation
  for (int i = tid; i < m; i += blockDim.x)
    if (!(A[i * m + i].x == A[i * m + i].x)) A[i * m + i].x = -INFINITY;
  __syncthreads();
  // sort descending (rank by count; ties by index) and write FP64 results
  for (int i = tid; i < m; i += blockDim.x) {
    const T li = A[i * m + i].x;
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const T lj = A[j * m + j].x;
      rank += (lj > li) || (lj == li && j < i);
    }
    evals[rank] = (double)li;
    // accumulated rotations drift from unit norm by O(sweeps m eps); renormalise
    double nrm = 0.0;
    for (int row = 0; row < m; ++row) {
      const double2 v = to_d2(Vec[row * m + i]);
      nrm += v.x * v.x + v.y * v.y;
    }
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
    for (int row = 0; row < m; ++row) {
      const double2 v = to_d2(Vec[row * m + i]);
      evecs[(size_t)row * m + rank] = make_double2(v.x * inv, v.y * inv);
    }
  }
  __syncthreads();
  __threadfence_block();
  if (tid == 0) {
    double total = 0.0;
    for (int i = 0; i < m; ++i) total += evals[i] > 0 ? evals[i] : 0.0;
    int k;
    if (r > 0) {
      k = r < m ? r : m;
    } else {
      double cs = 0.0;
      k = m;
      for (int i = 0; i < m; ++i) {
        cs += evals[i] > 0 ? evals[i] : 0.0;
        if (cs >= (1.0 - eps) * total) { k = i + 1; break; }
      }
      if (k < 1) k = 1;
    }
    double kept = 0.0, dropped = 0.0;
    for (int i = 0; i < m; ++i) {
      const double v = evals[i] > 0 ? evals[i] : 0.0;
      if (i < k) kept += v; else dropped += v;
    }
    const double l1 = fabs(evals[0]) > 0 ? fabs(evals[0]) : 1.0;
    out->k = k;
    out->sweeps = sweep;
    out->status = converged ? 0 : 1;
    out->dropped = dropped;
    out->kept = kept;
    out->gap = k < m ? (evals[k - 1] - evals[k]) / l1 : __longlong_as_double(0x7ff0000000000000ll);
    out->trace = s_trace;
  }
}

size_t eigh_work_bytes(int m, bool fp64) {
  return 2ull * m * m * (fp64 ? sizeof(double2) : sizeof(float2));
}

template <typename T>
cudaError_t launch_eigh(const double2* G, int m, void* work, double* evals, double2* evecs, EigOut* out,
                        int r, double eps, cudaStream_t s) {
  if (m > 256) return cudaErrorInvalidValue;  // rotation tables hold 128 pairs
  const size_t need = 2ull * m * m * sizeof(cx<T>);
  const int use_smem = need <= EIG_SMEM_LIMIT;
  const size_t dyn = use_smem ? need : 0;
  if (use_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_eigh_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)EIG_SMEM_LIMIT);
    if (e != cudaSuccess) return e;
  }
  k_eigh_jacobi<T><<<1, EIG_THREADS, dyn, s>>>(G, m, (cx<T>*)work, use_smem, evals, evecs, out, r, eps);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_eigh<float>(const double2*, int, void*, double*, double2*, EigOut*, int, double,
                                        cudaStream_t);
template cudaError_t launch_eigh<double>(const double2*, int, void*, double*, double2*, EigOut*, int, double,
                                         cudaStream_t);

}  // namespace lret
