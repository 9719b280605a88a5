// FP64 refinement of the kept eigenvectors of a truncation (Sec. II.B: rho is
// cut to the span of the leading eigenvectors of the Gram matrix G = V'^dag V',
// Theorem 1 of App. B) after an eigensolve in FP32 arithmetic that returned
// every eigenvector.
//
// The truncated rho = V' P V'^dag depends on the kept eigenvectors only through
// the projector P onto their span, so only the components of the kept vectors
// along the discarded ones need FP64 accuracy; rotations inside the kept set do
// not matter, their orthonormality does. One refinement step, in the spirit of
// Ogita and Aishima's refinement of a symmetric eigendecomposition by matrix
// products (Japan J. Indust. Appl. Math. 35, 2018), restricted to the kept
// columns X (m x k) and using the FP32 discarded vectors Xd as the basis of
// the complement:
//   W = G X, R = X^dag X                          (FP64; the only FP64 products)
//   mu_i = Re(x_i^dag w_i) / R_ii                 (Rayleigh quotients)
//   res_i = w_i - mu_i x_i                        (FP64; small, ~u32 |G|)
//   e_ji = (xd_j^dag res_i) / (mu_i - lam_j)      (discarded j, lam_j its FP32
//                                                  eigenvalue; an FP32 product of the
//                                                  small residual suffices)
//   X <- X (I - (R - I) / 2) + Xd E               (first-order orthonormalisation
//                                                  and the complement correction)
// A kept/discarded pair closer than the FP32 solve resolves (|mu_i - lam_j| <=
// 2^-24 |mu_1|), or whose correction is not small (|e_ji| > 1/2), is left alone:
// there the FP32 basis cannot tell the two apart (and any basis of a tied cluster
// is a correct truncation). One step takes the kept subspace from the FP32 solve's
// accuracy to FP64 accuracy where the FP32 discarded basis is accurate; where it is
// not (clusters the FP32 solve did not resolve, rank-deficient Gram matrices) the
// step can leave the kept vectors slightly non-orthonormal, and a second step would
// amplify that. So the runtime runs one step (iters = 1) followed by three FP64
// orthonormalisation steps X <- X (I - (X^dag X - I) / 2), each of which squares
// the deviation from orthonormality. The kept eigenvalues are the FP64 Rayleigh
// quotients of the refined vectors (formed with G X in the last of those steps).
// Kept vectors are not rotated among themselves (that leaves rho unchanged), so a
// kept eigenvalue inside a cluster the FP32 solve did not resolve (spread below
// about u32 |G|) is the Rayleigh quotient of a vector of that cluster; the sum of
// the kept eigenvalues, trace(X^dag G X), is accurate in FP64 either way. The kept
// eigenvalues become the FP64 Rayleigh quotients and the discarded mass
// trace(G) - their sum.
#include "common.cuh"
#include "kernels.h"

namespace lret {

namespace {

constexpr int RT = 16;   // output tile (RT x RT), one output per thread
constexpr int RK = 32;   // K chunk staged in shared memory
constexpr int RF_SPLITS_MAX = 8;
constexpr int RF_ORTHO = 3;  // FP64 orthonormalisation steps after the corrections

// P[s] = [G ; X^dag] X over the K chunk s (rows r < m: G[r][:], rows m + i: conj(X[:, i])),
// output rows from row0 (0: both products; m: X^dag X only).
__global__ void __launch_bounds__(RT* RT)
    k_rf_gemm64(const double2* __restrict__ G, int m, const double2* __restrict__ X, int ldx,
                const EigOut* __restrict__ eo, int kmax, int row0, double2* __restrict__ P) {
  const int k = eo->k < kmax ? eo->k : kmax;
  const int r0 = row0 + blockIdx.y * RT, c0 = blockIdx.x * RT, s = blockIdx.z;
  if (c0 >= k || r0 >= m + k) return;
  __shared__ double2 As[RT][RK + 1];
  __shared__ double2 Bs[RK][RT + 1];
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  const int kb = s * RK;
  for (int e = tid; e < RT * RK; e += RT * RT) {
    const int rr = e / RK, kk = e % RK;
    const int row = r0 + rr, kg = kb + kk;
    double2 a = make_double2(0.0, 0.0);
    if (kg < m) {
      if (row < m) a = G[(size_t)row * m + kg];
      else if (row < m + k) a = conjg(X[(size_t)kg * ldx + (row - m)]);
    }
    As[rr][kk] = a;
  }
  for (int e = tid; e < RK * RT; e += RT * RT) {
    const int kk = e / RT, cc = e % RT;
    const int kg = kb + kk, col = c0 + cc;
    Bs[kk][cc] = (kg < m && col < k) ? X[(size_t)kg * ldx + col] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  double2 acc = make_double2(0.0, 0.0);
#pragma unroll 8
  for (int kk = 0; kk < RK; ++kk) cfma(acc, As[ty][kk], Bs[kk][tx]);
  const int row = r0 + ty, col = c0 + tx;
  if (row < m + k && col < k) P[((size_t)s * (m + kmax) + row) * kmax + col] = acc;
}

// One block per kept column i: W[:, i] and R[:, i] from the split partials (fixed
// order), mu_i, res_i = w_i - mu_i x_i (stored in FP32), R (FP64).
__global__ void __launch_bounds__(256)
    k_rf_res(const double2* __restrict__ P, int splits, int m, const double2* __restrict__ X, int ldx,
             const EigOut* __restrict__ eo, int kmax, double* __restrict__ mu, double2* __restrict__ R,
             float2* __restrict__ Res) {
  const int k = eo->k < kmax ? eo->k : kmax;
  const int i = blockIdx.x;
  if (i >= k) return;
  __shared__ double red[32];
  __shared__ double s_mu;
  const int t = threadIdx.x;
  const size_t sstride = (size_t)(m + kmax) * kmax;
  double2 w = make_double2(0.0, 0.0), x = make_double2(0.0, 0.0);
  double q = 0.0;
  if (t < m) {
    for (int s = 0; s < splits; ++s) w = cadd(w, P[s * sstride + (size_t)t * kmax + i]);
    x = X[(size_t)t * ldx + i];
    q = x.x * w.x + x.y * w.y;  // Re(conj(x) w)
  }
  if (t < k) {
    double2 rv = make_double2(0.0, 0.0);
    for (int s = 0; s < splits; ++s) rv = cadd(rv, P[s * sstride + (size_t)(m + t) * kmax + i]);
    R[(size_t)t * kmax + i] = rv;
  }
  q = block_sum(q, red);
  if (t == 0) {
    double nrm = 0.0;
    for (int s = 0; s < splits; ++s) nrm += P[s * sstride + (size_t)(m + i) * kmax + i].x;
    const double v = nrm > 0.0 ? q / nrm : 0.0;
    s_mu = v;
    mu[i] = v;
  }
  __syncthreads();
  if (t < m) {
    const double2 rs = csub(w, cscale(x, s_mu));
    Res[(size_t)t * kmax + i] = make_float2((float)rs.x, (float)rs.y);
  }
}

// A = Xall^dag Res (m x k): x_j^dag res_i for every column j of the FP32 solve, an
// FP32 product (res is small).
__global__ void __launch_bounds__(RT* RT)
    k_rf_proj(const double2* __restrict__ Xall, int m, const float2* __restrict__ Res,
              const EigOut* __restrict__ eo, int kmax, float2* __restrict__ A) {
  const int k = eo->k < kmax ? eo->k : kmax;
  const int r0 = blockIdx.y * RT, c0 = blockIdx.x * RT;
  if (c0 >= k || r0 >= m) return;
  __shared__ float2 As[RT][RK + 1];  // conj(Xall[kg][row])
  __shared__ float2 Bs[RK][RT + 1];  // Res[kg][col]
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  float2 acc = make_float2(0.f, 0.f);
  for (int kb = 0; kb < m; kb += RK) {
    for (int e = tid; e < RT * RK; e += RT * RT) {
      const int rr = e % RT, kk = e / RT;
      const int kg = kb + kk, rw = r0 + rr;
      float2 a = make_float2(0.f, 0.f);
      if (kg < m && rw < m) {
        const double2 v = Xall[(size_t)kg * m + rw];
        a = make_float2((float)v.x, -(float)v.y);
      }
      As[rr][kk] = a;
    }
    for (int e = tid; e < RK * RT; e += RT * RT) {
      const int kk = e / RT, cc = e % RT;
      const int kg = kb + kk, cl = c0 + cc;
      Bs[kk][cc] = (kg < m && cl < k) ? Res[(size_t)kg * kmax + cl] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < RK; ++kk) cfma(acc, As[ty][kk], Bs[kk][tx]);
    __syncthreads();
  }
  const int row = r0 + ty, col = c0 + tx;
  if (row < m && col < k) A[(size_t)row * kmax + col] = acc;
}

// Whether the complement correction of kept vector i along discarded vector j is
// applied, and its value e = a / den: not for a kept vector whose eigenvalue is below
// the FP32 solve's noise floor (a numerically null direction: it does not change rho),
// not for eigenvalue differences within that solve's resolution (unit roundoff x
// lambda_1: there the FP32 basis and numerators are noise), and not where the
// correction is not small (|e| > 1/2).
__device__ __forceinline__ bool rf_pair(int j, int i, const float2* __restrict__ A, const double* __restrict__ mu,
                                        const double* __restrict__ lam, int kmax, double& ex, double& ey,
                                        double& den) {
  const double res = 5.9604644775390625e-8 * fabs(mu[0]);
  if (!(fabs(mu[i]) > res)) return false;
  den = mu[i] - lam[j];
  if (!(fabs(den) > res)) return false;
  const float2 a = A[(size_t)j * kmax + i];
  ex = (double)a.x / den;
  ey = (double)a.y / den;
  return ex * ex + ey * ey <= 0.25;
}

// e_ji of the update: kept j: the orthonormalising term -(R - I)_ji / 2 (FP64 R);
// discarded j: alpha_i x_j^dag res_i / (mu_i - lambda_j) where rf_pair applies it
// (alpha_i < 1 damps a column whose corrections are large in total).
__device__ __forceinline__ float2 rf_coef(int j, int i, int k, const float2* __restrict__ A,
                                          const double* __restrict__ mu, const double* __restrict__ lam,
                                          const double2* __restrict__ R, const double* __restrict__ alpha,
                                          int kmax) {
  if (j < k) {
    const double2 rv = R[(size_t)j * kmax + i];
    return make_float2((float)(-0.5 * (rv.x - (j == i ? 1.0 : 0.0))), (float)(-0.5 * rv.y));
  }
  double ex, ey, den;
  if (!rf_pair(j, i, A, mu, lam, kmax, ex, ey, den)) return make_float2(0.f, 0.f);
  return make_float2((float)(alpha[i] * ex), (float)(alpha[i] * ey));
}

// Xout = Xin + [Xin | Xd] E, E formed while staged (rf_coef); FP32 products
// accumulated onto the FP64 Xin
__global__ void __launch_bounds__(RT* RT)
    k_rf_update(const double2* __restrict__ Xall, int m, const double2* __restrict__ Xin, int ldi,
                const float2* __restrict__ A, const double* __restrict__ mu, const double* __restrict__ lam,
                const double2* __restrict__ R, const double* __restrict__ alpha, const EigOut* __restrict__ eo,
                int kmax, double2* __restrict__ Xout, int ldo) {
  const int k = eo->k < kmax ? eo->k : kmax;
  const int r0 = blockIdx.y * RT, c0 = blockIdx.x * RT;
  if (c0 >= k || r0 >= m) return;
  __shared__ float2 As[RT][RK + 1];  // [Xin | Xd][row][kg]
  __shared__ float2 Bs[RK][RT + 1];  // E[kg][col]
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  float2 acc = make_float2(0.f, 0.f);
  for (int kb = 0; kb < m; kb += RK) {
    for (int e = tid; e < RT * RK; e += RT * RT) {
      const int rr = e / RK, kk = e % RK;
      const int kg = kb + kk, rw = r0 + rr;
      float2 a = make_float2(0.f, 0.f);
      if (kg < m && rw < m) {
        const double2 v = kg < k ? Xin[(size_t)rw * ldi + kg] : Xall[(size_t)rw * m + kg];
        a = make_float2((float)v.x, (float)v.y);
      }
      As[rr][kk] = a;
    }
    for (int e = tid; e < RK * RT; e += RT * RT) {
      const int kk = e / RT, cc = e % RT;
      const int kg = kb + kk, cl = c0 + cc;
      Bs[kk][cc] = (kg < m && cl < k) ? rf_coef(kg, cl, k, A, mu, lam, R, alpha, kmax) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < RK; ++kk) cfma(acc, As[ty][kk], Bs[kk][tx]);
    __syncthreads();
  }
  const int row = r0 + ty, col = c0 + tx;
  if (row < m && col < k) {
    const double2 x = Xin[(size_t)row * ldi + col];
    Xout[(size_t)row * ldo + col] = make_double2(x.x + (double)acc.x, x.y + (double)acc.y);
  }
}

// Per kept column i, over the pairs rf_pair applies: s_i = sum_j |e_ji|^2 sets the
// damping alpha_i = min(1, sqrt(S_MAX / s_i)): a column whose corrections would move
// it far from unit norm takes a shorter step, so that the orthonormalisation steps
// (which square the deviation from orthonormality) converge.
constexpr double RF_SMAX = 1e-2;
__global__ void __launch_bounds__(256)
    k_rf_damp(const float2* __restrict__ A, const double* __restrict__ lam, int m, const EigOut* __restrict__ eo,
              int kmax, const double* __restrict__ mu, double* __restrict__ alpha) {
  const int k = eo->k < kmax ? eo->k : kmax;
  const int i = blockIdx.x;
  if (i >= k) return;
  __shared__ double red[32];
  const int j = k + threadIdx.x;
  double e2 = 0.0;
  if (j < m) {
    double ex, ey, den;
    if (rf_pair(j, i, A, mu, lam, kmax, ex, ey, den)) e2 = ex * ex + ey * ey;
  }
  e2 = block_sum(e2, red);
  if (threadIdx.x == 0) alpha[i] = e2 > RF_SMAX ? sqrt(RF_SMAX / e2) : 1.0;
}

// Xout = Xin (I - (R - I) / 2), R = Xin^dag Xin summed from the split partials (FP64)
__global__ void __launch_bounds__(RT* RT)
    k_rf_lowdin(const double2* __restrict__ P, int splits, int m, const double2* __restrict__ Xin, int ldi,
                const EigOut* __restrict__ eo, int kmax, double2* __restrict__ Xout, int ldo) {
  const int k = eo->k < kmax ? eo->k : kmax;
  const int r0 = blockIdx.y * RT, c0 = blockIdx.x * RT;
  if (c0 >= k || r0 >= m) return;
  __shared__ double2 As[RT][RK + 1];  // Xin[row][j]
  __shared__ double2 Bs[RK][RT + 1];  // -(R - I)[j][col] / 2
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  const size_t sstride = (size_t)(m + kmax) * kmax;
  double2 acc = make_double2(0.0, 0.0);
  for (int jb = 0; jb < k; jb += RK) {
    for (int e = tid; e < RT * RK; e += RT * RT) {
      const int rr = e / RK, jj = e % RK;
      const int rw = r0 + rr, j = jb + jj;
      As[rr][jj] = (rw < m && j < k) ? Xin[(size_t)rw * ldi + j] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < RK * RT; e += RT * RT) {
      const int jj = e / RT, cc = e % RT;
      const int j = jb + jj, cl = c0 + cc;
      double2 v = make_double2(0.0, 0.0);
      if (j < k && cl < k) {
        for (int s = 0; s < splits; ++s) v = cadd(v, P[s * sstride + (size_t)(m + j) * kmax + cl]);
        v = make_double2(-0.5 * (v.x - (j == cl ? 1.0 : 0.0)), -0.5 * v.y);
      }
      Bs[jj][cc] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < RK; ++jj) cfma(acc, As[ty][jj], Bs[jj][tx]);
    __syncthreads();
  }
  const int row = r0 + ty, col = c0 + tx;
  if (row < m && col < k) Xout[(size_t)row * ldo + col] = cadd(Xin[(size_t)row * ldi + col], acc);
}

// kept eigenvalues = FP64 Rayleigh quotients of the refined vectors, discarded mass =
// trace(G) - their sum
__global__ void __launch_bounds__(256)
    k_rf_finish(const double* __restrict__ mu, double* __restrict__ evals, int m, EigOut* __restrict__ eo,
                int kmax) {
  __shared__ double red[32];
  const int k = eo->k < kmax ? eo->k : kmax;
  const int t = threadIdx.x;
  double v = 0.0;
  if (t < k) {
    v = mu[t];
    evals[t] = v;
  }
  const double kept = block_sum(v, red);
  if (t == 0) {
    // the trace the truncation removes (for a positive semidefinite G this is the sum
    // of the discarded eigenvalues up to rounding)
    eo->kept = kept;
    eo->dropped = eo->trace - kept;
    if (k < m) {
      const double l1 = fabs(mu[0]) > 0.0 ? fabs(mu[0]) : 1.0;
      eo->gap = (mu[k - 1] - evals[k]) / l1;
    }
  }
}

}  // namespace

size_t eig_refine_work_bytes(int m) {
  const size_t kmax = (size_t)m;
  return (size_t)RF_SPLITS_MAX * (m + kmax) * kmax * sizeof(double2)  // P
         + (size_t)m * kmax * sizeof(double2)                           // Xn
         + (size_t)kmax * kmax * sizeof(double2)                        // R
         + (size_t)m * kmax * sizeof(float2) * 2                        // Res, A
         + (size_t)3 * kmax * sizeof(double) + 256;                     // mu, mu2, alpha
}

cudaError_t launch_eig_refine(const double2* G, int m, double* evals, double2* evecs, EigOut* eo, int kmax,
                              int iters, void* work, cudaStream_t s) {
  if (m < 2 || m > 256 || kmax < 1 || iters < 1) return cudaErrorInvalidValue;
  if (kmax > m) kmax = m;
  const int splits = (m + RK - 1) / RK;
  char* p = (char*)work;
  double2* P = (double2*)p;
  p += (size_t)RF_SPLITS_MAX * (m + m) * m * sizeof(double2);
  double2* Xn = (double2*)p;
  p += (size_t)m * m * sizeof(double2);
  double2* R = (double2*)p;
  p += (size_t)m * m * sizeof(double2);
  float2* Res = (float2*)p;
  p += (size_t)m * m * sizeof(float2);
  float2* A = (float2*)p;  // Xall^dag Res
  p += (size_t)m * m * sizeof(float2);
  double* mu = (double*)p;
  double* mu2 = mu + m;     // Rayleigh quotients of the refined vectors
  double* alpha = mu2 + m;  // damping of each kept column's step
  const dim3 tb(RT * RT);
  const dim3 g64((kmax + RT - 1) / RT, (m + kmax + RT - 1) / RT, splits);
  const dim3 gR((kmax + RT - 1) / RT, (kmax + RT - 1) / RT, splits);
  const dim3 g32((kmax + RT - 1) / RT, (m + RT - 1) / RT);
  // `iters` correction steps, then RF_ORTHO orthonormalisation steps; the steps
  // alternate between evecs' kept columns and Xn and the last one ends in evecs
  const int nsteps = iters + RF_ORTHO;
  for (int it = 0; it < nsteps; ++it) {
    const bool to_evecs = ((nsteps - 1 - it) % 2) == 0;
    const double2* Xin = to_evecs ? Xn : evecs;
    const int ldi = to_evecs ? kmax : m;
    double2* Xout = to_evecs ? evecs : Xn;
    const int ldo = to_evecs ? m : kmax;
    if (it == 0 && to_evecs) {
      // an odd number of steps starts from a copy so input and output differ
      cudaError_t e = cudaMemcpy2DAsync(Xn, kmax * sizeof(double2), evecs, m * sizeof(double2),
                                        kmax * sizeof(double2), m, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return e;
    }
    if (it < iters) {
      k_rf_gemm64<<<g64, tb, 0, s>>>(G, m, Xin, ldi, eo, kmax, 0, P);
      k_rf_res<<<kmax, 256, 0, s>>>(P, splits, m, Xin, ldi, eo, kmax, mu, R, Res);
      k_rf_proj<<<g32, tb, 0, s>>>(evecs, m, Res, eo, kmax, A);
      k_rf_damp<<<kmax, 256, 0, s>>>(A, evals, m, eo, kmax, mu, alpha);
      k_rf_update<<<g32, tb, 0, s>>>(evecs, m, Xin, ldi, A, mu, evals, R, alpha, eo, kmax, Xout, ldo);
      note_launches(5);
    } else if (it + 1 < nsteps) {
      k_rf_gemm64<<<gR, tb, 0, s>>>(G, m, Xin, ldi, eo, kmax, m, P);
      k_rf_lowdin<<<g32, tb, 0, s>>>(P, splits, m, Xin, ldi, eo, kmax, Xout, ldo);
      note_launches(2);
    } else {
      // the last step also forms G X: the kept eigenvalues are the Rayleigh quotients
      // of its input (nearly orthonormal by now, so the step changes them only at
      // second order in its tiny change)
      k_rf_gemm64<<<g64, tb, 0, s>>>(G, m, Xin, ldi, eo, kmax, 0, P);
      k_rf_res<<<kmax, 256, 0, s>>>(P, splits, m, Xin, ldi, eo, kmax, mu2, R, Res);
      k_rf_lowdin<<<g32, tb, 0, s>>>(P, splits, m, Xin, ldi, eo, kmax, Xout, ldo);
      note_launches(3);
    }
  }
  k_rf_finish<<<1, 256, 0, s>>>(mu2, evals, m, eo, kmax);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace lret
