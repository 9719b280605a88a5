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
// quotients of the input of the last of those steps (G X formed once more in FP64).
// Only G X, X^dag X and the Lowdin product X (R - I) / 2 are FP64 products; the
// complement projections and the update are FP32 products of small quantities.
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

// One truncation's operands and its workspace, carved as eig_refine_work_bytes lays it
// out. The steps read and write three buffers of kept columns: evecs (ld m; the FP32
// solve's vectors X0, which stay there until the last step writes the result) and
// the scratch buffers Xa, Xb (ld kmax). A step code st (the same for every
// truncation of a launch) names the input (st & 3) and the output (st >> 2):
// 0 = evecs, 1 = Xa, 2 = Xb.
struct RfView {
  const double2* G;
  int m, kmax, splits;
  double2 *evecs, *P, *Xa, *Xb, *R;
  float2 *Res, *A;
  double *evals, *mu, *mu2, *alpha;
  EigOut* eo;
};

__host__ __device__ __forceinline__ RfView rf_view(const RefineTask& t) {
  RfView v;
  v.G = t.G;
  v.m = t.m;
  v.kmax = t.kmax < t.m ? t.kmax : t.m;
  v.splits = (t.m + RK - 1) / RK;
  v.evecs = t.evecs;
  v.evals = t.evals;
  v.eo = t.eo;
  const size_t m = (size_t)t.m;
  char* p = (char*)t.work;
  v.P = (double2*)p;
  p += (size_t)RF_SPLITS_MAX * (m + m) * m * sizeof(double2);
  v.Xa = (double2*)p;
  p += m * m * sizeof(double2);
  v.Xb = (double2*)p;
  p += m * m * sizeof(double2);
  v.R = (double2*)p;
  p += m * m * sizeof(double2);
  v.Res = (float2*)p;
  p += m * m * sizeof(float2);
  v.A = (float2*)p;  // Xall^dag Res
  p += m * m * sizeof(float2);
  v.mu = (double*)p;
  v.mu2 = v.mu + m;     // Rayleigh quotients of the refined vectors
  v.alpha = v.mu2 + m;  // damping of each kept column's step
  return v;
}

__device__ __forceinline__ int rf_k(const RfView& v) { return v.eo->k < v.kmax ? v.eo->k : v.kmax; }
__device__ __forceinline__ double2* rf_buf(const RfView& v, int sel) {
  return sel == 0 ? v.evecs : (sel == 1 ? v.Xa : v.Xb);
}
__device__ __forceinline__ const double2* rf_in(const RfView& v, int st) { return rf_buf(v, st & 3); }
__device__ __forceinline__ int rf_ldin(const RfView& v, int st) { return (st & 3) == 0 ? v.m : v.kmax; }
__device__ __forceinline__ double2* rf_out(const RfView& v, int st) { return rf_buf(v, st >> 2); }
__device__ __forceinline__ int rf_ldout(const RfView& v, int st) { return (st >> 2) == 0 ? v.m : v.kmax; }

// P[s] = [G ; X^dag] X over the K chunk s (rows r < m: G[r][:], rows m + i: conj(X[:, i])),
// output rows from row0 (0: both products; m: X^dag X only).
__device__ __forceinline__ void rf_gemm64(const RfView& v, int st, int x_rows_only, int bx, int by, int s) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax;
  const double2* __restrict__ G = v.G;
  const double2* __restrict__ X = rf_in(v, st);
  const int ldx = rf_ldin(v, st);
  const int row0 = x_rows_only ? m : 0;
  const int r0 = row0 + by * RT, c0 = bx * RT;
  if (s >= v.splits || c0 >= k || r0 >= m + k) return;
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
  if (row < m + k && col < k) v.P[((size_t)s * (m + kmax) + row) * kmax + col] = acc;
}

// One block per kept column i: W[:, i] and R[:, i] from the split partials (fixed
// order), mu_i, res_i = w_i - mu_i x_i (stored in FP32), R (FP64).
__device__ __forceinline__ void rf_res(const RfView& v, int st, int i) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax, splits = v.splits;
  if (i >= k) return;
  const double2* __restrict__ P = v.P;
  const double2* __restrict__ X = rf_in(v, st);
  const int ldx = rf_ldin(v, st);
  double* mu = v.mu;
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
    v.R[(size_t)t * kmax + i] = rv;
  }
  q = block_sum(q, red);
  if (t == 0) {
    double nrm = 0.0;
    for (int s = 0; s < splits; ++s) nrm += P[s * sstride + (size_t)(m + i) * kmax + i].x;
    const double val = nrm > 0.0 ? q / nrm : 0.0;
    s_mu = val;
    mu[i] = val;
  }
  __syncthreads();
  if (t < m) {
    const double2 rs = csub(w, cscale(x, s_mu));
    v.Res[(size_t)t * kmax + i] = make_float2((float)rs.x, (float)rs.y);
  }
}

// Row tile of the m x k products: TM rows x RT columns per block (TM x RT threads, one
// output each; four-row tiles, measured, restage every coefficient four times as often
// and ran slower)
constexpr int TM = 16;

// A = Xall^dag Res (m x k): x_j^dag res_i for every column j of the FP32 solve, an
// FP32 product (res is small).
__device__ __forceinline__ void rf_proj(const RfView& v, int bx, int by) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax;
  const double2* __restrict__ Xall = v.evecs;
  const float2* __restrict__ Res = v.Res;
  const int r0 = by * TM, c0 = bx * RT;
  if (c0 >= k || r0 >= m) return;
  __shared__ float2 As[TM][RK + 1];  // conj(Xall[kg][row])
  __shared__ float2 Bs[RK][RT + 1];  // Res[kg][col]
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  float2 acc = make_float2(0.f, 0.f);
  for (int kb = 0; kb < m; kb += RK) {
    for (int e = tid; e < TM * RK; e += TM * RT) {
      const int rr = e % TM, kk = e / TM;
      const int kg = kb + kk, rw = r0 + rr;
      float2 a = make_float2(0.f, 0.f);
      if (kg < m && rw < m) {
        const double2 x = Xall[(size_t)kg * m + rw];
        a = make_float2((float)x.x, -(float)x.y);
      }
      As[rr][kk] = a;
    }
    for (int e = tid; e < RK * RT; e += TM * RT) {
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
  if (row < m && col < k) v.A[(size_t)row * kmax + col] = acc;
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

// Xout = Xin + [Xin | Xd] E with E the coefficients rf_coefs wrote over A; FP32
// products accumulated onto the FP64 Xin
__device__ __forceinline__ void rf_update(const RfView& v, int st, int bx, int by) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax;
  const double2* __restrict__ Xall = v.evecs;
  const double2* __restrict__ Xin = rf_in(v, st);
  const int ldi = rf_ldin(v, st);
  double2* __restrict__ Xout = rf_out(v, st);
  const int ldo = rf_ldout(v, st);
  const float2* __restrict__ E = v.A;
  const int r0 = by * TM, c0 = bx * RT;
  if (c0 >= k || r0 >= m) return;
  __shared__ float2 As[TM][RK + 1];  // [Xin | Xd][row][kg]
  __shared__ float2 Bs[RK][RT + 1];  // E[kg][col]
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  float2 acc = make_float2(0.f, 0.f);
  for (int kb = 0; kb < m; kb += RK) {
    for (int e = tid; e < TM * RK; e += TM * RT) {
      const int rr = e / RK, kk = e % RK;
      const int kg = kb + kk, rw = r0 + rr;
      float2 a = make_float2(0.f, 0.f);
      if (kg < m && rw < m) {
        const double2 x = kg < k ? Xin[(size_t)rw * ldi + kg] : Xall[(size_t)rw * m + kg];
        a = make_float2((float)x.x, (float)x.y);
      }
      As[rr][kk] = a;
    }
    for (int e = tid; e < RK * RT; e += TM * RT) {
      const int kk = e / RT, cc = e % RT;
      const int kg = kb + kk, cl = c0 + cc;
      Bs[kk][cc] = (kg < m && cl < k) ? E[(size_t)kg * kmax + cl] : make_float2(0.f, 0.f);
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

// Coefficients E of the update, one block per kept column i, thread j per row of E,
// written over A (each entry by the thread that read it): kept j: the
// orthonormalising term -(R - I)_ji / 2 (FP64 R); discarded j: alpha_i x_j^dag res_i /
// (mu_i - lambda_j) where rf_pair applies it, else 0. Over the pairs rf_pair applies,
// s_i = sum_j |e_ji|^2 sets the damping alpha_i = min(1, sqrt(S_MAX / s_i)): a column
// whose corrections would move it far from unit norm takes a shorter step, so that
// the orthonormalisation steps (which square the deviation from orthonormality)
// converge.
constexpr double RF_SMAX = 1e-2;
__device__ __forceinline__ void rf_coefs(const RfView& v, int i) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax;
  if (i >= k) return;
  __shared__ double red[32];
  const int j = threadIdx.x;
  double ex = 0.0, ey = 0.0, den, e2 = 0.0;
  bool use = false;
  if (j >= k && j < m) {
    use = rf_pair(j, i, v.A, v.mu, v.evals, kmax, ex, ey, den);
    if (use) e2 = ex * ex + ey * ey;
  }
  e2 = block_sum(e2, red);  // (its barriers also order every read of A before the writes)
  const double alpha = e2 > RF_SMAX ? sqrt(RF_SMAX / e2) : 1.0;
  if (j < k) {
    const double2 rv = v.R[(size_t)j * kmax + i];
    v.A[(size_t)j * kmax + i] = make_float2((float)(-0.5 * (rv.x - (j == i ? 1.0 : 0.0))), (float)(-0.5 * rv.y));
  } else if (j < m) {
    v.A[(size_t)j * kmax + i] = use ? make_float2((float)(alpha * ex), (float)(alpha * ey)) : make_float2(0.f, 0.f);
  }
}

// Xout = Xin (I - (R - I) / 2), R = Xin^dag Xin summed from the split partials (FP64).
// The product Xin (R - I) / 2 is formed in FP64 where a coefficient of this block's
// columns exceeds RF_LOW32 and in FP32 otherwise: with |R - I| <= 1e-9 the FP32
// rounding of Xin and of the sums moves a column by at most about
// 2^-24 sqrt(k) 1e-9 ~ 5e-16, below the FP64 accuracy the steps aim at. After the
// correction step the deviation is the square of the corrections (1e-14 for
// undamped columns), so the FP64 products are needed only behind damped columns.
constexpr double RF_LOW32 = 1e-9;
__device__ __forceinline__ void rf_lowdin(const RfView& v, int st, int bx, int by) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax, splits = v.splits;
  const double2* __restrict__ P = v.P;
  const double2* __restrict__ Xin = rf_in(v, st);
  const int ldi = rf_ldin(v, st);
  double2* __restrict__ Xout = rf_out(v, st);
  const int ldo = rf_ldout(v, st);
  const int r0 = by * TM, c0 = bx * RT;
  if (c0 >= k || r0 >= m) return;
  __shared__ double2 As[TM][RK + 1];  // Xin[row][j]
  __shared__ double2 Bs[RK][RT + 1];  // -(R - I)[j][col] / 2
  __shared__ int s_big;
  const int tx = threadIdx.x % RT, ty = threadIdx.x / RT, tid = threadIdx.x;
  const size_t sstride = (size_t)(m + kmax) * kmax;
  auto coef = [&](int j, int cl) {
    double2 x = make_double2(0.0, 0.0);
    for (int s = 0; s < splits; ++s) x = cadd(x, P[s * sstride + (size_t)(m + j) * kmax + cl]);
    return make_double2(-0.5 * (x.x - (j == cl ? 1.0 : 0.0)), -0.5 * x.y);
  };
  if (tid == 0) s_big = 0;
  __syncthreads();
  bool big = false;
  for (int e = tid; e < k * RT; e += TM * RT) {
    const int j = e / RT, cl = c0 + e % RT;
    if (cl < k) {
      const double2 x = coef(j, cl);
      if (fabs(x.x) > RF_LOW32 || fabs(x.y) > RF_LOW32) big = true;
    }
  }
  if (big) s_big = 1;
  __syncthreads();
  const bool f64 = s_big != 0;
  double2 acc = make_double2(0.0, 0.0);
  float2 acc32 = make_float2(0.f, 0.f);
  for (int jb = 0; jb < k; jb += RK) {
    for (int e = tid; e < TM * RK; e += TM * RT) {
      const int rr = e / RK, jj = e % RK;
      const int rw = r0 + rr, j = jb + jj;
      As[rr][jj] = (rw < m && j < k) ? Xin[(size_t)rw * ldi + j] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < RK * RT; e += TM * RT) {
      const int jj = e / RT, cc = e % RT;
      const int j = jb + jj, cl = c0 + cc;
      Bs[jj][cc] = (j < k && cl < k) ? coef(j, cl) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (f64) {
#pragma unroll 8
      for (int jj = 0; jj < RK; ++jj) cfma(acc, As[ty][jj], Bs[jj][tx]);
    } else {
#pragma unroll 8
      for (int jj = 0; jj < RK; ++jj) {
        const double2 a = As[ty][jj], b = Bs[jj][tx];
        cfma(acc32, make_float2((float)a.x, (float)a.y), make_float2((float)b.x, (float)b.y));
      }
    }
    __syncthreads();
  }
  if (!f64) acc = make_double2((double)acc32.x, (double)acc32.y);
  const int row = r0 + ty, col = c0 + tx;
  if (row < m && col < k) Xout[(size_t)row * ldo + col] = cadd(Xin[(size_t)row * ldi + col], acc);
}

// mu2_i = x_i^dag G x_i / x_i^dag x_i from G X and X^dag X of this step's input (split
// partials in P, summed in FP64); one block per kept column.
__device__ __forceinline__ void rf_mu2(const RfView& v, int st, int i) {
  const int k = rf_k(v), m = v.m, kmax = v.kmax, splits = v.splits;
  if (i >= k) return;
  const double2* __restrict__ P = v.P;
  const double2* __restrict__ X = rf_in(v, st);
  const int ldx = rf_ldin(v, st);
  __shared__ double red[32];
  const int t = threadIdx.x;
  const size_t sstride = (size_t)(m + kmax) * kmax;
  double q = 0.0;
  if (t < m) {
    double2 w0 = make_double2(0.0, 0.0);
    for (int s = 0; s < splits; ++s) w0 = cadd(w0, P[s * sstride + (size_t)t * kmax + i]);
    const double2 x = X[(size_t)t * ldx + i];
    q = x.x * w0.x + x.y * w0.y;
  }
  q = block_sum(q, red);
  if (t == 0) {
    double nrm = 0.0;
    for (int s = 0; s < splits; ++s) nrm += P[s * sstride + (size_t)(m + i) * kmax + i].x;
    v.mu2[i] = nrm > 0.0 ? q / nrm : 0.0;
  }
}

// kept eigenvalues = FP64 Rayleigh quotients of the refined vectors, discarded mass =
// trace(G) - their sum
__device__ __forceinline__ void rf_finish(const RfView& v) {
  __shared__ double red[32];
  const int k = rf_k(v), m = v.m;
  const double* mu = v.mu2;
  EigOut* eo = v.eo;
  const int t = threadIdx.x;
  double x = 0.0;
  if (t < k) {
    x = mu[t];
    v.evals[t] = x;
  }
  const double kept = block_sum(x, red);
  if (t == 0) {
    // the trace the truncation removes (for a positive semidefinite G this is the sum
    // of the discarded eigenvalues up to rounding)
    eo->kept = kept;
    eo->dropped = eo->trace - kept;
    if (k < m) {
      const double l1 = fabs(mu[0]) > 0.0 ? fabs(mu[0]) : 1.0;
      eo->gap = (mu[k - 1] - v.evals[k]) / l1;
    }
  }
}

// Kernels: each phase as one truncation (task passed by value) or as a batch (task
// blockIdx.z / zper of the array; zper = the blocks in z one truncation uses)
enum RfPhase { RF_GEMM = 0, RF_RES, RF_PROJ, RF_COEFS, RF_UPDATE, RF_LOWDIN, RF_MU2, RF_FINISH };

template <int PHASE>
__device__ __forceinline__ void rf_phase(const RefineTask& t, int a0, int a1, int bz) {
  const RfView v = rf_view(t);
  if constexpr (PHASE == RF_GEMM) rf_gemm64(v, a0, a1, blockIdx.x, blockIdx.y, bz);
  else if constexpr (PHASE == RF_RES) rf_res(v, a0, blockIdx.x);
  else if constexpr (PHASE == RF_PROJ) rf_proj(v, blockIdx.x, blockIdx.y);
  else if constexpr (PHASE == RF_COEFS) rf_coefs(v, blockIdx.x);
  else if constexpr (PHASE == RF_UPDATE) rf_update(v, a0, blockIdx.x, blockIdx.y);
  else if constexpr (PHASE == RF_LOWDIN) rf_lowdin(v, a0, blockIdx.x, blockIdx.y);
  else if constexpr (PHASE == RF_MU2) rf_mu2(v, a0, blockIdx.x);
  else rf_finish(v);
}

template <int PHASE>
__global__ void __launch_bounds__(256, 1) k_rf(RefineTask t, int a0, int a1) {
  rf_phase<PHASE>(t, a0, a1, blockIdx.z);
}

template <int PHASE>
__global__ void __launch_bounds__(256, 1) k_rf_batch(const RefineTask* __restrict__ tasks, int zper, int a0, int a1) {
  rf_phase<PHASE>(tasks[blockIdx.z / zper], a0, a1, blockIdx.z % zper);
}

// Grid of one phase for a truncation of size m with kmax kept columns.
struct RfGrid {
  dim3 g;
  int threads;
};
RfGrid rf_grid(int phase, int m, int kmax, int x_rows_only) {
  const int kb = (kmax + RT - 1) / RT, splits = (m + RK - 1) / RK;
  switch (phase) {
    case RF_GEMM: return {dim3(kb, ((x_rows_only ? kmax : m + kmax) + RT - 1) / RT, splits), RT * RT};
    case RF_RES: case RF_COEFS: case RF_MU2: return {dim3(kmax), 256};
    case RF_PROJ: case RF_UPDATE: case RF_LOWDIN: return {dim3(kb, (m + TM - 1) / TM), TM * RT};
    default: return {dim3(1), 256};
  }
}

// Launches one phase: ntasks == 0 -> the single task t by value; else tasks[0..ntasks)
// with the grid of the largest (m_max, kmax_max).
template <int PHASE>
void rf_launch(const RefineTask& t, const RefineTask* tasks, int ntasks, int m_max, int kmax_max, int a0, int a1,
               cudaStream_t s) {
  const int rows_only = PHASE == RF_GEMM ? a1 : 0;
  RfGrid gr = ntasks == 0 ? rf_grid(PHASE, t.m, t.kmax < t.m ? t.kmax : t.m, rows_only)
                          : rf_grid(PHASE, m_max, kmax_max, rows_only);
  if (ntasks == 0) {
    k_rf<PHASE><<<gr.g, gr.threads, 0, s>>>(t, a0, a1);
  } else {
    const int zper = (int)gr.g.z;
    dim3 g = gr.g;
    g.z = (unsigned)(zper * ntasks);
    k_rf_batch<PHASE><<<g, gr.threads, 0, s>>>(tasks, zper, a0, a1);
  }
}

// The whole refinement: `iters` correction steps, then RF_ORTHO orthonormalisation
// steps. Step 0 reads evecs; step it > 0 reads Xa (it odd) or Xb (it even); every step
// but the last writes the other scratch buffer, the last writes evecs.
int rf_step_code(int it, int nsteps) {
  const int in = it == 0 ? 0 : ((it - 1) % 2 == 0 ? 1 : 2);
  const int out = it == nsteps - 1 ? 0 : (it % 2 == 0 ? 1 : 2);
  return in | (out << 2);
}

cudaError_t rf_run(const RefineTask& t, const RefineTask* tasks, int ntasks, int m_max, int kmax_max, int iters,
                   cudaStream_t s) {
  const int nsteps = iters + RF_ORTHO;
  long long launches = 0;
  for (int it = 0; it < nsteps; ++it) {
    const int st = rf_step_code(it, nsteps);
    if (it < iters) {
      rf_launch<RF_GEMM>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      rf_launch<RF_RES>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      rf_launch<RF_PROJ>(t, tasks, ntasks, m_max, kmax_max, 0, 0, s);
      rf_launch<RF_COEFS>(t, tasks, ntasks, m_max, kmax_max, 0, 0, s);
      rf_launch<RF_UPDATE>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      launches += 5;
    } else if (it + 1 < nsteps) {
      rf_launch<RF_GEMM>(t, tasks, ntasks, m_max, kmax_max, st, 1, s);
      rf_launch<RF_LOWDIN>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      launches += 2;
    } else {
      // the last step's input is nearly orthonormal: its Rayleigh quotients (the kept
      // eigenvalues) change only at second order in the step's tiny change; G X of the
      // input in FP64 (an expansion around G X0 with an FP32 G Delta would carry about
      // 2^-24 |Delta|^2 lambda_1, above 1e-13 lambda_1 for a column the correction step
      // moved by more than about 1e-3, as damped columns can be)
      rf_launch<RF_GEMM>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      rf_launch<RF_MU2>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      rf_launch<RF_LOWDIN>(t, tasks, ntasks, m_max, kmax_max, st, 0, s);
      launches += 3;
    }
  }
  rf_launch<RF_FINISH>(t, tasks, ntasks, m_max, kmax_max, 0, 0, s);
  note_launches(launches + 1);
  return cudaGetLastError();
}

}  // namespace

size_t eig_refine_work_bytes(int m) {
  const size_t kmax = (size_t)m;
  return (size_t)RF_SPLITS_MAX * (m + kmax) * kmax * sizeof(double2)  // P
         + (size_t)2 * m * kmax * sizeof(double2)                       // Xa, Xb
         + (size_t)kmax * kmax * sizeof(double2)                        // R
         + (size_t)m * kmax * sizeof(float2) * 2                        // Res, A
         + (size_t)3 * kmax * sizeof(double) + 256;                     // mu, mu2, alpha
}


cudaError_t launch_eig_refine(const double2* G, int m, double* evals, double2* evecs, EigOut* eo, int kmax,
                              int iters, void* work, cudaStream_t s) {
  if (m < 2 || m > 256 || kmax < 1 || iters < 1) return cudaErrorInvalidValue;
  RefineTask t{G, m, kmax < m ? kmax : m, evals, evecs, eo, work};
  return rf_run(t, nullptr, 0, 0, 0, iters, s);
}

cudaError_t launch_eig_refine_batch(const RefineTask* tasks, int ntasks, int m_max, int kmax_max, int iters,
                                    cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (m_max < 2 || m_max > 256 || kmax_max < 1 || iters < 1) return cudaErrorInvalidValue;
  RefineTask none{};
  return rf_run(none, tasks, ntasks, m_max, kmax_max < m_max ? kmax_max : m_max, iters, s);
}

}  // namespace lret
