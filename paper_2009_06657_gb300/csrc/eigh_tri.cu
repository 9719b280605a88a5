// Hermitian eigensolver for large truncation Gram matrices (m up to 256):
// Householder reduction to real tridiagonal form, bisection for every
// eigenvalue, inverse iteration for the needed eigenvectors, back-transform.
//
// The truncation of Sec. II.B needs the leading eigenpairs of G = V'^dag V'
// (Theorem 1, App. B). Two-sided Jacobi costs O(m^3) per sweep over many
// sweeps; this path does one O(m^3) reduction and O(m^2) per eigenpair after
// it, so it is the fast path for the FP32 state at r*K = 256.
//
// Stages (one thread block of 1024 threads):
//  1. Reduction. For j = 0..m-2 a reflector H_j = I - tau v v^dag (v_0 = 1,
//     acting on rows j+1..m-1) maps column j below the diagonal to beta e_1
//     with beta real; the trailing block becomes H^dag A H through
//     p = tau A v, w = p - (1/2) conj(tau) (v^dag p) v, A <- A - w v^dag - v w^dag.
//     The lower triangle is stored packed by columns; the trailing columns
//     live in shared memory, the first ones in a global scratch slab.
//  2. The tridiagonal T (diagonal d, real off-diagonal e) is split where e is
//     negligible; Sturm-count bisection gives each eigenvalue of each block.
//  3. Eigenvalues are sorted descending; the kept count and the FP64
//     kept/discarded sums are formed.
//  4. Inverse iteration with a pivoted tridiagonal LU (one warp per vector, all
//     vectors in parallel) gives eigenvectors of T; a modified Gram-Schmidt
//     pass in rank order makes the set exactly orthonormal.
//  5. Back-transform y = H_0 H_1 ... H_{m-2} z, reflectors staged through
//     shared memory in chunks shared by all warps.
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace lret {

template <typename T> struct TEps;
template <> struct TEps<float> { static constexpr float v = FLT_EPSILON; static constexpr float tiny = 1e-30f; };
template <> struct TEps<double> { static constexpr double v = DBL_EPSILON; static constexpr double tiny = 1e-290; };

constexpr int TRI_THREADS = 1024;
constexpr int TRI_MAXM = 256;
template <typename T> struct LuWarps { static constexpr int v = sizeof(T) == 4 ? 24 : 12; };
constexpr int TRI_CHUNK = 8;  // reflectors staged per back-transform chunk

__host__ __device__ __forceinline__ int packed_off(int c, int m) { return c * m - (c * (c - 1)) / 2; }

template <typename T>
__device__ __forceinline__ T block_reduce(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
  const T den = b.x * b.x + b.y * b.y;
  return mk<T>((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

// Division in the Sturm recurrence: only the signs of the pivots are used, so a
// fast FP32 quotient (a few ulp) is enough there.
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }

// Sturm count: number of eigenvalues of the block [lo, hi] smaller than x.
template <typename T>
__device__ int sturm(const T* d, const T* e2, int lo, int hi, T x, T pivmin) {
  int cnt = 0;
  T q = d[lo] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = lo + 1; i <= hi; ++i) {
    q = d[i] - x - sdiv(e2[i - 1], q);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

template <typename T>
__device__ __forceinline__ void eigh_tri_body(const double2* __restrict__ G, int m, int c_split,
                                              cx<T>* gpacked, T* gZ, double* __restrict__ evals,
                                              double2* __restrict__ evecs, EigOut* __restrict__ out,
                                              int r, double eps, int all_vecs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ cx<T>* colptr[TRI_MAXM];
  __shared__ cx<T> sv[TRI_MAXM], sp[TRI_MAXM], stau[TRI_MAXM];
  __shared__ T sd[TRI_MAXM], se[TRI_MAXM], se2[TRI_MAXM], slam[TRI_MAXM];
  __shared__ short sblo[TRI_MAXM], sbhi[TRI_MAXM];  // block range of position / sorted eigenvalue
  __shared__ short sorder[TRI_MAXM];                  // sorted rank -> position index
  __shared__ int s_k;
  __shared__ T red[32], red2[32];
  __shared__ cx<T> s_tau, s_scale;
  __shared__ T s_c;
  __shared__ double s_trace;
  __shared__ double dred[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int moff_split = packed_off(c_split, m);
  long long t_mark = clock64();
  long long t_ph[6] = {0, 0, 0, 0, 0, 0};
  cx<T>* spk = (cx<T>*)smem_raw;

  // ---- 1. load the lower triangle, packed by columns ----------------------
  for (int c = tid; c < m; c += blockDim.x) {
    const int o = packed_off(c, m);
    colptr[c] = (c >= c_split) ? spk + (o - moff_split) : gpacked + o;
  }
  double tr = 0.0;
  for (int i = tid; i < m; i += blockDim.x) tr += G[(size_t)i * m + i].x;
  {
    const double t = block_sum(tr, dred);
    if (tid == 0) s_trace = t;
  }
  __syncthreads();
  // work on G / trace (entries of order one, so FP32 squares of small entries
  // stay normal); eigenvalues are scaled back when written out
  const double gscale = s_trace > 0.0 ? s_trace : 1.0;
  const double ginv = 1.0 / gscale;
  for (int e = tid; e < m * m; e += blockDim.x) {
    const int i = e / m, c = e % m;
    if (i >= c) {
      const double2 g = G[e];
      colptr[c][i - c] = mk<T>((T)(g.x * ginv), (T)(g.y * ginv));
    }
  }
  __syncthreads();

  // ---- reduction to tridiagonal form --------------------------------------
  for (int j = 0; j < m - 1; ++j) {
    const int n1 = m - j - 1;
    cx<T>* colj = colptr[j];
    // norms are taken on values scaled by the column's largest magnitude, so
    // squares of tiny entries cannot underflow to zero (which would give beta = 0)
    // one pass: largest magnitude and unscaled sum of squares of x[1:]; the
    // scaled sum is recomputed serially only when the plain one underflowed
    T amax = 0, part = 0;
    for (int i = tid + 1; i <= n1; i += blockDim.x) {
      const cx<T> x = colj[i];
      amax = fmax(amax, fmax(fabs(x.x), fabs(x.y)));
      if (i >= 2) part += x.x * x.x + x.y * x.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      part += __shfl_xor_sync(0xffffffffu, part, o);
    }
    __syncthreads();
    if (lane == 0) { red[warp] = amax; red2[warp] = part; }
    __syncthreads();
    amax = 0;
    T xn2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { amax = fmax(amax, red[w]); xn2 += red2[w]; }
    const T inv_amax = amax > (T)0 ? (T)1 / amax : (T)0;
    T xn2s = xn2 * inv_amax * inv_amax;  // ||x[1:]||^2 / amax^2
    if (tid == 0 && amax > (T)0 && xn2 < (T)1e-30) {  // squares may have underflowed
      T sacc = 0;
      for (int i = 2; i <= n1; ++i) {
        const T a = colj[i].x * inv_amax, b = colj[i].y * inv_amax;
        sacc += a * a + b * b;
      }
      xn2s = sacc;
    }
    if (tid == 0) {
      const cx<T> alpha = colj[1];
      T beta;
      cx<T> tau, scale;
      // a column already zero to 1e-30 of the (unit) trace needs no reflector
      if (amax <= (T)1e-30 || (xn2s == (T)0 && alpha.y == (T)0)) {
        tau = mk<T>(0, 0);
        beta = alpha.x;
        scale = mk<T>(0, 0);
      } else {
        const T ar = alpha.x * inv_amax, ai = alpha.y * inv_amax;
        const T bs = -copysign(sqrt(ar * ar + ai * ai + xn2s), ar);  // beta / amax
        beta = amax * bs;
        tau = mk<T>((bs - ar) / bs, -ai / bs);
        // 1 / (alpha - beta) = (1 / amax) / ((alpha - beta) / amax), the latter of order one
        const cx<T> z = cdiv<T>(mk<T>(1, 0), mk<T>(ar - bs, ai));
        scale = mk<T>(z.x * inv_amax, z.y * inv_amax);
      }
      sd[j] = colj[0].x;
      se[j] = beta;
      stau[j] = tau;
      s_tau = tau;
      s_scale = scale;
      colj[1] = mk<T>(beta, 0);
    }
    __syncthreads();
    const cx<T> tau = s_tau;
    if (tau.x == (T)0 && tau.y == (T)0) continue;  // H = I (x[1:] is already zero)
    const cx<T> scale = s_scale;
    for (int t = tid; t < n1; t += blockDim.x) {
      const int row = j + 1 + t;
      if (t == 0) {
        sv[row] = mk<T>(1, 0);
      } else {
        const cx<T> v = cmul(colj[t + 1], scale);
        colj[t + 1] = v;
        sv[row] = v;
      }
    }
    __syncthreads();
    // p = tau * A22 v, four threads per row
    {
      const int rr = tid >> 2, sub = tid & 3;
      const int row = j + 1 + rr;
      cx<T> acc = mk<T>(0, 0);
      if (rr < n1) {
#pragma unroll 4
        for (int col = j + 1 + sub; col < m; col += 4) {
          const cx<T> a = (col <= row) ? colptr[col][row - col] : conjg(colptr[row][col - row]);
          cfma(acc, a, sv[col]);
        }
      }
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (rr < n1 && sub == 0) sp[row] = cmul(tau, acc);
    }
    __syncthreads();
    // c = (1/2) Re(conj(tau) * (v^dag p)), both parts in one reduction
    {
      T pr = 0, pi = 0;
      for (int t = tid; t < n1; t += blockDim.x) {
        const int row = j + 1 + t;
        const cx<T> v = sv[row], p = sp[row];
        pr += v.x * p.x + v.y * p.y;
        pi += v.x * p.y - v.y * p.x;
      }
      for (int o = 16; o > 0; o >>= 1) {
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
      }
      if (lane == 0) { red[warp] = pr; red2[warp] = pi; }
      __syncthreads();
      if (tid == 0) {
        T dr = 0, di = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { dr += red[w]; di += red2[w]; }
        s_c = (T)0.5 * (tau.x * dr + tau.y * di);
      }
      __syncthreads();
    }
    const T cc = s_c;
    for (int t = tid; t < n1; t += blockDim.x) {
      const int row = j + 1 + t;
      sp[row] = csub(sp[row], cscale(sv[row], cc));  // w = p - c v
    }
    __syncthreads();
    // A22 <- A22 - w v^dag - v w^dag (lower triangle), one warp per column
    for (int col = j + 1 + warp; col < m; col += (blockDim.x >> 5)) {
      cx<T>* cp = colptr[col];
      const cx<T> vc = conjg(sv[col]), wc = conjg(sp[col]);
      for (int row = col + lane; row < m; row += 32) {
        cx<T> a = cp[row - col];
        a = csub(a, cadd(cmul(sp[row], vc), cmul(sv[row], wc)));
        if (row == col) a.y = 0;
        cp[row - col] = a;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    sd[m - 1] = colptr[m - 1][0].x;
    if (m >= 1) se[m - 1] = 0;
  }
  __syncthreads();
  if (tid == 0) { const long long t = clock64(); t_ph[0] = t - t_mark; t_mark = t; }
  // move the shared part of the packed reflectors to global (shared memory is reused below)
  {
    const int total = packed_off(m, m) - moff_split;
    for (int e = tid; e < total; e += blockDim.x) gpacked[moff_split + e] = spk[e];
  }

  // ---- 2. split into unreduced blocks, bisection ---------------------------
  __shared__ T s_tnorm, s_pivmin;
  if (tid == 0) {
    T tn = 0, emax2 = 0;
    for (int i = 0; i < m; ++i) {
      const T a = fabs(sd[i]) + (i > 0 ? fabs(se[i - 1]) : (T)0) + (i < m - 1 ? fabs(se[i]) : (T)0);
      tn = a > tn ? a : tn;
    }
    for (int i = 0; i < m - 1; ++i) {
      if (fabs(se[i]) <= TEps<T>::v * (fabs(sd[i]) + fabs(sd[i + 1])) || fabs(se[i]) <= TEps<T>::v * TEps<T>::v * tn)
        se[i] = 0;
      se2[i] = se[i] * se[i];
      emax2 = se2[i] > emax2 ? se2[i] : emax2;
    }
    int lo = 0;
    for (int i = 0; i < m; ++i) {
      if (i == m - 1 || se[i] == (T)0) {
        for (int t = lo; t <= i; ++t) { sblo[t] = (short)lo; sbhi[t] = (short)i; }
        lo = i + 1;
      }
    }
    s_tnorm = tn > (T)0 ? tn : (T)1;
    s_pivmin = TEps<T>::tiny * (emax2 > (T)1 ? emax2 : (T)1);
  }
  __syncthreads();
  const T tnorm = s_tnorm, pivmin = s_pivmin;
  for (int t = tid; t < m; t += blockDim.x) {
    const int lo = sblo[t], hi = sbhi[t], li = t - lo;
    T gl = sd[lo], gu = sd[lo];
    for (int i = lo; i <= hi; ++i) {
      const T rad = (i > lo ? fabs(se[i - 1]) : (T)0) + (i < hi ? fabs(se[i]) : (T)0);
      gl = fmin(gl, sd[i] - rad);
      gu = fmax(gu, sd[i] + rad);
    }
    T a = gl - TEps<T>::v * tnorm * 2 - pivmin, b = gu + TEps<T>::v * tnorm * 2 + pivmin;
    for (int it = 0; it < 100; ++it) {
      const T mid = (T)0.5 * (a + b);
      if (b - a <= (T)2 * TEps<T>::v * fmax(fabs(a), fabs(b)) + TEps<T>::v * tnorm * (T)1e-3 || mid == a || mid == b)
        break;
      if (sturm<T>(sd, se2, lo, hi, mid, pivmin) <= li) a = mid; else b = mid;
    }
    slam[t] = (T)0.5 * (a + b);
  }
  __syncthreads();

  if (tid == 0) { const long long t = clock64(); t_ph[1] = t - t_mark; t_mark = t; }
  // ---- 3. sort descending, rank choice, FP64 accounting --------------------
  // a NaN (from a non-finite input) sorts last so ranks stay a permutation
  for (int t = tid; t < m; t += blockDim.x)
    if (!(slam[t] == slam[t])) slam[t] = -INFINITY;
  __syncthreads();
  for (int t = tid; t < m; t += blockDim.x) {
    const T lt = slam[t];
    int rank = 0;
    for (int u = 0; u < m; ++u) {
      const T lu = slam[u];
      rank += (lu > lt) || (lu == lt && u < t);
    }
    sorder[rank] = (short)t;
    evals[rank] = (double)lt * gscale;
  }
  __syncthreads();
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
    }
    double kept = 0.0, dropped = 0.0;
    for (int i = 0; i < m; ++i) {
      const double v = evals[i] > 0 ? evals[i] : 0.0;
      if (i < k) kept += v; else dropped += v;
    }
    const double l1 = fabs(evals[0]) > 0 ? fabs(evals[0]) : 1.0;
    out->k = k;
    out->sweeps = 0;
    out->status = isfinite(evals[m - 1]) ? 0 : 2;
    out->dropped = dropped;
    out->kept = kept;
    out->gap = k < m ? (evals[k - 1] - evals[k]) / l1 : __longlong_as_double(0x7ff0000000000000ll);
    out->trace = s_trace;
    s_k = k;
  }
  __syncthreads();
  const int nvec = all_vecs ? m : s_k;
  if (tid == 0) { const long long t = clock64(); t_ph[2] = t - t_mark; t_mark = t; }

  // ---- 4. inverse iteration: one warp per needed eigenvector, all in parallel ----
  // Each vector starts from its own pseudo-random vector, so vectors of nearly
  // equal eigenvalues span their joint invariant subspace; the orthonormalisation
  // below then gives an exact orthonormal basis of the kept (and, when needed,
  // discarded) subspaces, which is what the truncation uses.
  {
    T* ws = (T*)smem_raw;  // per-warp scratch: dl, dd, du, du2, x (5 * m) + piv
    constexpr int NLU = LuWarps<T>::v;
    if (warp < NLU) {
      T* dl = ws + (size_t)warp * (6 * TRI_MAXM);
      T* dd = dl + TRI_MAXM;
      T* du = dd + TRI_MAXM;
      T* du2 = du + TRI_MAXM;
      T* x = du2 + TRI_MAXM;
      unsigned char* piv = (unsigned char*)(x + TRI_MAXM);
      for (int i = warp; i < nvec; i += NLU) {
        const int pos = sorder[i];
        const int lo = sblo[pos], hi = sbhi[pos], s = hi - lo + 1;
        T* z = gZ + (size_t)i * m;  // column i of Z, stored contiguously
        for (int t = lane; t < m; t += 32) z[t] = 0;
        __syncwarp();
        if (s == 1) {
          if (lane == 0) z[lo] = 1;
          __syncwarp();
          continue;
        }
        const T lam = slam[pos];
        if (lane == 0) {
          // LU with partial pivoting of (T_block - lam I)
          const T tiny = TEps<T>::v * tnorm;
          for (int t = 0; t < s; ++t) {
            dd[t] = sd[lo + t] - lam;
            if (t < s - 1) { dl[t] = se[lo + t]; du[t] = se[lo + t]; du2[t] = 0; }
          }
          for (int t = 0; t < s - 1; ++t) {
            if (fabs(dd[t]) >= fabs(dl[t])) {
              if (dd[t] == (T)0) dd[t] = tiny;
              const T l = dl[t] / dd[t];
              dl[t] = l;
              dd[t + 1] -= l * du[t];
              piv[t] = 0;
            } else {
              const T l = dd[t] / dl[t];
              dd[t] = dl[t];
              dl[t] = l;
              const T tmp = du[t];
              du[t] = dd[t + 1];
              dd[t + 1] = tmp - l * dd[t + 1];
              if (t < s - 2) {
                du2[t] = du[t + 1];
                du[t + 1] = -l * du[t + 1];
              }
              piv[t] = 1;
            }
          }
          if (dd[s - 1] == (T)0) dd[s - 1] = tiny;
        }
        // pseudo-random start vector (integer hash of vector and row index)
        for (int t = lane; t < s; t += 32) {
          unsigned h = (unsigned)(t + 1) * 2654435761u ^ ((unsigned)(i + 7) * 40503u + 0x9e3779b9u);
          h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
          const T u = (T)(h & 0xffffu) * (T)(1.0 / 65536.0) + (T)0.5;
          x[t] = (h & 0x10000u) ? -u : u;
        }
        __syncwarp();
        for (int it = 0; it < 2; ++it) {
          if (lane == 0) {
            for (int t = 0; t < s - 1; ++t) {
              if (piv[t] == 0) {
                x[t + 1] -= dl[t] * x[t];
              } else {
                const T tmp = x[t];
                x[t] = x[t + 1];
                x[t + 1] = tmp - dl[t] * x[t + 1];
              }
            }
            x[s - 1] /= dd[s - 1];
            x[s - 2] = (x[s - 2] - du[s - 2] * x[s - 1]) / dd[s - 2];
            for (int t = s - 3; t >= 0; --t) x[t] = (x[t] - du[t] * x[t + 1] - du2[t] * x[t + 2]) / dd[t];
          }
          __syncwarp();
          // max-scale (squares cannot overflow), then unit norm
          T xmax = 0;
          for (int t = lane; t < s; t += 32) xmax = fmax(xmax, fabs(x[t]));
          for (int o = 16; o > 0; o >>= 1) xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
          if (!(xmax <= (T)3e38)) xmax = 0;  // inf or NaN: restart from a unit vector
          const T sx = xmax > (T)0 ? (T)1 / xmax : (T)0;
          for (int t = lane; t < s; t += 32) x[t] = xmax > (T)0 ? x[t] * sx : (T)(t == 0);
          __syncwarp();
          T nrm = 0;
          for (int t = lane; t < s; t += 32) nrm += x[t] * x[t];
          for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
          const T inv = nrm > (T)0 ? (T)1 / sqrt(nrm) : (T)1;
          for (int t = lane; t < s; t += 32) x[t] *= inv;
          __syncwarp();
        }
        for (int t = lane; t < s; t += 32) z[lo + t] = x[t];
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // ---- 4b. modified Gram-Schmidt over the needed vectors, in rank order --------
  // Vectors of one block and well-separated eigenvalues are orthogonal already
  // (the projections are at rounding level); near-equal eigenvalues get an
  // orthonormal basis of their common invariant subspace.
  {
    __shared__ T s_inv;
    __shared__ T s_dot[TRI_MAXM];
    const int nw = blockDim.x >> 5;
    // z_i -= sum_{j < i} (z_j . z_i) z_j (classical Gram-Schmidt against every earlier,
    // finished vector; dots first, then one pass over the rows)
    auto reorth = [&](T* zi, int i) {
      for (int j = warp; j < i; j += nw) {
        const T* zj = gZ + (size_t)j * m;
        T dot = 0;
        for (int t = lane; t < m; t += 32) dot += zj[t] * zi[t];
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) s_dot[j] = dot;
      }
      __syncthreads();
      for (int t = tid; t < m; t += blockDim.x) {
        T acc = zi[t];
        for (int j = 0; j < i; ++j) acc -= s_dot[j] * gZ[(size_t)j * m + t];
        zi[t] = acc;
      }
      __syncthreads();
    };
    for (int i = 0; i < nvec; ++i) {
      T* zi = gZ + (size_t)i * m;
      T part = 0;
      for (int t = tid; t < m; t += blockDim.x) part += zi[t] * zi[t];
      T nrm = block_reduce(part, red);
      // A vector that lost most of its (unit) norm to the earlier ones (inverse iteration
      // on eigenvalues the FP32 arithmetic does not separate, e.g. a cluster in the noise
      // floor, returns nearly parallel vectors): one modified Gram-Schmidt pass leaves
      // its remainder far from orthogonal, so it is orthogonalised twice more against
      // every earlier vector; if nothing is left, a pseudo-random vector takes its place
      // (any direction is an eigenvector to the FP32 solve's resolution there).
      if (nrm < (T)0.25) {
        for (int pass = 0; pass < 3; ++pass) {
          if (pass == 2 || !(nrm > (T)1e-12)) {
            if (pass == 2 && nrm > (T)1e-12) break;
            for (int t = tid; t < m; t += blockDim.x) {
              unsigned h = (unsigned)(t + 1) * 2654435761u ^ ((unsigned)(i + 7919) * 40503u + 0x85ebca6bu);
              h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
              zi[t] = (T)(h & 0xffffu) * (T)(1.0 / 65536.0) - (T)0.5;
            }
            __syncthreads();
            reorth(zi, i);
          }
          reorth(zi, i);
          part = 0;
          for (int t = tid; t < m; t += blockDim.x) part += zi[t] * zi[t];
          nrm = block_reduce(part, red);
        }
      }
      if (tid == 0) s_inv = nrm > (T)0 ? (T)1 / sqrt(nrm) : (T)0;
      __syncthreads();
      const T inv = s_inv;
      for (int t = tid; t < m; t += blockDim.x) zi[t] *= inv;
      __syncthreads();
      for (int j = i + 1 + warp; j < nvec; j += (blockDim.x >> 5)) {
        T* zj = gZ + (size_t)j * m;
        T dot = 0;
        for (int t = lane; t < m; t += 32) dot += zi[t] * zj[t];
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        for (int t = lane; t < m; t += 32) zj[t] -= dot * zi[t];
      }
      __syncthreads();
    }
  }

  // ---- 5. back-transform: y = H_0 (H_1 (... H_{m-2} z)) ----------------------
  // Each warp owns output columns (ranks); reflectors are staged in shared
  // memory TRI_CHUNK at a time, from the last to the first.
  {
    cx<T>* sref = (cx<T>*)smem_raw;        // TRI_CHUNK reflectors, each m long (row-indexed)
    cx<T>* ycols = sref + TRI_CHUNK * m;    // per-warp working column (m)
    const int nw = blockDim.x >> 5;
    cx<T>* y = ycols + (size_t)warp * m;
    // the columns a warp handles are processed in rounds so all warps stay in step
    for (int base = 0; base < nvec; base += nw) {
      const int col = base + warp;
      const bool active = col < nvec;
      if (active) {
        const T* zc = gZ + (size_t)col * m;
        for (int t = lane; t < m; t += 32) y[t] = mk<T>(zc[t], 0);
      }
      for (int jend = m - 2; jend >= 0; jend -= TRI_CHUNK) {
        const int jbeg = jend - TRI_CHUNK + 1 < 0 ? 0 : jend - TRI_CHUNK + 1;
        __syncthreads();
        for (int jj = jbeg; jj <= jend; ++jj) {
          cx<T>* dst = sref + (size_t)(jj - jbeg) * m;
          const cx<T>* src = gpacked + packed_off(jj, m);
          for (int t = tid; t < m; t += blockDim.x) {
            cx<T> v = mk<T>(0, 0);
            if (t == jj + 1) v = mk<T>(1, 0);
            else if (t > jj + 1) v = src[t - jj];
            dst[t] = v;
          }
        }
        __syncthreads();
        if (active) {
          for (int jj = jend; jj >= jbeg; --jj) {
            const cx<T> tau = stau[jj];
            if (tau.x == (T)0 && tau.y == (T)0) continue;
            const cx<T>* v = sref + (size_t)(jj - jbeg) * m;
            // s = v^dag y (rows jj+1..m-1)
            T sr = 0, si = 0;
            for (int t = jj + 1 + lane; t < m; t += 32) {
              const cx<T> a = v[t], b = y[t];
              sr += a.x * b.x + a.y * b.y;
              si += a.x * b.y - a.y * b.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
              sr += __shfl_xor_sync(0xffffffffu, sr, o);
              si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            const cx<T> f = cmul(tau, mk<T>(sr, si));
            for (int t = jj + 1 + lane; t < m; t += 32) y[t] = csub(y[t], cmul(f, v[t]));
            __syncwarp();
          }
        }
      }
      if (active) {
        // reflectors in T are unitary only to O(m eps); renormalise so the kept
        // mass u^dag G u carries no systematic norm error
        double nrm = 0.0;
        for (int t = lane; t < m; t += 32) nrm += (double)y[t].x * y[t].x + (double)y[t].y * y[t].y;
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
        for (int t = lane; t < m; t += 32) {
          const double2 v = to_d2(y[t]);
          evecs[(size_t)t * m + col] = make_double2(v.x * inv, v.y * inv);
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    const long long t = clock64();
    t_ph[4] = t - t_mark;
    for (int p = 0; p < 5; ++p) out->cycles[p] = t_ph[p];
  }
}

template <typename T>
__global__ void __launch_bounds__(TRI_THREADS) k_eigh_tri(const double2* __restrict__ G, int m, int c_split,
                                                          cx<T>* gpacked, T* gZ, double* __restrict__ evals,
                                                          double2* __restrict__ evecs, EigOut* __restrict__ out,
                                                          int r, double eps, int all_vecs) {
  eigh_tri_body<T>(G, m, c_split, gpacked, gZ, evals, evecs, out, r, eps, all_vecs);
}

constexpr size_t TRI_DYN_MAX = 180 * 1024;

// smallest c such that packed columns c..m-1 fit in the budget
__host__ __device__ __forceinline__ int tri_split_for(int m, size_t elem, size_t budget) {
  for (int c = 0; c < m; ++c)
    if ((size_t)(packed_off(m, m) - packed_off(c, m)) * elem <= budget) return c;
  return m;
}

// one circuit's eigensolve per block (task tasks[sel[blockIdx.x]]); every eigenvector
// only where a refinement follows
template <typename T>
__global__ void __launch_bounds__(TRI_THREADS)
    k_eigh_tri_batch(const TruncTask* __restrict__ tasks, const int* __restrict__ sel, int all_vecs) {
  const TruncTask& tk = tasks[sel[blockIdx.x]];
  const int m = tk.m;
  const int c_split = tri_split_for(m, sizeof(cx<T>), TRI_DYN_MAX);
  cx<T>* gpacked = (cx<T>*)tk.eigwork;
  T* gZ = (T*)(gpacked + packed_off(m, m));
  eigh_tri_body<T>(tk.G, m, c_split, gpacked, gZ, tk.evals, tk.evecs, tk.eo, tk.k, 0.0, all_vecs);
}

template <typename T>
cudaError_t prepare_eigh_tri_batch() {
  return cudaFuncSetAttribute(k_eigh_tri_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRI_DYN_MAX);
}

// prepare_eigh_tri_batch<T>() must have run once (it is not a stream operation,
// so it stays outside graph capture)
template <typename T>
cudaError_t launch_eigh_tri_batch(const TruncTask* tasks, const int* sel, int nsel, int all_vecs, cudaStream_t s) {
  if (nsel <= 0) return cudaSuccess;
  k_eigh_tri_batch<T><<<nsel, TRI_THREADS, TRI_DYN_MAX, s>>>(tasks, sel, all_vecs);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t prepare_eigh_tri_batch<float>();
template cudaError_t prepare_eigh_tri_batch<double>();
template cudaError_t launch_eigh_tri_batch<float>(const TruncTask*, const int*, int, int, cudaStream_t);
template cudaError_t launch_eigh_tri_batch<double>(const TruncTask*, const int*, int, int, cudaStream_t);

template <typename T>
static int tri_c_split(int m, size_t budget) {
  // smallest c such that columns c..m-1 (packed) fit in the budget
  for (int c = 0; c < m; ++c) {
    const size_t bytes = (size_t)(packed_off(m, m) - packed_off(c, m)) * sizeof(cx<T>);
    if (bytes <= budget) return c;
  }
  return m;
}

template <typename T>
size_t tri_smem_bytes(int m) {
  const size_t lu = (size_t)LuWarps<T>::v * 6 * TRI_MAXM * sizeof(T);
  const size_t bt = (size_t)(TRI_CHUNK + TRI_THREADS / 32) * m * sizeof(cx<T>);
  return lu > bt ? lu : bt;
}

template <typename T>
cudaError_t launch_eigh_tri(const double2* G, int m, void* work, double* evals, double2* evecs, EigOut* out,
                            int r, double eps, int all_vecs, cudaStream_t s) {
  if (m > TRI_MAXM || m < 1) return cudaErrorInvalidValue;
  const size_t dyn_max = 180 * 1024;
  size_t need_min = tri_smem_bytes<T>(m);
  const int c_split = tri_c_split<T>(m, dyn_max);
  size_t packed_smem = (size_t)(packed_off(m, m) - packed_off(c_split, m)) * sizeof(cx<T>);
  size_t dyn = packed_smem > need_min ? packed_smem : need_min;
  if (dyn > dyn_max) dyn = dyn_max;
  cudaError_t e = cudaFuncSetAttribute(k_eigh_tri<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
  if (e != cudaSuccess) return e;
  cx<T>* gpacked = (cx<T>*)work;
  T* gZ = (T*)(gpacked + packed_off(m, m));
  k_eigh_tri<T><<<1, TRI_THREADS, dyn, s>>>(G, m, c_split, gpacked, gZ, evals, evecs, out, r, eps, all_vecs);
  note_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_eigh_tri<float>(const double2*, int, void*, double*, double2*, EigOut*, int, double,
                                            int, cudaStream_t);
template cudaError_t launch_eigh_tri<double>(const double2*, int, void*, double*, double2*, EigOut*, int, double,
                                             int, cudaStream_t);

}  // namespace lret
