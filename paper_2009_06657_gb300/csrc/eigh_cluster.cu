// Hermitian eigensolver of the truncation (Sec. II.B, Theorem 1) on a thread
// block cluster: the same method as eigh_tri.cu (Householder reduction to a
// real tridiagonal T, bisection, inverse iteration, orthonormalisation,
// back-transform), spread over CL = 8 CTAs (8 SMs) with distributed shared
// memory.
//
// Data layout: the full Hermitian matrix (G / trace, both triangles) is held in
// shared memory by rows, row i in CTA i % CL (m / CL rows per CTA, at most
// 32 x 256 complex). Step j of the reduction:
//   * the owner of row j forms x = conj(A[j][j+1:]) (= column j below the
//     diagonal), the reflector H_j = I - tau v v^dag with H_j^dag x = beta e_1,
//     and writes v and tau into every CTA's shared memory;           [barrier]
//   * every CTA forms p_i = tau sum_c A[i][c] v_c for its rows, writes them and
//     its share of v^dag p into every CTA;                           [barrier]
//   * every CTA forms w = p - (1/2) conj(tau) (v^dag p) v and updates its rows,
//     A[i][c] -= v_i conj(w_c) + w_i conj(v_c).
// v and p live in two alternating buffers, so two cluster barriers per step
// suffice. The reflectors are also written to global memory for the
// back-transform. Eigenvalue bisection, inverse iteration and the
// back-transform are divided over the CTAs by eigenvalue / vector index; the
// orthonormalisation of the kept vectors (modified Gram-Schmidt, sequential in
// the vector index) runs on CTA 0.
#include <cooperative_groups.h>
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace lret {

namespace {

constexpr int CL = 8;
constexpr int CL_THREADS = 512;
constexpr int CL_MAXM = 256;
constexpr int CL_ROWS = CL_MAXM / CL;  // rows per CTA at most

template <typename T> struct CEps;
template <> struct CEps<float> { static constexpr float v = FLT_EPSILON; static constexpr float tiny = 1e-30f; };
template <> struct CEps<double> { static constexpr double v = DBL_EPSILON; static constexpr double tiny = 1e-290; };

__device__ __forceinline__ float cdivq(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double cdivq(double a, double b) { return a / b; }

template <typename T>
__device__ int sturm_count(const T* d, const T* e2, int lo, int hi, T x, T pivmin) {
  int cnt = 0;
  T q = d[lo] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = lo + 1; i <= hi; ++i) {
    q = d[i] - x - cdivq(e2[i - 1], q);
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
struct ClusterShared {
  cx<T> A[CL_ROWS][CL_MAXM];  // this CTA's rows (row i = CL * li + rank)
  cx<T> v[2][CL_MAXM];        // reflector of step j in buffer j & 1 (rows j+1..m-1)
  cx<T> p[2][CL_MAXM];
  T dotp[2][CL][2];           // per-CTA shares of v^dag p (re, im)
  cx<T> tau[2];
  T d[CL_MAXM], e[CL_MAXM], e2[CL_MAXM], lam[CL_MAXM];
  short sblo[CL_MAXM], sbhi[CL_MAXM], order[CL_MAXM];
  T red[32];
  int k;
  double trace, dred[32];
};

}  // namespace

template <typename T>
__global__ void __launch_bounds__(CL_THREADS, 1)
    k_eigh_cluster(const double2* __restrict__ G, int m, cx<T>* __restrict__ gref, T* __restrict__ gZ,
                   double* __restrict__ evals, double2* __restrict__ evecs, EigOut* __restrict__ out, int r,
                   double eps, int all_vecs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ClusterShared<T>& sh = *reinterpret_cast<ClusterShared<T>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = CL_THREADS / 32;
  const int nrows = (m - rank + CL - 1) / CL;  // rows rank, rank + CL, ...
  ClusterShared<T>* peer[CL];
#pragma unroll
  for (int q = 0; q < CL; ++q) peer[q] = cluster.map_shared_rank(&sh, q);

  // ---- load G / trace (every CTA its rows) --------------------------------
  double tr = 0.0;
  for (int i = tid; i < m; i += CL_THREADS) tr += G[(size_t)i * m + i].x;
  tr = block_sum(tr, sh.dred);
  if (tid == 0) sh.trace = tr;
  __syncthreads();
  const double gscale = sh.trace > 0.0 ? sh.trace : 1.0;
  const double ginv = 1.0 / gscale;
  for (int e = tid; e < nrows * m; e += CL_THREADS) {
    const int li = e / m, col = e % m;
    const int i = li * CL + rank;
    const double2 g = G[(size_t)i * m + col];
    sh.A[li][col] = mk<T>((T)(g.x * ginv), (T)(g.y * ginv));
  }
  cluster.sync();

  // ---- reduction to tridiagonal form ----------------------------------------
  for (int j = 0; j < m - 1; ++j) {
    const int n1 = m - j - 1;
    const int buf = j & 1;
    const int owner = j % CL;
    if (rank == owner) {
      // x = conj(A[j][j+1:]), alpha = x_0; scaled norms (no underflow)
      const int lj = j / CL;
      T amax = 0, part = 0;
      for (int t = tid; t < n1; t += CL_THREADS) {
        const cx<T> a = sh.A[lj][j + 1 + t];
        amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
        if (t >= 1) part += a.x * a.x + a.y * a.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        part += __shfl_xor_sync(0xffffffffu, part, o);
      }
      __syncthreads();
      if (lane == 0) { sh.red[warp] = amax; sh.lam[warp] = part; }  // lam used as scratch here
      __syncthreads();
      __shared__ cx<T> s_tau, s_scale;
      __shared__ T s_beta;
      if (tid == 0) {
        T am = 0, x2 = 0;
        for (int w = 0; w < nw; ++w) { am = fmax(am, sh.red[w]); x2 += sh.lam[w]; }
        const cx<T> alpha = conjg(sh.A[lj][j + 1]);
        const T inv = am > (T)0 ? (T)1 / am : (T)0;
        T xn2s = x2 * inv * inv;
        if (am > (T)0 && x2 < (T)1e-30) {  // squares may have underflowed
          T sacc = 0;
          for (int t = 1; t < n1; ++t) {
            const cx<T> a = sh.A[lj][j + 1 + t];
            sacc += (a.x * inv) * (a.x * inv) + (a.y * inv) * (a.y * inv);
          }
          xn2s = sacc;
        }
        cx<T> tau, scale;
        T beta;
        if (am <= (T)1e-30 || (xn2s == (T)0 && alpha.y == (T)0)) {
          tau = mk<T>(0, 0);
          beta = alpha.x;
          scale = mk<T>(0, 0);
        } else {
          const T ar = alpha.x * inv, ai = alpha.y * inv;
          const T bs = -copysign(sqrt(ar * ar + ai * ai + xn2s), ar);
          beta = am * bs;
          tau = mk<T>((bs - ar) / bs, -ai / bs);
          const T den = (ar - bs) * (ar - bs) + ai * ai;
          scale = mk<T>((ar - bs) / den * inv, -ai / den * inv);
        }
        s_tau = tau;
        s_scale = scale;
        s_beta = beta;
      }
      __syncthreads();
      const cx<T> tau = s_tau, scale = s_scale;
      // v (rows j+1..m-1; v_{j+1} = 1) to every CTA and to global memory
      cx<T>* gv = gref + (size_t)j * CL_MAXM;
      for (int t = tid; t < n1; t += CL_THREADS) {
        const cx<T> vt = t == 0 ? mk<T>(1, 0) : cmul(conjg(sh.A[lj][j + 1 + t]), scale);
        gv[t] = vt;
#pragma unroll
        for (int q = 0; q < CL; ++q) peer[q]->v[buf][j + 1 + t] = vt;
      }
      if (tid < CL) peer[tid]->tau[buf] = tau;
      if (tid == 0) {
        // diagonal, off-diagonal and tau of T for every CTA
        const T dj = sh.A[lj][j].x, be = s_beta;
        for (int q = 0; q < CL; ++q) {
          peer[q]->d[j] = dj;
          peer[q]->e[j] = be;
        }
        reinterpret_cast<cx<T>*>(gref + (size_t)(CL_MAXM - 1) * CL_MAXM)[j] = tau;  // tau row of gref
      }
    }
    cluster.sync();
    const cx<T> tau = sh.tau[buf];
    const bool skip = (tau.x == (T)0 && tau.y == (T)0);
    // p_i = tau sum_c A[i][c] v_c for local rows i > j; v^dag p share
    T dr = 0, di = 0;
    if (!skip) {
      for (int li = warp; li < nrows; li += nw) {
        const int i = li * CL + rank;
        if (i <= j) continue;
        cx<T> acc = mk<T>(0, 0);
        for (int col = j + 1 + lane; col < m; col += 32) cfma(acc, sh.A[li][col], sh.v[buf][col]);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        const cx<T> pi = cmul(tau, acc);
        if (lane < CL) peer[lane]->p[buf][i] = pi;
        if (lane == 0) {
          const cx<T> vi = sh.v[buf][i];
          dr += vi.x * pi.x + vi.y * pi.y;  // Re conj(v_i) p_i
          di += vi.x * pi.y - vi.y * pi.x;  // Im conj(v_i) p_i
        }
      }
    }
    if (lane == 0) { sh.red[warp] = dr; sh.lam[warp] = di; }
    __syncthreads();
    if (tid == 0) {
      T sr = 0, si = 0;
      for (int w = 0; w < nw; ++w) { sr += sh.red[w]; si += sh.lam[w]; }
      for (int q = 0; q < CL; ++q) {
        peer[q]->dotp[buf][rank][0] = sr;
        peer[q]->dotp[buf][rank][1] = si;
      }
    }
    cluster.sync();
    if (!skip) {
      T sr = 0, si = 0;
#pragma unroll
      for (int q = 0; q < CL; ++q) { sr += sh.dotp[buf][q][0]; si += sh.dotp[buf][q][1]; }
      const T cc = (T)0.5 * (tau.x * sr + tau.y * si);
      // w = p - c v (full vector, every CTA); kept in p[buf]
      for (int t = tid; t < n1; t += CL_THREADS) {
        const int col = j + 1 + t;
        sh.p[buf][col] = csub(sh.p[buf][col], cscale(sh.v[buf][col], cc));
      }
      __syncthreads();
      // rank-2 update of local rows i > j (full rows, columns > j)
      for (int li = warp; li < nrows; li += nw) {
        const int i = li * CL + rank;
        if (i <= j) continue;
        const cx<T> vi = sh.v[buf][i], wi = sh.p[buf][i];
        for (int col = j + 1 + lane; col < m; col += 32) {
          cx<T> a = sh.A[li][col];
          a = csub(a, cadd(cmul(vi, conjg(sh.p[buf][col])), cmul(wi, conjg(sh.v[buf][col]))));
          if (col == i) a.y = 0;
          sh.A[li][col] = a;
        }
      }
    }
    __syncthreads();
  }
  if (rank == (m - 1) % CL && tid == 0) {
    const T dl = sh.A[(m - 1) / CL][m - 1].x;
    for (int q = 0; q < CL; ++q) {
      peer[q]->d[m - 1] = dl;
      peer[q]->e[m - 1] = 0;
    }
  }
  cluster.sync();

  // ---- split, bisection (eigenvalues t = rank, rank + CL, ...) ---------------
  __shared__ T s_tnorm, s_pivmin;
  if (tid == 0) {
    T tn = 0, emax2 = 0;
    for (int i = 0; i < m; ++i) {
      const T a = fabs(sh.d[i]) + (i > 0 ? fabs(sh.e[i - 1]) : (T)0) + (i < m - 1 ? fabs(sh.e[i]) : (T)0);
      tn = a > tn ? a : tn;
    }
    for (int i = 0; i < m - 1; ++i) {
      if (fabs(sh.e[i]) <= CEps<T>::v * (fabs(sh.d[i]) + fabs(sh.d[i + 1])) ||
          fabs(sh.e[i]) <= CEps<T>::v * CEps<T>::v * tn)
        sh.e[i] = 0;
      sh.e2[i] = sh.e[i] * sh.e[i];
      emax2 = sh.e2[i] > emax2 ? sh.e2[i] : emax2;
    }
    int lo = 0;
    for (int i = 0; i < m; ++i)
      if (i == m - 1 || sh.e[i] == (T)0) {
        for (int t = lo; t <= i; ++t) { sh.sblo[t] = (short)lo; sh.sbhi[t] = (short)i; }
        lo = i + 1;
      }
    s_tnorm = tn > (T)0 ? tn : (T)1;
    s_pivmin = CEps<T>::tiny * (emax2 > (T)1 ? emax2 : (T)1);
  }
  __syncthreads();
  const T tnorm = s_tnorm, pivmin = s_pivmin;
  for (int t = rank + CL * tid; t < m; t += CL * CL_THREADS) {
    const int lo = sh.sblo[t], hi = sh.sbhi[t], li = t - lo;
    T gl = sh.d[lo], gu = sh.d[lo];
    for (int i = lo; i <= hi; ++i) {
      const T rad = (i > lo ? fabs(sh.e[i - 1]) : (T)0) + (i < hi ? fabs(sh.e[i]) : (T)0);
      gl = fmin(gl, sh.d[i] - rad);
      gu = fmax(gu, sh.d[i] + rad);
    }
    T a = gl - CEps<T>::v * tnorm * 2 - pivmin, b = gu + CEps<T>::v * tnorm * 2 + pivmin;
    for (int it = 0; it < 100; ++it) {
      const T mid = (T)0.5 * (a + b);
      if (b - a <= (T)2 * CEps<T>::v * fmax(fabs(a), fabs(b)) + CEps<T>::v * tnorm * (T)1e-3 || mid == a || mid == b)
        break;
      if (sturm_count<T>(sh.d, sh.e2, lo, hi, mid, pivmin) <= li) a = mid; else b = mid;
    }
    T lt = (T)0.5 * (a + b);
    if (!(lt == lt)) lt = -INFINITY;
    for (int q = 0; q < CL; ++q) peer[q]->lam[t] = lt;
  }
  cluster.sync();

  // ---- sort (every CTA), rank choice and accounting (CTA 0) -------------------
  for (int t = tid; t < m; t += CL_THREADS) {
    const T lt = sh.lam[t];
    int rk = 0;
    for (int u = 0; u < m; ++u) {
      const T lu = sh.lam[u];
      rk += (lu > lt) || (lu == lt && u < t);
    }
    sh.order[rk] = (short)t;
    if (rank == 0) evals[rk] = (double)lt * gscale;
  }
  __syncthreads();
  if (tid == 0) {
    int k;
    double total = 0.0;
    for (int i = 0; i < m; ++i) {
      const double v = (double)sh.lam[sh.order[i]] * gscale;
      total += v > 0 ? v : 0.0;
    }
    if (r > 0) {
      k = r < m ? r : m;
    } else {
      double cs = 0.0;
      k = m;
      for (int i = 0; i < m; ++i) {
        const double v = (double)sh.lam[sh.order[i]] * gscale;
        cs += v > 0 ? v : 0.0;
        if (cs >= (1.0 - eps) * total) { k = i + 1; break; }
      }
    }
    sh.k = k;
    if (rank == 0) {
      double kept = 0.0, dropped = 0.0;
      for (int i = 0; i < m; ++i) {
        const double v = (double)sh.lam[sh.order[i]] * gscale;
        if (i < k) kept += v > 0 ? v : 0.0; else dropped += v > 0 ? v : 0.0;
      }
      const double l1v = (double)sh.lam[sh.order[0]] * gscale;
      const double l1 = fabs(l1v) > 0 ? fabs(l1v) : 1.0;
      out->k = k;
      out->sweeps = 0;
      out->status = isfinite(l1v) ? 0 : 2;
      out->dropped = dropped;
      out->kept = kept;
      out->gap = k < m ? ((double)sh.lam[sh.order[k - 1]] - (double)sh.lam[sh.order[k]]) * gscale / l1
                       : __longlong_as_double(0x7ff0000000000000ll);
      out->trace = sh.trace;
    }
  }
  __syncthreads();
  const int nvec = all_vecs ? m : sh.k;

  // ---- inverse iteration: vectors i = rank + CL * (warp + nw * ...) ---------
  {
    // per-warp LU scratch reuses this CTA's matrix rows (no longer needed)
    T* ws = reinterpret_cast<T*>(&sh.A[0][0]);
    constexpr int SLOT = 6 * CL_MAXM;
    const int nlu = (int)(sizeof(sh.A) / (SLOT * sizeof(T)));
    if (warp < nlu) {
      T* dl = ws + (size_t)warp * SLOT;
      T* dd = dl + CL_MAXM;
      T* du = dd + CL_MAXM;
      T* du2 = du + CL_MAXM;
      T* x = du2 + CL_MAXM;
      unsigned char* piv = reinterpret_cast<unsigned char*>(x + CL_MAXM);
      const int wn = nlu < nw ? nlu : nw;
      for (int i = rank + CL * warp; i < nvec; i += CL * wn) {
        const int pos = sh.order[i];
        const int lo = sh.sblo[pos], hi = sh.sbhi[pos], s = hi - lo + 1;
        T* z = gZ + (size_t)i * m;
        for (int t = lane; t < m; t += 32) z[t] = 0;
        __syncwarp();
        if (s == 1) {
          if (lane == 0) z[lo] = 1;
          __syncwarp();
          continue;
        }
        const T lam = sh.lam[pos];
        if (lane == 0) {
          const T tiny = CEps<T>::v * tnorm;
          for (int t = 0; t < s; ++t) {
            dd[t] = sh.d[lo + t] - lam;
            if (t < s - 1) { dl[t] = sh.e[lo + t]; du[t] = sh.e[lo + t]; du2[t] = 0; }
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
              if (t < s - 2) { du2[t] = du[t + 1]; du[t + 1] = -l * du[t + 1]; }
              piv[t] = 1;
            }
          }
          if (dd[s - 1] == (T)0) dd[s - 1] = tiny;
        }
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
          T xmax = 0;
          for (int t = lane; t < s; t += 32) xmax = fmax(xmax, fabs(x[t]));
          for (int o = 16; o > 0; o >>= 1) xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
          if (!(xmax <= (T)3e38)) xmax = 0;
          const T sx = xmax > (T)0 ? (T)1 / xmax : (T)0;
          for (int t = lane; t < s; t += 32) x[t] = xmax > (T)0 ? x[t] * sx : (T)(t == 0);
          __syncwarp();
          T nrm = 0;
          for (int t = lane; t < s; t += 32) nrm += x[t] * x[t];
          nrm = warp_sum(nrm);
          const T inv = nrm > (T)0 ? (T)1 / sqrt(nrm) : (T)1;
          for (int t = lane; t < s; t += 32) x[t] *= inv;
          __syncwarp();
        }
        for (int t = lane; t < s; t += 32) z[lo + t] = x[t];
        __syncwarp();
      }
    }
  }
  __threadfence();
  cluster.sync();

  // ---- modified Gram-Schmidt of the needed vectors (CTA 0) --------------------
  if (rank == 0) {
    __shared__ T s_inv;
    for (int i = 0; i < nvec; ++i) {
      T* zi = gZ + (size_t)i * m;
      T part = 0;
      for (int t = tid; t < m; t += CL_THREADS) part += zi[t] * zi[t];
      part = warp_sum(part);
      if (lane == 0) sh.red[warp] = part;
      __syncthreads();
      if (tid == 0) {
        T nrm = 0;
        for (int w = 0; w < nw; ++w) nrm += sh.red[w];
        s_inv = nrm > (T)0 ? (T)1 / sqrt(nrm) : (T)0;
      }
      __syncthreads();
      const T inv = s_inv;
      for (int t = tid; t < m; t += CL_THREADS) zi[t] *= inv;
      __syncthreads();
      for (int jv = i + 1 + warp; jv < nvec; jv += nw) {
        T* zj = gZ + (size_t)jv * m;
        T dot = 0;
        for (int t = lane; t < m; t += 32) dot += zi[t] * zj[t];
        dot = warp_sum(dot);
        for (int t = lane; t < m; t += 32) zj[t] -= dot * zi[t];
      }
      __syncthreads();
    }
    __threadfence();
  }
  cluster.sync();

  // ---- back-transform y = H_0 (... (H_{m-2} z)); columns i = rank + CL * w ------
  {
    const cx<T>* taus = reinterpret_cast<const cx<T>*>(gref + (size_t)(CL_MAXM - 1) * CL_MAXM);
    cx<T>* y = reinterpret_cast<cx<T>*>(&sh.A[0][0]) + (size_t)warp * CL_MAXM;  // per-warp column
    for (int col = rank + CL * warp; col < nvec; col += CL * nw) {
      const T* zc = gZ + (size_t)col * m;
      for (int t = lane; t < m; t += 32) y[t] = mk<T>(zc[t], 0);
      __syncwarp();
      for (int jj = m - 2; jj >= 0; --jj) {
        const cx<T> tau = taus[jj];
        if (tau.x == (T)0 && tau.y == (T)0) continue;
        const cx<T>* v = gref + (size_t)jj * CL_MAXM;  // v[t] for row jj + 1 + t
        T sr = 0, si = 0;
        for (int t = lane; t < m - jj - 1; t += 32) {
          const cx<T> a = v[t], b = y[jj + 1 + t];
          sr += a.x * b.x + a.y * b.y;
          si += a.x * b.y - a.y * b.x;
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        const cx<T> f = cmul(tau, mk<T>(sr, si));
        for (int t = lane; t < m - jj - 1; t += 32) y[jj + 1 + t] = csub(y[jj + 1 + t], cmul(f, v[t]));
        __syncwarp();
      }
      double nrm = 0.0;
      for (int t = lane; t < m; t += 32) nrm += (double)y[t].x * y[t].x + (double)y[t].y * y[t].y;
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
      for (int t = lane; t < m; t += 32) {
        const double2 vv = to_d2(y[t]);
        evecs[(size_t)t * m + col] = make_double2(vv.x * inv, vv.y * inv);
      }
      __syncwarp();
    }
  }
  cluster.sync();
}

template <typename T>
size_t eigh_cluster_smem() {
  return sizeof(ClusterShared<T>);
}

template <typename T>
cudaError_t launch_eigh_cluster(const double2* G, int m, void* work, double* evals, double2* evecs, EigOut* out,
                                int r, double eps, int all_vecs, cudaStream_t s) {
  if (m < 2 || m > CL_MAXM) return cudaErrorInvalidValue;
  const size_t smem = sizeof(ClusterShared<T>);
  static bool attr[2] = {false, false};
  if (!attr[sizeof(T) == 8]) {
    cudaError_t e = cudaFuncSetAttribute(k_eigh_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr[sizeof(T) == 8] = true;
  }
  // work: reflectors (CL_MAXM x CL_MAXM complex; last row holds tau) then Z (m x m real)
  cx<T>* gref = (cx<T>*)work;
  T* gZ = (T*)(gref + (size_t)CL_MAXM * CL_MAXM);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(CL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_eigh_cluster<T>, G, m, gref, gZ, evals, evecs, out, r, eps, all_vecs);
}

size_t eigh_cluster_work_bytes(bool fp64) {
  const size_t e = fp64 ? sizeof(double) : sizeof(float);
  return (size_t)CL_MAXM * CL_MAXM * 2 * e + (size_t)CL_MAXM * CL_MAXM * e;
}

template cudaError_t launch_eigh_cluster<float>(const double2*, int, void*, double*, double2*, EigOut*, int, double,
                                                int, cudaStream_t);
template cudaError_t launch_eigh_cluster<double>(const double2*, int, void*, double*, double2*, EigOut*, int,
                                                 double, int, cudaStream_t);

}  // namespace lret
