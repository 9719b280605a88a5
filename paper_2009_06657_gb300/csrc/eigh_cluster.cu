// Hermitian eigensolver of the truncation (Sec. II.B, Theorem 1) on a thread
// block cluster: the same method as eigh_tri.cu (Householder reduction to a
// real tridiagonal T, bisection, inverse iteration, orthonormalisation,
// back-transform), spread over CL = 8 CTAs (8 SMs) with distributed shared
// memory.
//
// Data layout during the reduction: the Hermitian matrix G / trace (both
// triangles) is distributed by rows, row i in CTA i % CL, and held in registers:
// warp w of a CTA holds its local rows w and w + 16, lane l the columns l + 32 e
// (at most 32 rows x 256 columns per CTA). Every CTA holds the current reflector
// v_j, tau_j (H_j = I - tau v v^dag, H_j^dag x = beta e_1 for x = conj(A[j][j+1:])).
// Step j:
//   * every CTA forms p_i = tau sum_c A[i][c] v_c for its rows and sends them,
//     with one partial of v^dag p per warp, to every CTA           [barrier]
//   * every warp updates its rows, A[i][c] -= v_i conj(w_c) + w_i conj(v_c) with
//     w = p - (1/2) conj(tau)(v^dag p) v; the warp holding row j + 3 also stores
//     it in global memory;
//   * warps 0-3 (the reflector group) form v_{j+1}, tau_{j+1} from their shared-
//     memory copy of row j + 1 (stored by its owner two steps earlier, copied with
//     cp.async one step earlier) after applying the updates of steps j - 1 and j
//     to it, then start the copy of row j + 2. Every CTA computes the same
//     reflector, so there is no second exchange: one cluster barrier per step.
// The step state (v, p, partials, tau) rotates through three slots because a
// CTA may run one step ahead of another. One CTA also writes each reflector to
// global memory for the back-transform. A step costs about the same whatever the
// size of the trailing block (it is bound by the cluster barrier and the chain of
// the reflector), so the last TAIL_N steps run on CTA 0 alone: the trailing
// block is gathered into its shared memory and each step takes two block
// barriers (matvec; rank-2 update beside the next reflector).
//
// Eigenvalues: multisection (each eigenvalue is bracketed by 16 threads that
// evaluate the Sturm count at 16 interior points, a 17-fold shrink per round).
// Eigenvectors of T: inverse iteration, one warp per vector (the serial LU and
// solves carry their running values in registers); then modified Gram-Schmidt
// of the needed vectors on CTA 0 with the vectors held in registers (one
// barrier per vector). Back-transform y = H_0 (H_1 (... H_{m-2} z)): one warp per column,
// the column in registers, reflectors staged in shared memory 32 at a time (one
// bulk asynchronous copy per block) and
// applied in groups of 4 (FP32) or 2 (FP64): the group's inner products
// v_k^dag y are reduced together and corrected with the reflectors' own inner
// products v_k^dag v_l.
#include <cooperative_groups.h>
#include <float.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace lret {

namespace {

constexpr int CL = 8;
constexpr int CL_THREADS = 512;
constexpr int CL_NW = CL_THREADS / 32;
constexpr int CL_MAXM = 256;
constexpr int CL_ROWS = CL_MAXM / CL;  // rows per CTA at most
constexpr int MS = 16;                 // threads (and interior points) per eigenvalue in multisection
constexpr int TAIL_N = 90;             // trailing block finished by CTA 0 alone
static_assert(TAIL_N * TAIL_N <= CL_ROWS * CL_MAXM && TAIL_N <= 96, "trailing block: scratch A, 3 columns a lane");
constexpr int BT_STAGE = 32;           // reflectors staged per shared-memory block in the back-transform
template <typename T> struct BtGroup { static constexpr int v = 4; };  // reflectors applied together
template <> struct BtGroup<double> { static constexpr int v = 2; };  // (register budget of 512 threads)
// inverse-iteration scratch slots (6 m values each) beyond the 10 that fit in the
// matrix rows' shared memory, in extra dynamic shared memory: 6 more for FP32, so that
// all 16 warps of a CTA run one vector each (128 vectors per round over the cluster)
template <typename T> struct LuExtra { static constexpr int slots = 6; };
template <> struct LuExtra<double> { static constexpr int slots = 0; };
constexpr int MBK = CL_NW;                 // vectors per orthonormalisation block
constexpr int MSL = CL_MAXM / (MBK * CL);  // blocks a CTA owns at most (2)

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
  cx<T> A[CL_ROWS][CL_MAXM];  // this CTA's rows (row i = CL * li + rank); later scratch
  // state of step j in slot j % 3 (a step reads the slots of j and j - 1 while
  // faster CTAs already write slot j + 1)
  cx<T> v[3][CL_MAXM];        // reflector (rows j+1..m-1)
  cx<T> p[3][CL_MAXM];        // p = tau A v, all rows (each CTA sends its own)
  cx<T> dpart[3][CL * CL_NW]; // per-warp partials of v^dag p, all CTAs
  cx<T> tau[3];
  T ccs[3];                   // (1/2) Re(conj(tau) v^dag p)
  __align__(16) cx<T> nrow[2][CL_MAXM];  // prefetched copy of a future step's row
  T gred[4][2];               // reflector group: per-warp max and sum of squares
  cx<T> gscl;                 // reflector group: alpha
  cx<T> gram[BT_STAGE / BtGroup<T>::v][BtGroup<T>::v][BtGroup<T>::v];  // v_k^dag v_l, staged reflectors
  cx<T> btau[BT_STAGE];
  T d[CL_MAXM], e[CL_MAXM], e2[CL_MAXM], lam[CL_MAXM];
  short sblo[CL_MAXM], sbhi[CL_MAXM], order[CL_MAXM];
  int k;
  double trace, dred[32];
  unsigned long long mbar;    // back-transform staging (bulk copy completion)
#ifdef LRET_EIG_PROFILE
  long long gdbg[4];          // diagnostic build: reflector-group sub-steps
#endif
};

// The reflector group (warps 0-3) of every CTA forms the same v_{j+1},
// tau_{j+1} from row j + 1. The row's owner stored it in global memory during
// step j - 2 (as updated through that step); the group copied it into shared
// memory during step j - 1 (cp.async), and at step j applies the updates of
// steps j - 1 and j to it and forms H = I - tau v v^dag with H^dag x = beta e_1,
// x = conj(row[j+2:]) (scaled norms, no underflow).
constexpr int RG = 128;  // reflector group threads

__device__ __forceinline__ void bar_group() { asm volatile("barrier.sync 2, %0;" ::"n"(RG) : "memory"); }

// copy of columns [c0, m) of a stored row into shared memory, 16 bytes per cp.async
template <typename T>
__device__ __forceinline__ void prefetch_row(cx<T>* dst, const cx<T>* src, int c0, int m, int gt) {
  constexpr int PER = 16 / sizeof(cx<T>);
  for (int g = c0 / PER + gt; g < (m + PER - 1) / PER; g += RG) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + g * PER);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src + g * PER) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// row r's update of step s: a -= v_r conj(w_c) + w_r conj(v_c), w = p - cc v
template <typename T>
__device__ __forceinline__ cx<T> upd1(const ClusterShared<T>& sh, int sl, T cc, int r, int col, cx<T> a) {
  const cx<T> vr = sh.v[sl][r], vc = sh.v[sl][col];
  const cx<T> wr = csub(sh.p[sl][r], cscale(vr, cc)), wc = csub(sh.p[sl][col], cscale(vc, cc));
  return csub(a, cadd(cmul(vr, conjg(wc)), cmul(wr, conjg(vc))));
}

template <typename T>
__device__ void group_reflector(ClusterShared<T>& sh, const cx<T>* __restrict__ row, int jr, int m, int slv,
                                int sl0, bool up0, int sl1, bool up1, bool store, cx<T>* __restrict__ gref,
                                int gt) {
  const int lane = gt & 31, w = gt >> 5;
#ifdef LRET_EIG_PROFILE
  long long gq = clock64();
#define LRET_GSTEP(k) if (gt == 0) { const long long g2 = clock64(); sh.gdbg[k] += g2 - gq; gq = g2; }
#else
#define LRET_GSTEP(k)
#endif
  // this thread's entries of row jr: columns jr + gt and jr + gt + RG (the
  // diagonal, column jr, is entry 0)
  cx<T> x[2];
  T amax = 0, part = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int col = jr + gt + h * RG;
    cx<T> a = mk<T>(0, 0);
    if (col < m) {
      a = row[col];
      if (up0) a = upd1(sh, sl0, sh.ccs[sl0], jr, col, a);
      if (up1) a = upd1(sh, sl1, sh.ccs[sl1], jr, col, a);
      if (col == jr) a.y = 0;
      if (col > jr) {
        amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
        if (col > jr + 1) part += a.x * a.x + a.y * a.y;
      }
    }
    x[h] = a;
  }
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    part += __shfl_xor_sync(0xffffffffu, part, o);
  }
  if (lane == 0) { sh.gred[w][0] = amax; sh.gred[w][1] = part; }
  if (gt == 0) sh.d[jr] = x[0].x;
  if (gt == 1) sh.gscl = conjg(x[0]);  // alpha = conj(A[jr][jr+1]) (entry 1)
  LRET_GSTEP(0)
  bar_group();
  LRET_GSTEP(1)
  const T am = fmax(fmax(sh.gred[0][0], sh.gred[1][0]), fmax(sh.gred[2][0], sh.gred[3][0]));
  const T x2 = (sh.gred[0][1] + sh.gred[1][1]) + (sh.gred[2][1] + sh.gred[3][1]);
  const T inv = am > (T)0 ? (T)1 / am : (T)0;
  T xn2s = x2 * inv * inv;
  const cx<T> alpha = sh.gscl;
  if (am > (T)0 && x2 < (T)1e-30) {  // squares may have underflowed: sum scaled values
    T sacc = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = jr + gt + h * RG;
      if (col > jr + 1 && col < m) sacc += (x[h].x * inv) * (x[h].x * inv) + (x[h].y * inv) * (x[h].y * inv);
    }
    sacc = warp_sum(sacc);
    bar_group();
    if (lane == 0) sh.gred[w][1] = sacc;
    bar_group();
    xn2s = (sh.gred[0][1] + sh.gred[1][1]) + (sh.gred[2][1] + sh.gred[3][1]);
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
  LRET_GSTEP(2)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int col = jr + gt + h * RG;
    if (col > jr && col < m) sh.v[slv][col] = col == jr + 1 ? mk<T>(1, 0) : cmul(conjg(x[h]), scale);
  }
  if (store) {  // full-length row of the reflector store: zero outside jr+1..m-1
    cx<T>* gv = gref + (size_t)jr * CL_MAXM;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = jr + gt + h * RG;
      if (col > jr && col < m) gv[col] = col == jr + 1 ? mk<T>(1, 0) : cmul(conjg(x[h]), scale);
    }
    for (int rr = gt; rr <= jr; rr += RG) gv[rr] = mk<T>(0, 0);
    for (int rr = m + gt; rr < CL_MAXM; rr += RG) gv[rr] = mk<T>(0, 0);
    if (gt == 0) reinterpret_cast<cx<T>*>(gref + (size_t)(CL_MAXM - 1) * CL_MAXM)[jr] = tau;  // tau row
  }
  if (gt == 0) {
    sh.tau[slv] = tau;
    sh.e[jr] = beta;
  }
  LRET_GSTEP(3)
#undef LRET_GSTEP
}

// One warp forms v, tau from row jr of the trailing block (columns jr .. m - 1, at
// most 96 of them: lane l holds columns jr + l + 32 h) after applying the update
// of the current step, a -= v_r conj(w_c) + w_r conj(v_c) with r = jr; vv and ww
// hold v and w at the lane's columns. Same scalars as group_reflector. For
// jr = m - 1 only the last diagonal entry is formed.
template <typename T>
__device__ void warp_reflector(ClusterShared<T>& sh, const cx<T>* __restrict__ row, int jr, int m, int slv,
                               const cx<T> (&vv)[3], const cx<T> (&ww)[3], bool upd, cx<T>* __restrict__ gref,
                               int lane) {
  const cx<T> vr = mk<T>(__shfl_sync(0xffffffffu, vv[0].x, 0), __shfl_sync(0xffffffffu, vv[0].y, 0));
  const cx<T> wr = mk<T>(__shfl_sync(0xffffffffu, ww[0].x, 0), __shfl_sync(0xffffffffu, ww[0].y, 0));
  cx<T> x[3];
  T amax = 0, part = 0;
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const int col = jr + lane + 32 * h;
    cx<T> a = mk<T>(0, 0);
    if (col < m) {
      a = row[col];
      if (upd) a = csub(a, cadd(cmul(vr, conjg(ww[h])), cmul(wr, conjg(vv[h]))));
      if (col == jr) a.y = 0;
      if (col > jr) {
        amax = fmax(amax, fmax(fabs(a.x), fabs(a.y)));
        if (col > jr + 1) part += a.x * a.x + a.y * a.y;
      }
    }
    x[h] = a;
  }
  if (jr == m - 1) {  // last diagonal entry
    if (lane == 0) {
      sh.d[jr] = x[0].x;
      sh.e[jr] = 0;
    }
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    part += __shfl_xor_sync(0xffffffffu, part, o);
  }
  // alpha = conj(A[jr][jr+1]), entry h = 0 of lane 1
  const cx<T> alpha = mk<T>(__shfl_sync(0xffffffffu, x[0].x, 1), -__shfl_sync(0xffffffffu, x[0].y, 1));
  const T am = amax;
  const T inv = am > (T)0 ? (T)1 / am : (T)0;
  T xn2s = part * inv * inv;
  if (am > (T)0 && part < (T)1e-30) {  // squares may have underflowed: sum scaled values
    T sacc = 0;
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      const int col = jr + lane + 32 * h;
      if (col > jr + 1 && col < m) sacc += (x[h].x * inv) * (x[h].x * inv) + (x[h].y * inv) * (x[h].y * inv);
    }
    xn2s = warp_sum(sacc);
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
  cx<T>* gv = gref + (size_t)jr * CL_MAXM;  // full-length row of the reflector store
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const int col = jr + lane + 32 * h;
    if (col > jr && col < m) {
      const cx<T> v = col == jr + 1 ? mk<T>(1, 0) : cmul(conjg(x[h]), scale);
      sh.v[slv][col] = v;
      gv[col] = v;
    }
  }
  for (int rr = lane; rr <= jr; rr += 32) gv[rr] = mk<T>(0, 0);
  for (int rr = m + lane; rr < CL_MAXM; rr += 32) gv[rr] = mk<T>(0, 0);
  if (lane == 0) {
    sh.d[jr] = x[0].x;
    gref[(size_t)(CL_MAXM - 1) * CL_MAXM + jr] = tau;  // tau row
    sh.tau[slv] = tau;
    sh.e[jr] = beta;
  }
}

// Inverse iteration on rows lo..hi of the real tridiagonal T (diagonal sh.d,
// off-diagonal sh.e) with shift lam: LU with partial pivoting of T - lam I by lane 0
// (the recurrence is serial; running values in registers), then `iters` rounds of
// solve (lane 0) and normalisation (the warp). x holds the s = hi - lo + 1 start
// values and receives the result; sc is scratch of 6 CL_MAXM values (the factors in
// the first four, pivots in the sixth; x may be the fifth).
template <typename T>
__device__ void tri_inverse_iteration(const ClusterShared<T>& sh, int lo, int hi, T lam, T tnorm, T* __restrict__ sc,
                                      T* __restrict__ x, int iters, int lane) {
  const int s = hi - lo + 1;
  T* dl = sc;
  T* dd = dl + CL_MAXM;  // reciprocals of the LU diagonal
  T* du = dd + CL_MAXM;
  T* du2 = du + CL_MAXM;
  unsigned char* piv = reinterpret_cast<unsigned char*>(sc + 5 * CL_MAXM);
  if (lane == 0) {
    const T tiny = CEps<T>::v * tnorm;
    T cd = sh.d[lo] - lam, cu = sh.e[lo];
#pragma unroll 4
    for (int t = 0; t < s - 1; ++t) {
      const T sub = sh.e[lo + t];
      const T nd = sh.d[lo + t + 1] - lam;
      const T nu = t < s - 2 ? sh.e[lo + t + 1] : (T)0;
      if (fabs(cd) >= fabs(sub)) {
        if (cd == (T)0) cd = tiny;
        const T l = sub / cd;
        dl[t] = l; dd[t] = (T)1 / cd; du[t] = cu; du2[t] = 0; piv[t] = 0;
        cd = nd - l * cu;
        cu = nu;
      } else {
        const T l = cd / sub;
        dl[t] = l; dd[t] = (T)1 / sub; du[t] = nd; du2[t] = nu; piv[t] = 1;
        cd = cu - l * nd;
        cu = -l * nu;
      }
    }
    if (cd == (T)0) cd = tiny;
    dd[s - 1] = (T)1 / cd;
  }
  __syncwarp();
  for (int it = 0; it < iters; ++it) {
    if (lane == 0) {
      // forward (L with row swaps), then backward (U); carried values in registers
      T xt = x[0];
#pragma unroll 4
      for (int t = 0; t < s - 1; ++t) {
        const T xn = x[t + 1], l = dl[t];
        if (piv[t] == 0) {
          x[t] = xt;
          xt = xn - l * xt;
        } else {
          x[t] = xn;
          xt = xt - l * xn;
        }
      }
      T x1 = xt * dd[s - 1];  // x[t + 1]
      x[s - 1] = x1;
      T x2 = 0;               // x[t + 2]
#pragma unroll 4
      for (int t = s - 2; t >= 0; --t) {
        const T xv = (x[t] - du[t] * x1 - du2[t] * x2) * dd[t];
        x[t] = xv;
        x2 = x1;
        x1 = xv;
      }
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
}

// Out-of-line retry of a replacement vector that cancelled against the earlier ones
// (a rarely taken path of the orthonormalisation, kept out of the kernel's register
// allocation). Vector vec of the rank order, rv its remainder after the projection
// with squared norm nr. A kept vector, or a discarded one above the FP32 noise floor,
// on a block of T with more than one row: one inverse-iteration solve on that block
// from the normalised remainder (the directions the earlier vectors do not span), so
// repeated rounds deflate the members of an unresolved cluster that are already taken.
// Otherwise (any direction of the noise-floor subspace will do) a pseudo-random vector.
template <typename T>
__device__ __noinline__ void replace_step(const ClusterShared<T>& sh, int vec, int m, const T* tnorm_p, T* rv, T nr,
                                          int att) {
  const int lane = threadIdx.x & 31;
  const T tnorm = *tnorm_p;
  T* sc = const_cast<T*>(reinterpret_cast<const T*>(&sh.A[0][0])) + (size_t)(MSL * MBK + 1 + CL_NW) * CL_MAXM;
  const int pos = sh.order[vec];
  const bool noise = vec >= sh.k && !(fabs(sh.lam[pos]) > (T)16 * CEps<T>::v * fabs(sh.lam[sh.order[0]]));
  const int lo = sh.sblo[pos], hi = sh.sbhi[pos], sblk = hi - lo + 1;
  if (!noise && sblk > 1 && att < 3) {
    T* xs = sc + 4 * CL_MAXM;
    const T inv = nr > (T)0 ? (T)1 / sqrt(nr) : (T)0;
    for (int r2 = lane; r2 < sblk; r2 += 32) xs[r2] = nr > (T)0 ? rv[lo + r2] * inv : (T)(r2 == att);
    __syncwarp();
    tri_inverse_iteration<T>(sh, lo, hi, sh.lam[pos], tnorm, sc, xs, 1, lane);
    for (int row = lane; row < CL_MAXM; row += 32) rv[row] = (row >= lo && row <= hi) ? xs[row - lo] : (T)0;
  } else {
    for (int row = lane; row < CL_MAXM; row += 32) {
      unsigned h = (unsigned)(row + 1) * 2654435761u ^ ((unsigned)(vec + 1013 + att) * 40503u + 0x85ebca6bu);
      h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
      rv[row] = row < m ? (T)(h & 0xffffu) * (T)(1.0 / 65536.0) - (T)0.5 : (T)0;
    }
  }
  __syncwarp();
}

// Back-transform of the tridiagonal eigenvectors z (real, gZ) to those of the
// Hermitian matrix, y = H_0 (H_1 (... H_{m-2} z)), into evecs (FP64 storage, column
// normalised). Warp w of CTA `rank` carries the NC columns rank + CL (w + CL_NW c); the
// reflectors (full-length rows of gref, tau in its last row) are staged BT_STAGE at a
// time by one bulk asynchronous copy and applied in groups of BT_GROUP: the group's
// inner products v_k^dag y are reduced together and corrected with the reflectors'
// own inner products v_k^dag v_l. Returns false if the bounded wait on a copy gave up.
template <typename T, int NC>
__device__ __noinline__ bool back_transform(ClusterShared<T>& sh, const cx<T>* __restrict__ gref, const T* __restrict__ gZ,
                               double2* __restrict__ evecs, int m, int nvec, int rank) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const cx<T>* taus = reinterpret_cast<const cx<T>*>(gref + (size_t)(CL_MAXM - 1) * CL_MAXM);
  cx<T>* stage = reinterpret_cast<cx<T>*>(&sh.A[0][0]);  // BT_STAGE full-length reflectors
  static_assert(BT_STAGE * CL_MAXM <= CL_ROWS * CL_MAXM, "staging buffer");
  constexpr int E = CL_MAXM / 32;
  // reflectors applied together (fewer for two columns: register budget of 512 threads)
  constexpr int BT_GROUP = NC == 1 ? BtGroup<T>::v : BtGroup<T>::v / 2;
  cx<T>* gram = &sh.gram[0][0][0];  // [BT_STAGE / BT_GROUP][BT_GROUP][BT_GROUP]
  const int nref = m - 1;
  bool bt_ok = true;
  int bt_phase = 0;
  int col[NC];
  bool has[NC];
  cx<T> y[NC][E];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    col[c] = rank + CL * (warp + CL_NW * c);
    has[c] = col[c] < nvec;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int row = lane + 32 * e;
      y[c][e] = mk<T>(has[c] && row < m ? gZ[(size_t)col[c] * m + row] : (T)0, 0);
    }
  }
  const bool any = has[0];
  // reflector blocks from the last one down: [b0, b0 + nb)
  for (int top = nref; top > 0; top -= BT_STAGE) {
    const int b0 = top - BT_STAGE > 0 ? top - BT_STAGE : 0;
    const int nb = top - b0;
    __syncthreads();  // the previous block is no longer read
    if (tid == 0 && bt_ok) {
      // rows b0 .. b0 + nb - 1 of the reflector store are full-length rows (zero
      // outside each reflector's support): one bulk copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::bulk_load(tc::smem_u32(stage), gref + (size_t)b0 * CL_MAXM, (uint32_t)(nb * CL_MAXM * sizeof(cx<T>)),
                    tc::smem_u32(&sh.mbar));
    }
    if (tid < BT_STAGE) sh.btau[tid] = tid < nb ? taus[b0 + tid] : mk<T>(0, 0);
    if (bt_ok) bt_ok = tc::mbar_wait(tc::smem_u32(&sh.mbar), (uint32_t)(bt_phase & 1));
    ++bt_phase;
    bt_ok = __syncthreads_and(bt_ok) != 0;
    if (!bt_ok) continue;
    if (nb < BT_STAGE) {  // rows past the last reflector: zero, not stale
      for (int e = nb * CL_MAXM + tid; e < BT_STAGE * CL_MAXM; e += CL_THREADS) stage[e] = mk<T>(0, 0);
      __syncthreads();
    }
    // inner products of the reflectors within each group of BT_GROUP
    for (int pr = warp; pr < (BT_STAGE / BT_GROUP) * BT_GROUP * BT_GROUP; pr += CL_NW) {
      const int g = pr / (BT_GROUP * BT_GROUP), kk = (pr / BT_GROUP) % BT_GROUP, ll = pr % BT_GROUP;
      if (ll <= kk) continue;
      const cx<T>* vk = stage + (size_t)(g * BT_GROUP + kk) * CL_MAXM;
      const cx<T>* vl = stage + (size_t)(g * BT_GROUP + ll) * CL_MAXM;
      cx<T> acc = mk<T>(0, 0);
      for (int t = lane; t < m; t += 32) cfmac(acc, vk[t], vl[t]);
      acc.x = warp_sum(acc.x);
      acc.y = warp_sum(acc.y);
      if (lane == 0) gram[(g * BT_GROUP + kk) * BT_GROUP + ll] = acc;
    }
    __syncthreads();
    if (any) {
      for (int g = BT_STAGE / BT_GROUP - 1; g >= 0; --g) {
        // s_k = v_k^dag y for the group's reflectors and the warp's columns, reduced together
        T sre[NC][BT_GROUP], sim[NC][BT_GROUP];
#pragma unroll
        for (int kk = 0; kk < BT_GROUP; ++kk) {
          const cx<T>* vk = stage + (size_t)(g * BT_GROUP + kk) * CL_MAXM;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            cx<T> acc = mk<T>(0, 0);
#pragma unroll
            for (int e = 0; e < E; ++e) cfmac(acc, vk[lane + 32 * e], y[c][e]);
            sre[c][kk] = acc.x;
            sim[c][kk] = acc.y;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int kk = 0; kk < BT_GROUP; ++kk) {
              sre[c][kk] += __shfl_xor_sync(0xffffffffu, sre[c][kk], o);
              sim[c][kk] += __shfl_xor_sync(0xffffffffu, sim[c][kk], o);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          // f_k = tau_k (s_k - sum_{l > k} (v_k^dag v_l) f_l), k descending
          cx<T> f[BT_GROUP];
#pragma unroll
          for (int kk = BT_GROUP - 1; kk >= 0; --kk) {
            cx<T> sk = mk<T>(sre[c][kk], sim[c][kk]);
#pragma unroll
            for (int ll = kk + 1; ll < BT_GROUP; ++ll)
              sk = csub(sk, cmul(gram[(g * BT_GROUP + kk) * BT_GROUP + ll], f[ll]));
            f[kk] = cmul(sh.btau[g * BT_GROUP + kk], sk);
          }
#pragma unroll
          for (int kk = 0; kk < BT_GROUP; ++kk) {
            const cx<T>* vk = stage + (size_t)(g * BT_GROUP + kk) * CL_MAXM;
#pragma unroll
            for (int e = 0; e < E; ++e) y[c][e] = csub(y[c][e], cmul(f[kk], vk[lane + 32 * e]));
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (has[c] && bt_ok) {
      double nrm = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) nrm += (double)y[c][e].x * y[c][e].x + (double)y[c][e].y * y[c][e].y;
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int row = lane + 32 * e;
        if (row < m) {
          const double2 vv = to_d2(y[c][e]);
          evecs[(size_t)row * m + col[c]] = make_double2(vv.x * inv, vv.y * inv);
        }
      }
    }
  }
  return bt_ok;
}

__device__ __forceinline__ long long phase_clock() { return clock64(); }

}  // namespace

// The arguments are references: the single-matrix kernel binds them to its parameters
// and the batched kernel to its launch's task list (also kernel parameters), so that
// neither holds them in registers across the solve.
template <typename T>
__device__ __forceinline__ void eigh_cluster_body(const double2* __restrict__ const& G, const int& m,
                                                  cx<T>* __restrict__ const& gref, T* __restrict__ const& gZ,
                                                  double* __restrict__ const& evals,
                                                  double2* __restrict__ const& evecs,
                                                  EigOut* __restrict__ const& out, const int& r, const double& eps,
                                                  const int& all_vecs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ClusterShared<T>& sh = *reinterpret_cast<ClusterShared<T>*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nrows = (m - rank + CL - 1) / CL;  // rows rank, rank + CL, ...
  // peer(q): CTA q's shared block (mapped on use; holding 8 pointers costs 16 registers)
  auto peer = [&](int q) { return cluster.map_shared_rank(&sh, q); };
  __shared__ long long t_ph[6];
#ifdef LRET_EIG_PROFILE
  if (tid < 4) sh.gdbg[tid] = 0;
#endif
  long long t0 = phase_clock();

  // ---- load G / trace (every CTA its rows) --------------------------------
  double tr = 0.0;
  for (int i = tid; i < m; i += CL_THREADS) tr += G[(size_t)i * m + i].x;
  tr = block_sum(tr, sh.dred);
  if (tid == 0) sh.trace = tr;
  __syncthreads();
  const double gscale = sh.trace > 0.0 ? sh.trace : 1.0;
  const double ginv = 1.0 / gscale;
  // This CTA's rows live in registers during the reduction: warp w holds local
  // rows w and w + 16 (rows CL w + rank, CL (w + 16) + rank), lane l columns
  // l + 32 e.
  constexpr int E = CL_MAXM / 32;
  const int li0 = warp, li1 = warp + CL_NW;
  const int i0 = li0 * CL + rank, i1 = li1 * CL + rank;
  cx<T> A0[E], A1[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int c = lane + 32 * e;
    A0[e] = mk<T>(0, 0);
    A1[e] = mk<T>(0, 0);
    if (c < m) {
      if (li0 < nrows) {
        const double2 g = G[(size_t)i0 * m + c];
        A0[e] = mk<T>((T)(g.x * ginv), (T)(g.y * ginv));
      }
      if (li1 < nrows) {
        const double2 g = G[(size_t)i1 * m + c];
        A1[e] = mk<T>((T)(g.x * ginv), (T)(g.y * ginv));
      }
    }
  }
  if (tid == 0) { const long long t1 = phase_clock(); t_ph[0] = t1 - t0; t0 = t1; }

  // ---- reduction to tridiagonal form ----------------------------------------
  // Every CTA holds v_j and tau_j. Step j: every CTA forms p_i = tau sum_c
  // A[i][c] v_c for its rows and sends them, with one partial of v^dag p per
  // warp, to every CTA [cluster barrier]. Then warps 4-15 update this CTA's rows,
  // A[i][c] -= v_i conj(w_c) + w_i conj(v_c), w = p - (1/2) conj(tau)(v^dag p) v
  // (the owner of row j + 3 also stores it in global memory), while warps 0-3
  // form v_{j+1}, tau_{j+1} from their prefetched copy of row j + 1 and start the
  // copy of row j + 2. Every CTA computes the same reflector, so one barrier per
  // step suffices.
  cx<T>* grow = reinterpret_cast<cx<T>*>(gZ + (size_t)CL_MAXM * CL_MAXM);  // three row buffers
  // a warp's row into row buffer rb (columns from c0)
  auto store_row = [&](const cx<T>(&R)[E], int rb, int c0) {
    cx<T>* dst = grow + (size_t)rb * CL_MAXM;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane + 32 * e;
      if (c >= c0 && c < m) dst[c] = R[e];
    }
  };
  if (rank < 3 && rank < m && warp == 0) store_row(A0, rank, 0);  // rows 0, 1, 2 as loaded
  cluster.sync();
  if (tid < RG) {
    // reflector 0 from row 0; row 1 into the prefetch buffer
    prefetch_row<T>(sh.nrow[0], grow, 0, m, tid);
    prefetch_row<T>(sh.nrow[1], grow + CL_MAXM, 1, m, tid);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    bar_group();
    group_reflector<T>(sh, sh.nrow[0], 0, m, 0, 0, false, 0, false, rank == 0, gref, tid);
  }
  __syncthreads();
#ifdef LRET_EIG_PROFILE
  // diagnostic build: cycles of the reduction's sub-steps on CTA 0, thread 0
  long long sp[6] = {0, 0, 0, 0, 0, 0}, tq = clock64();
#define LRET_SUBSTEP(k) { const long long t2 = clock64(); sp[k] += t2 - tq; tq = t2; }
#else
#define LRET_SUBSTEP(k)
#endif
  // The last steps act on a trailing block of at most TAIL_N rows: CTA 0 finishes
  // them alone from shared memory (block barriers instead of cluster barriers).
  const int s0 = m - 1 > TAIL_N ? m - 1 - TAIL_N : 0;
#if defined(LRET_EIG_PROFILE) && LRET_EIG_PROFILE >= 3
  const long long tloop0 = clock64();
#endif
  for (int j = 0; j < s0; ++j) {
    const int sl = j % 3, slp = (j + 2) % 3, sln = (j + 1) % 3;  // slots of steps j, j - 1, j + 1
    const int nx = j + 1;
    const cx<T> tau = sh.tau[sl];
    const bool skip = (tau.x == (T)0 && tau.y == (T)0);
    const bool a0 = li0 < nrows && i0 > j, a1 = li1 < nrows && i1 > j;
    {
      // p_i = tau sum_c A[i][c] v_c for this warp's rows (two, reduced together)
      T dr = 0, di = 0;
      if (!skip && (a0 || a1)) {
        cx<T> acc0 = mk<T>(0, 0), acc1 = mk<T>(0, 0);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int c = lane + 32 * e;
          if (c > j && c < m) {
            const cx<T> vc = sh.v[sl][c];
            cfma(acc0, A0[e], vc);
            cfma(acc1, A1[e], vc);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          acc0.x += __shfl_xor_sync(0xffffffffu, acc0.x, o);
          acc0.y += __shfl_xor_sync(0xffffffffu, acc0.y, o);
          acc1.x += __shfl_xor_sync(0xffffffffu, acc1.x, o);
          acc1.y += __shfl_xor_sync(0xffffffffu, acc1.y, o);
        }
        if (a0) {
          const cx<T> pi = cmul(tau, acc0);
          if (lane < CL) peer(lane)->p[sl][i0] = pi;
          const cx<T> vi = sh.v[sl][i0];
          dr += vi.x * pi.x + vi.y * pi.y;  // Re conj(v_i) p_i
          di += vi.x * pi.y - vi.y * pi.x;  // Im conj(v_i) p_i
        }
        if (a1) {
          const cx<T> pi = cmul(tau, acc1);
          if (lane < CL) peer(lane)->p[sl][i1] = pi;
          const cx<T> vi = sh.v[sl][i1];
          dr += vi.x * pi.x + vi.y * pi.y;
          di += vi.x * pi.y - vi.y * pi.x;
        }
      }
      if (lane < CL) peer(lane)->dpart[sl][rank * CL_NW + warp] = mk<T>(dr, di);
    }
    LRET_SUBSTEP(0)
    cluster.sync();
    LRET_SUBSTEP(1)
    T cc = 0;
    if (!skip) {
      cx<T> sp4 = mk<T>(0, 0);
      for (int q = lane; q < CL * CL_NW; q += 32) sp4 = cadd(sp4, sh.dpart[sl][q]);
      const T sr = warp_sum(sp4.x), si = warp_sum(sp4.y);
      cc = (T)0.5 * (tau.x * sr + tau.y * si);
      // rank-2 update of this warp's rows: A[i][c] -= v_i conj(w_c) + w_i conj(v_c)
      const cx<T> v0 = a0 ? sh.v[sl][i0] : mk<T>(0, 0), v1 = a1 ? sh.v[sl][i1] : mk<T>(0, 0);
      const cx<T> w0 = a0 ? csub(sh.p[sl][i0], cscale(v0, cc)) : mk<T>(0, 0);
      const cx<T> w1 = a1 ? csub(sh.p[sl][i1], cscale(v1, cc)) : mk<T>(0, 0);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int c = lane + 32 * e;
        if (c > j && c < m) {
          const cx<T> vc = sh.v[sl][c];
          const cx<T> wc = csub(sh.p[sl][c], cscale(vc, cc));
          if (a0) {
            A0[e] = csub(A0[e], cadd(cmul(v0, conjg(wc)), cmul(w0, conjg(vc))));
            if (c == i0) A0[e].y = 0;
          }
          if (a1) {
            A1[e] = csub(A1[e], cadd(cmul(v1, conjg(wc)), cmul(w1, conjg(vc))));
            if (c == i1) A1[e].y = 0;
          }
        }
      }
    }
    if (tid == 0) sh.ccs[sl] = cc;
    // row j + 3 (as updated through this step) for the reflector group two steps ahead
    if (j + 3 < m && rank == (j + 3) % CL) {
      const int lst = (j + 3) / CL;
      if (lst == li0) store_row(A0, (j + 3) % 3, j + 1);
      else if (lst == li1) store_row(A1, (j + 3) % 3, j + 1);
    }
    LRET_SUBSTEP(2)
    if (tid < RG) {
      const bool up0 = j >= 1 && !(sh.tau[slp].x == (T)0 && sh.tau[slp].y == (T)0);
      asm volatile("cp.async.wait_group 0;" ::: "memory");  // row nx, copied during step j - 1
      bar_group();                                          // (also publishes ccs[sl])
      const cx<T>* row = sh.nrow[nx & 1];
      if (nx < m - 1) {
        group_reflector<T>(sh, row, nx, m, sln, slp, up0, sl, !skip, rank == nx % CL, gref, tid);
      } else if (tid == 0) {  // last diagonal entry
        cx<T> a = row[nx];
        if (up0) a = upd1(sh, slp, sh.ccs[slp], nx, nx, a);
        if (!skip) a = upd1(sh, sl, cc, nx, nx, a);
        sh.d[m - 1] = a.x;
        sh.e[m - 1] = 0;
      }
      // row j + 2 (stored during step j - 1) for the next step
      if (nx + 1 < m) prefetch_row<T>(sh.nrow[(nx + 1) & 1], grow + (size_t)((nx + 1) % 3) * CL_MAXM, nx + 1, m, tid);
      LRET_SUBSTEP(3)
    }
    __syncthreads();
    LRET_SUBSTEP(4)
  }
#undef LRET_SUBSTEP
#if defined(LRET_EIG_PROFILE) && LRET_EIG_PROFILE >= 3
  const long long tloop1 = clock64();
#endif
  // ---- trailing block on CTA 0 ------------------------------------------------
  // Rows and columns s0 + 1 .. m - 1 (updated through step s0 - 1; v_s0, tau_s0,
  // d_s0, e_s0 are known to every CTA) go to CTA 0's scratch A, nt x nt.
  const int nt = m - 1 - s0;
  if (tid < RG) asm volatile("cp.async.wait_group 0;" ::: "memory");
  {
    cx<T>* tb0 = &peer(0)->A[0][0];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int c = lane + 32 * e;
      if (c > s0 && c < m) {
        if (li0 < nrows && i0 > s0) tb0[(size_t)(i0 - s0 - 1) * nt + (c - s0 - 1)] = A0[e];
        if (li1 < nrows && i1 > s0) tb0[(size_t)(i1 - s0 - 1) * nt + (c - s0 - 1)] = A1[e];
      }
    }
  }
  cluster.sync();
#if defined(LRET_EIG_PROFILE) && LRET_EIG_PROFILE >= 3
  // diagnostic build: cycles of the trailing block's sub-steps (3: thread 0, 4: thread 128)
  __shared__ long long tdbg[6];
  long long tp3[4] = {0, 0, 0, 0}, tq3 = clock64();
  if (tid == 0) tdbg[1] = tq3;
#define LRET_TAILSTEP(k) { const long long t2 = clock64(); tp3[k] += t2 - tq3; tq3 = t2; }
#else
#define LRET_TAILSTEP(k)
#endif
  if (rank == 0) {
    cx<T>* tb = &sh.A[0][0];
    auto trow = [&](int i) { return tb + (ptrdiff_t)(i - s0 - 1) * nt - (s0 + 1); };  // indexed by column
    cx<T>* pq = &sh.nrow[0][0];  // matvec partials, four column quarters x 128 rows
    for (int j = s0; j < m - 1; ++j) {
      const int sl = j % 3, sln = (j + 1) % 3;
      const cx<T> tau = sh.tau[sl];
      const bool skip = (tau.x == (T)0 && tau.y == (T)0);
      const int n1 = m - 1 - j;  // trailing rows and columns j + 1 .. m - 1
      // A v by column quarters: thread (q, il) sums conj(A[c][i]) v_c = A[i][c] v_c over
      // quarter q of the columns for row i = j + 1 + il (column reads: consecutive
      // threads read consecutive entries of row c)
      if (!skip) {
        const int q = tid >> 7, il = tid & 127;
        if (il < n1) {
          const int len = (n1 + 3) >> 2;
          const int ca = j + 1 + q * len, cb = min(ca + len, m);
          const int i = j + 1 + il;
          cx<T> acc0 = mk<T>(0, 0), acc1 = mk<T>(0, 0);
          int c = ca;
          for (; c + 1 < cb; c += 2) {
            cfma(acc0, conjg(trow(c)[i]), sh.v[sl][c]);
            cfma(acc1, conjg(trow(c + 1)[i]), sh.v[sl][c + 1]);
          }
          if (c < cb) cfma(acc0, conjg(trow(c)[i]), sh.v[sl][c]);
          pq[q * 128 + il] = cadd(acc0, acc1);
        }
      }
      LRET_TAILSTEP(0)
      __syncthreads();
      LRET_TAILSTEP(1)
      // every warp: p_c = tau (A v)_c, v_c for its lanes' columns c = j + 1 + lane + 32 h,
      // then cc = (1/2) Re(conj(tau) v^dag p) by its own (identical) reduction
      cx<T> vv[3], ww[3];
      T cc = 0;
      {
        cx<T> pp[3];
        T dr = 0, di = 0;
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const int c = j + 1 + lane + 32 * h;
          vv[h] = mk<T>(0, 0);
          pp[h] = mk<T>(0, 0);
          if (c < m && !skip) {
            const int k = c - j - 1;
            vv[h] = sh.v[sl][c];
            pp[h] = cmul(tau, cadd(cadd(pq[k], pq[128 + k]), cadd(pq[256 + k], pq[384 + k])));
            dr += vv[h].x * pp[h].x + vv[h].y * pp[h].y;
            di += vv[h].x * pp[h].y - vv[h].y * pp[h].x;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dr += __shfl_xor_sync(0xffffffffu, dr, o);
          di += __shfl_xor_sync(0xffffffffu, di, o);
        }
        cc = (T)0.5 * (tau.x * dr + tau.y * di);
#pragma unroll
        for (int h = 0; h < 3; ++h) ww[h] = csub(pp[h], cscale(vv[h], cc));
      }
      if (warp == 0) {
        // v_{j+1}, tau_{j+1} from row j + 1 with this step's update applied (or d_{m-1})
        warp_reflector<T>(sh, trow(j + 1), j + 1, m, sln, vv, ww, !skip, gref, lane);
      } else if (!skip) {
        // rows j + 2 .. m - 1, columns j + 1 .. m - 1: A[i][c] -= v_i conj(w_c) + w_i conj(v_c)
        // (column j + 1 is no longer read); three rows per batch, loads first
        constexpr int UW = CL_NW - 1;
        for (int i0 = j + 2 + (warp - 1); i0 < m; i0 += 3 * UW) {
          cx<T> a[3][3], vi[3], wi[3];
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int i = i0 + t * UW;
            const int k = i - j - 1, hk = k >> 5, lk = k & 31;  // row i's entry in the lanes' columns
            const cx<T> vs = hk == 0 ? vv[0] : (hk == 1 ? vv[1] : vv[2]);
            const cx<T> ws = hk == 0 ? ww[0] : (hk == 1 ? ww[1] : ww[2]);
            vi[t] = mk<T>(__shfl_sync(0xffffffffu, vs.x, lk), __shfl_sync(0xffffffffu, vs.y, lk));
            wi[t] = mk<T>(__shfl_sync(0xffffffffu, ws.x, lk), __shfl_sync(0xffffffffu, ws.y, lk));
#pragma unroll
            for (int h = 0; h < 3; ++h) {
              const int c = j + 1 + lane + 32 * h;
              a[t][h] = (i < m && c < m) ? trow(i)[c] : mk<T>(0, 0);
            }
          }
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            const int i = i0 + t * UW;
            if (i < m) {
#pragma unroll
              for (int h = 0; h < 3; ++h) {
                const int c = j + 1 + lane + 32 * h;
                if (c < m) {
                  cx<T> x = csub(a[t][h], cadd(cmul(vi[t], conjg(ww[h])), cmul(wi[t], conjg(vv[h]))));
                  if (c == i) x.y = 0;
                  trow(i)[c] = x;
                }
              }
            }
          }
        }
      }
      LRET_TAILSTEP(2)
      __syncthreads();
      LRET_TAILSTEP(3)
    }
#if defined(LRET_EIG_PROFILE) && LRET_EIG_PROFILE >= 3
    if (tid == (LRET_EIG_PROFILE == 3 ? 0 : 128))
      for (int q = 0; q < 4; ++q) tdbg[2 + q] = tp3[q];
#endif
#undef LRET_TAILSTEP
    // the tail's diagonal and off-diagonal to the other CTAs
    for (int q = 1; q < CL; ++q) {
      ClusterShared<T>* pq = peer(q);
      for (int i = s0 + 1 + tid; i < m; i += CL_THREADS) {
        pq->d[i] = sh.d[i];
        pq->e[i] = sh.e[i];
      }
    }
  }
  cluster.sync();
  if (tid == 0) { const long long t1 = phase_clock(); t_ph[1] = t1 - t0; t0 = t1; }

  // ---- split, multisection (eigenvalues t = rank + CL * group) ----------------
  __shared__ T s_red[CL_NW];
  __shared__ T s_tnorm, s_pivmin;
  {
    // ||T||_inf, then negligible off-diagonals set to zero, then unreduced blocks
    T tn = 0;
    for (int i = tid; i < m; i += CL_THREADS)
      tn = fmax(tn, fabs(sh.d[i]) + (i > 0 ? fabs(sh.e[i - 1]) : (T)0) + (i < m - 1 ? fabs(sh.e[i]) : (T)0));
    for (int o = 16; o > 0; o >>= 1) tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    if (lane == 0) s_red[warp] = tn;
    __syncthreads();
    if (tid == 0) {
      T v = 0;
      for (int w = 0; w < CL_NW; ++w) v = fmax(v, s_red[w]);
      s_tnorm = v;
    }
    __syncthreads();
    tn = s_tnorm;
    T emax2 = 0;
    for (int i = tid; i < m - 1; i += CL_THREADS) {
      T ei = sh.e[i];
      if (fabs(ei) <= CEps<T>::v * (fabs(sh.d[i]) + fabs(sh.d[i + 1])) || fabs(ei) <= CEps<T>::v * CEps<T>::v * tn)
        ei = 0;
      sh.e[i] = ei;
      sh.e2[i] = ei * ei;
      emax2 = fmax(emax2, ei * ei);
    }
    for (int o = 16; o > 0; o >>= 1) emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
    __syncthreads();
    if (lane == 0) s_red[warp] = emax2;
    __syncthreads();
    if (warp == 0) {
      // block boundaries: sblo = last start <= i (prefix max), sbhi = first end >= i (suffix min);
      // lane l holds i = 8 l .. 8 l + 7
      int run = -1, lov[8], hiv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = lane * 8 + q;
        if (i < m && (i == 0 || sh.e[i - 1] == (T)0)) run = i;
        lov[q] = run;
      }
      int carry = run;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, carry, o);
        if (lane >= o) carry = max(carry, t);
      }
      int prev = __shfl_up_sync(0xffffffffu, carry, 1);
      if (lane == 0) prev = -1;
      constexpr int BIG = 1 << 20;
      run = BIG;
#pragma unroll
      for (int q = 7; q >= 0; --q) {
        const int i = lane * 8 + q;
        if (i < m && (i == m - 1 || sh.e[i] == (T)0)) run = i;
        hiv[q] = run;
      }
      carry = run;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_down_sync(0xffffffffu, carry, o);
        if (lane + o < 32) carry = min(carry, t);
      }
      int next = __shfl_down_sync(0xffffffffu, carry, 1);
      if (lane == 31) next = BIG;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = lane * 8 + q;
        if (i < m) {
          sh.sblo[i] = (short)max(lov[q], prev);
          sh.sbhi[i] = (short)min(hiv[q], next);
        }
      }
      if (lane == 0) {
        T v = 0;
        for (int w = 0; w < CL_NW; ++w) v = fmax(v, s_red[w]);
        s_tnorm = tn > (T)0 ? tn : (T)1;
        s_pivmin = CEps<T>::tiny * (v > (T)1 ? v : (T)1);
      }
    }
  }
  __syncthreads();
  const T tnorm = s_tnorm, pivmin = s_pivmin;
  {
    const int grp = tid / MS, sub = tid % MS;
    const unsigned hmask = 0xffffu << (lane & 16);
    for (int t = rank + CL * grp; t < m; t += CL * (CL_THREADS / MS)) {
      const int lo = sh.sblo[t], hi = sh.sbhi[t], li = t - lo;
      T gl = sh.d[lo], gu = sh.d[lo];
      for (int i = lo + sub; i <= hi; i += MS) {
        const T rad = (i > lo ? fabs(sh.e[i - 1]) : (T)0) + (i < hi ? fabs(sh.e[i]) : (T)0);
        gl = fmin(gl, sh.d[i] - rad);
        gu = fmax(gu, sh.d[i] + rad);
      }
      for (int o = MS / 2; o > 0; o >>= 1) {
        gl = fmin(gl, __shfl_xor_sync(hmask, gl, o));
        gu = fmax(gu, __shfl_xor_sync(hmask, gu, o));
      }
      T a = gl - CEps<T>::v * tnorm * 2 - pivmin, b = gu + CEps<T>::v * tnorm * 2 + pivmin;
      for (int it = 0; it < 48; ++it) {
        if (b - a <= (T)2 * CEps<T>::v * fmax(fabs(a), fabs(b)) + CEps<T>::v * tnorm * (T)1e-3) break;
        const T h = (b - a) / (T)(MS + 1);
        const T x = a + h * (T)(sub + 1);
        const bool below = sturm_count<T>(sh.d, sh.e2, lo, hi, x, pivmin) <= li;  // lambda_li >= x
        const unsigned bal = (__ballot_sync(hmask, below) >> (lane & 16)) & 0xffffu;
        const int nt = bal == 0xffffu ? MS : __ffs(~bal) - 1;  // first point with lambda_li < x
        const T na = nt > 0 ? a + h * (T)nt : a;
        const T nb = nt < MS ? a + h * (T)(nt + 1) : b;
        if (na == a && nb == b) break;  // no progress at this precision
        a = na;
        b = nb > na ? nb : na;
      }
      T lt = (T)0.5 * (a + b);
      if (!(lt == lt)) lt = -INFINITY;
      if (sub < CL) peer(sub)->lam[t] = lt;
    }
  }
  cluster.sync();

  // ---- sort (every CTA), rank choice and accounting ---------------------------
  {
    const int t = tid;  // m <= CL_THREADS: one eigenvalue per thread
    T lt = 0;
    int rk = CL_MAXM;
    if (t < m) {
      lt = sh.lam[t];
      rk = 0;
      for (int u = 0; u < m; ++u) {
        const T lu = sh.lam[u];
        rk += (lu > lt) || (lu == lt && u < t);
      }
      sh.order[rk] = (short)t;
      if (rank == 0) evals[rk] = (double)lt * gscale;
    }
    const double vpos = (t < m && lt > (T)0) ? (double)lt * gscale : 0.0;
    const double total = block_sum(vpos, sh.dred);  // valid in thread 0; the call synchronises
    __shared__ double s_total;
    if (tid == 0) s_total = total;
    __syncthreads();
    if (tid == 0) {
      int k;
      if (r > 0) {
        k = r < m ? r : m;
      } else {
        double cs = 0.0;
        k = m;
        for (int i = 0; i < m; ++i) {
          const double v = (double)sh.lam[sh.order[i]] * gscale;
          cs += v > 0 ? v : 0.0;
          if (cs >= (1.0 - eps) * s_total) { k = i + 1; break; }
        }
      }
      sh.k = k;
    }
    __syncthreads();
    const int k = sh.k;
    const double kept = block_sum(rk < k ? vpos : 0.0, sh.dred);
    const double dropped = block_sum(rk < k ? 0.0 : vpos, sh.dred);
    if (rank == 0 && tid == 0) {
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
  if (tid == 0) { const long long t1 = phase_clock(); t_ph[2] = t1 - t0; t0 = t1; }

  // ---- inverse iteration: vectors i = rank + CL * (warp + nw * ...) ---------
  {
    // per-warp LU scratch reuses this CTA's matrix rows (no longer needed)
    T* ws = reinterpret_cast<T*>(&sh.A[0][0]);
    constexpr int SLOT = 6 * CL_MAXM;
    const int nlu_a = (int)(sizeof(sh.A) / (SLOT * sizeof(T)));
    const int nlu = nlu_a + LuExtra<T>::slots;  // every warp has a slot for FP32
    if (warp < nlu) {
      T* dl = warp < nlu_a ? ws + (size_t)warp * SLOT
                           : reinterpret_cast<T*>(smem_raw + sizeof(ClusterShared<T>)) + (size_t)(warp - nlu_a) * SLOT;
      T* x = dl + 4 * CL_MAXM;  // the iterate (the factors before it, pivots after)
      const int wn = nlu < CL_NW ? nlu : CL_NW;
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
        for (int t = lane; t < s; t += 32) {
          unsigned h = (unsigned)(t + 1) * 2654435761u ^ ((unsigned)(i + 7) * 40503u + 0x9e3779b9u);
          h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
          const T u = (T)(h & 0xffffu) * (T)(1.0 / 65536.0) + (T)0.5;
          x[t] = (h & 0x10000u) ? -u : u;
        }
        __syncwarp();
        tri_inverse_iteration<T>(sh, lo, hi, lam, tnorm, dl, x, 2, lane);
        for (int t = lane; t < s; t += 32) z[lo + t] = x[t];
        __syncwarp();
      }
    }
  }
  __threadfence();
  cluster.sync();
  if (tid == 0) { const long long t1 = phase_clock(); t_ph[3] = t1 - t0; t0 = t1; }

  // ---- orthonormalisation of the needed vectors: block Gram-Schmidt over the cluster --
  // Vectors in rank order, in blocks of MBK = 16: block b is owned by CTA b % CL, its
  // vector MBK b + w held in registers by warp w (slot b / CL). Step b: the owner
  // orthonormalises the block (modified Gram-Schmidt, two passes, one vector per warp,
  // block barriers) and publishes it in its shared memory [cluster barrier]; every CTA
  // copies it into local shared memory and removes it, twice (classical Gram-Schmidt
  // against an orthonormal block, repeated), from its vectors of later blocks. A vector
  // that cancels (nearly dependent on earlier ones; inverse iteration can return almost
  // equal vectors for eigenvalues the FP32 arithmetic does not separate) is replaced by
  // a pseudo-random vector orthogonalised against every finished vector.
  {
    constexpr int E = CL_MAXM / 32;
    const int nblk = (nvec + MBK - 1) / MBK;
    T* pub = reinterpret_cast<T*>(&sh.A[0][0]);  // [MSL][MBK][CL_MAXM]: this CTA's finished blocks
    T* cpy = pub + MSL * MBK * CL_MAXM;          // [MBK][CL_MAXM]: the block being removed
    static_assert((MSL + 1) * MBK * CL_MAXM * sizeof(T) <= sizeof(ClusterShared<T>::A), "orthonormalisation buffers");
    T z[MSL][E];
#pragma unroll
    for (int sl = 0; sl < MSL; ++sl) {
      const int vec = MBK * (rank + CL * sl) + warp;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int row = lane + 32 * e;
        z[sl][e] = (vec < nvec && row < m) ? gZ[(size_t)vec * m + row] : (T)0;
      }
    }
    // remove the MBK vectors of cpy (orthonormal) from slot sl, twice; eight at a time
    // (the inner products of a group are reduced together)
    constexpr int MG = sizeof(T) == 4 ? 8 : 4;
    auto remove_block = [&](int sl) {
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        T nz = 0, nd = 0;  // |z|^2 before, |coefficients|^2 (repeat only if a sizeable part went)
        if (pass == 0) {
#pragma unroll
          for (int e = 0; e < E; ++e) nz += z[sl][e] * z[sl][e];
          nz = warp_sum(nz);
        }
#pragma unroll 1
        for (int g = 0; g < MBK; g += MG) {
          const T* cg = cpy + (size_t)g * CL_MAXM;
          T d[MG];
#pragma unroll
          for (int t = 0; t < MG; ++t) {
            T a = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) a += cg[t * CL_MAXM + lane + 32 * e] * z[sl][e];
            d[t] = a;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int t = 0; t < MG; ++t) d[t] += __shfl_xor_sync(0xffffffffu, d[t], o);
          }
#pragma unroll
          for (int t = 0; t < MG; ++t) nd += d[t] * d[t];
#pragma unroll
          for (int e = 0; e < E; ++e) {
            T a = z[sl][e];
#pragma unroll
            for (int t = 0; t < MG; ++t) a -= d[t] * cg[t * CL_MAXM + lane + 32 * e];
            z[sl][e] = a;
          }
        }
        if (pass == 0 && !(nd > (T)1e-4 * nz)) break;  // nearly orthogonal already
      }
    };
    // replacement of a cancelled vector: the whole CTA removes (twice) the first nprev
    // vectors of the rank order (earlier blocks from global memory, the owner's block
    // from pub) from rv
    auto project_rv = [&](int nprev) {
      const int b = nprev / MBK;
      const T* pb = pub + (size_t)(b / CL) * MBK * CL_MAXM;
      T* rv = cpy;
      T* part = cpy + CL_MAXM;
      for (int rep = 0; rep < 2; ++rep) {
        T acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0;
        for (int u = warp; u < nprev; u += CL_NW) {
          const T* q = u < MBK * b ? gZ + (size_t)u * m : pb + (size_t)(u - MBK * b) * CL_MAXM;
          T a = 0;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int row = lane + 32 * e;
            if (row < m) a += q[row] * rv[row];
          }
          a = warp_sum(a);
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int row = lane + 32 * e;
            if (row < m) acc[e] += a * q[row];
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) part[warp * CL_MAXM + lane + 32 * e] = acc[e];
        __syncthreads();
        for (int row = tid; row < m; row += CL_THREADS) {
          T sub = 0;
          for (int ww = 0; ww < CL_NW; ++ww) sub += part[ww * CL_MAXM + row];
          rv[row] -= sub;
        }
        __syncthreads();
      }
    };
    for (int b = 0; b < nblk; ++b) {
      const int owner = b % CL, osl = b / CL;
      if (rank == owner) {
        T* pb = pub + (size_t)osl * MBK * CL_MAXM;
        T* rv = cpy;                  // fallback: the replacement vector (cpy is idle here)
        T* part = cpy + CL_MAXM;      // fallback: per-warp partial corrections
        static_assert((MSL * MBK + 1 + CL_NW + 6) * CL_MAXM * sizeof(T) <= sizeof(ClusterShared<T>::A),
                      "fallback buffers");
        const int vec = MBK * b + warp;
        const bool mine = vec < nvec;
        // this warp's vector of the block (selected without indexing z by a runtime slot)
        T w[E];
#pragma unroll
        for (int e = 0; e < E; ++e) w[e] = osl == 0 ? z[0][e] : z[MSL - 1][e];
        T nrm0 = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) nrm0 += w[e] * w[e];
        nrm0 = warp_sum(nrm0);
        __shared__ int s_flag, s_again;
        if (tid == 0) s_again = 0;
        for (int pass = 0; pass < 2; ++pass) {
          if (pass == 1) {  // a second pass only where the first one cancelled much of a vector
            __syncthreads();
            if (s_again == 0) break;
          }
          for (int t = 0; t < MBK && MBK * b + t < nvec; ++t) {
            if (warp == t) {
              T nrm = 0;
#pragma unroll
              for (int e = 0; e < E; ++e) nrm += w[e] * w[e];
              nrm = warp_sum(nrm);
              // (vectors enter with unit norm from the inverse iteration)
              const bool cancelled = pass == 0 && !(nrm > (T)1e-6);
              if (pass == 0 && nrm < (T)0.25 * nrm0 && lane == 0) s_again = 1;
              if (lane == 0) s_flag = cancelled ? 1 : 0;
              if (cancelled) {
                // inverse iteration from a new pseudo-random start, on the block of T
                // that holds this eigenvalue, gives a vector of the same (nearly
                // degenerate) eigenspace; it is orthogonalised below by the whole CTA
                // against every earlier vector (earlier blocks from global memory). A
                // discarded vector whose eigenvalue lies in the FP32 noise floor (any
                // direction of that subspace will do) takes a plain pseudo-random vector.
                const int pos = sh.order[vec];
                const bool noise = vec >= sh.k &&
                                   !(fabs(sh.lam[pos]) > (T)16 * CEps<T>::v * fabs(sh.lam[sh.order[0]]));
                const int lo = noise ? 0 : sh.sblo[pos], hi = noise ? m - 1 : sh.sbhi[pos], sblk = hi - lo + 1;
                T* sc = pub + (size_t)(MSL * MBK + 1 + CL_NW) * CL_MAXM;  // LU scratch
                T* xs = sc + 4 * CL_MAXM;
                for (int r2 = lane; r2 < sblk; r2 += 32) {
                  unsigned h = (unsigned)(r2 + 1) * 2654435761u ^ ((unsigned)(vec + 11) * 40503u + 0x85ebca6bu);
                  h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
                  xs[r2] = (T)(h & 0xffffu) * (T)(1.0 / 65536.0) - (T)0.5;
                }
                __syncwarp();
                if (sblk > 1 && !noise) tri_inverse_iteration<T>(sh, lo, hi, sh.lam[pos], tnorm, sc, xs, 2, lane);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                  const int row = lane + 32 * e;
                  if (row < CL_MAXM) rv[row] = (row >= lo && row <= hi) ? xs[row - lo] : (T)0;
                }
              }
            }
            __syncthreads();
            if (s_flag) {
              if (tid == 0) atomicAdd(&out->sweeps, 1);  // diagnostics: replaced vectors
              const int nprev = MBK * b + t;
              project_rv(nprev);
              // cancelled again: inverse iteration on one eigenvalue of a cluster the FP32
              // arithmetic does not separate keeps returning the member nearest the shift,
              // which the earlier vectors already hold. Deflated inverse iteration: the
              // remainder after the projection (the directions the earlier vectors do not
              // span), normalised, starts another solve, projected again, up to four
              // rounds. Only a discarded vector in the FP32 noise floor (any direction of
              // that subspace will do) or a one-row block takes a plain pseudo-random vector.
              // (the round count lives in shared memory: registers are tight here)
              __shared__ int s_att;
              if (tid == 0) s_att = 0;
              for (;;) {
                if (warp == t) {
                  T nr = 0;
#pragma unroll
                  for (int e = 0; e < E; ++e) nr += rv[lane + 32 * e] * rv[lane + 32 * e];
                  nr = warp_sum(nr);
                  const bool ok = nr > (T)1e-6 || s_att >= 4;
                  __syncwarp();
                  if (lane == 0) s_flag = ok ? 0 : 2;
                  if (!ok) replace_step<T>(sh, vec, m, &s_tnorm, rv, nr, s_att);
                }
                __syncthreads();
                if (s_flag == 0) break;
                if (tid == 0) ++s_att;
                project_rv(nprev);
              }
              if (warp == t) {
#pragma unroll
                for (int e = 0; e < E; ++e) w[e] = rv[lane + 32 * e];
              }
              if (tid == 0) s_again = 1;  // and a second pass over the block
            }
            if (warp == t) {
              T nrm = 0;
#pragma unroll
              for (int e = 0; e < E; ++e) nrm += w[e] * w[e];
              nrm = warp_sum(nrm);
              const T inv = nrm > (T)0 ? (T)1 / sqrt(nrm) : (T)0;
#pragma unroll
              for (int e = 0; e < E; ++e) {
                w[e] *= inv;
                pb[t * CL_MAXM + lane + 32 * e] = w[e];
              }
            }
            __syncthreads();
            if (mine && warp > t) {
              T a = 0;
#pragma unroll
              for (int e = 0; e < E; ++e) a += pb[t * CL_MAXM + lane + 32 * e] * w[e];
              a = warp_sum(a);
#pragma unroll
              for (int e = 0; e < E; ++e) w[e] -= a * pb[t * CL_MAXM + lane + 32 * e];
            }
          }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (osl == 0) z[0][e] = w[e];
          else z[MSL - 1][e] = w[e];
        }
        // finished vectors also go to global memory (the fallback and the
        // back-transform read them there)
        if (mine) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int row = lane + 32 * e;
            if (row < m) gZ[(size_t)vec * m + row] = w[e];
          }
        }
        __threadfence();
      }
      cluster.sync();  // block b published (shared memory of its owner, and global memory)
      if (b + 1 < nblk) {
        const T* src = cluster.map_shared_rank(pub + (size_t)osl * MBK * CL_MAXM, owner);
        for (int i = tid; i < MBK * CL_MAXM; i += CL_THREADS) cpy[i] = src[i];
        __syncthreads();
#pragma unroll
        for (int sl = 0; sl < MSL; ++sl) {
          const int bb = rank + CL * sl;
          if (bb > b && MBK * bb + warp < nvec) remove_block(sl);
        }
        // cpy is rewritten only after the next cluster barrier, which every warp of this
        // CTA reaches after its last read of it
      }
    }
  }
  __threadfence();
  cluster.sync();
  if (tid == 0) { const long long t1 = phase_clock(); t_ph[4] = t1 - t0; t0 = t1; }

  // ---- back-transform y = H_0 (... (H_{m-2} z)): column rank + CL (warp + CL_NW c) ---
  {
    if (tid == 0) {
      tc::mbar_init(tc::smem_u32(&sh.mbar), 1);
      asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    // one pass over the reflectors; a warp carries two columns when there are more
    // than CL x CL_NW of them (every eigenvector for the FP64 refinement)
    const bool bt_ok = nvec > CL * CL_NW ? back_transform<T, 2>(sh, gref, gZ, evecs, m, nvec, rank)
                                         : back_transform<T, 1>(sh, gref, gZ, evecs, m, nvec, rank);
    if (!bt_ok && tid == 0) out->status = 3;  // a bounded wait gave up
  }
  cluster.sync();
  if (rank == 0 && tid == 0) {
    t_ph[5] = phase_clock() - t0;
    for (int q = 0; q < 6; ++q) out->cycles[q] = t_ph[q];
#ifdef LRET_EIG_PROFILE
    for (int q = 0; q < 6; ++q) out->cycles[q] = sp[q];
#if LRET_EIG_PROFILE >= 3
    out->cycles[0] = tloop1 - tloop0;      // cluster steps
    out->cycles[1] = tdbg[1] - tloop1;     // gather
    for (int q = 0; q < 4; ++q) out->cycles[2 + q] = tdbg[2 + q];  // matvec, barrier, group or update, barrier
#elif LRET_EIG_PROFILE != 2
    out->cycles[2] = sh.gdbg[0];  // x and its updates
    out->cycles[3] = sh.gdbg[1];  // first group barrier
    out->cycles[4] = sh.gdbg[2];  // norms and scalars
    out->cycles[5] = sh.gdbg[3];  // v, store
#endif
#endif
  }
}

template <typename T>
__global__ void __launch_bounds__(CL_THREADS, 1)
    k_eigh_cluster(const double2* __restrict__ G, int m, cx<T>* __restrict__ gref, T* __restrict__ gZ,
                   double* __restrict__ evals, double2* __restrict__ evecs, EigOut* __restrict__ out, int r,
                   double eps, int all_vecs) {
  eigh_cluster_body<T>(G, m, gref, gZ, evals, evecs, out, r, eps, all_vecs);
}

// One cluster of CL CTAs per task A.task[blockIdx.y]. The task list is a kernel
// parameter (constant bank): read through it, the solve keeps its arguments out of
// registers as the single-matrix kernel does.
struct ClusterBatchArgs {
  ClusterTask task[CL_BATCH_MAX];
  int all_vecs;
};

template <typename T>
__global__ void __launch_bounds__(CL_THREADS, 1)
    k_eigh_cluster_batch(const __grid_constant__ ClusterBatchArgs A) {
  const ClusterTask& tk = A.task[blockIdx.y];
  cx<T>* gref = (cx<T>*)tk.work;
  T* gZ = (T*)(gref + (size_t)CL_MAXM * CL_MAXM);
  const double eps = 0.0;
  eigh_cluster_body<T>(tk.G, tk.m, gref, gZ, tk.evals, tk.evecs, tk.out, tk.r, eps, A.all_vecs);
}

template <typename T>
size_t eigh_cluster_smem() {
  return sizeof(ClusterShared<T>) + (size_t)LuExtra<T>::slots * 6 * CL_MAXM * sizeof(T);
}

template <typename T>
cudaError_t launch_eigh_cluster(const double2* G, int m, void* work, double* evals, double2* evecs, EigOut* out,
                                int r, double eps, int all_vecs, cudaStream_t s) {
  if (m < 2 || m > CL_MAXM) return cudaErrorInvalidValue;
  const size_t smem = eigh_cluster_smem<T>();
  static std::atomic<uint64_t> attr_done{0};  // one per instantiation
  {
    cudaError_t e = set_dyn_smem_once(k_eigh_cluster<T>, (int)smem, attr_done);
    if (e != cudaSuccess) return e;
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
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_eigh_cluster<T>, G, m, gref, gZ, evals, evecs, out, r, eps, all_vecs);
  note_launches(1);
  return e;
}

template <typename T>
cudaError_t prepare_eigh_cluster_batch() {
  return cudaFuncSetAttribute(k_eigh_cluster_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)eigh_cluster_smem<T>());
}

template <typename T>
cudaError_t launch_eigh_cluster_batch(const ClusterTask* tasks, int n, int all_vecs, cudaStream_t s) {
  for (int t0 = 0; t0 < n; t0 += CL_BATCH_MAX) {
    const int cnt = n - t0 < CL_BATCH_MAX ? n - t0 : CL_BATCH_MAX;
    ClusterBatchArgs A;
    for (int i = 0; i < cnt; ++i) A.task[i] = tasks[t0 + i];
    A.all_vecs = all_vecs;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, cnt, 1);
    cfg.blockDim = dim3(CL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = eigh_cluster_smem<T>();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_eigh_cluster_batch<T>, A);
    note_launches(1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int eigh_cluster_max_m() { return CL_MAXM; }

size_t eigh_cluster_work_bytes(bool fp64) {
  const size_t e = fp64 ? sizeof(double) : sizeof(float);
  // reflectors (complex, last row tau), Z (real), three row buffers (complex)
  return (size_t)CL_MAXM * CL_MAXM * 2 * e + (size_t)CL_MAXM * CL_MAXM * e + (size_t)3 * CL_MAXM * 2 * e;
}

template cudaError_t launch_eigh_cluster<float>(const double2*, int, void*, double*, double2*, EigOut*, int, double,
                                                int, cudaStream_t);
template cudaError_t launch_eigh_cluster<double>(const double2*, int, void*, double*, double2*, EigOut*, int,
                                                 double, int, cudaStream_t);

template cudaError_t prepare_eigh_cluster_batch<float>();
template cudaError_t prepare_eigh_cluster_batch<double>();
template cudaError_t launch_eigh_cluster_batch<float>(const ClusterTask*, int, int, cudaStream_t);
template cudaError_t launch_eigh_cluster_batch<double>(const ClusterTask*, int, int, cudaStream_t);

}  // namespace lret
