// liblret host runtime: the C ABI of include/lret.h.
//
// A handle owns two N x cap slabs (V and the expansion target W, N = 2^n),
// the Gram / eigensolver workspaces and, when recording, the tape used by the
// adjoint pass. Gates and channels are queued and fused into one expansion
// kernel (Eqs. 3-4); a truncation (Sec. II.B) runs Gram -> eigensolve ->
// projection on the handle's stream without a host round trip unless the
// caller asks for a value.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "lret.h"

using namespace lret;
using zc = std::complex<double>;

namespace lret {
thread_local char g_errmsg[256];
void set_error(const char* fmt, const char* a, const char* b) { snprintf(g_errmsg, sizeof(g_errmsg), fmt, a, b); }
static std::atomic<long long> g_launches{0};
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace lret

extern "C" int64_t lr_launch_count(void) { return (int64_t)lret::launches_total(); }

namespace {

struct Stage {
  int type = 0;  // 0 = expansion, 1 = truncation, 2 = dense k-qubit gate, 3 = diagonal gate
  int c_in = 0, c_out = 0;
  GroupOp op{};
  DenseOp dop{};
  DiagOp gop{};
  void* gmat = nullptr;      // types 2/3: gate matrix / diagonal in the state's precision
  uint32_t* goff = nullptr;  // type 2: row offsets of the matrix indices
  int param_id = -1;
  int m = 0, k = 0;
  double2* U = nullptr;  // m x m eigenvectors (columns, descending)
  double* lam = nullptr; // m eigenvalues
  void* ckpt = nullptr;  // stage input snapshot (N x cap) or null
};

}  // namespace

struct lr_ctx {
  int n = 0;
  int64_t N = 0;
  int r = 0, dtype = 0, cap = 0;
  cudaStream_t stream = nullptr;
  size_t esz = 0;
  void* V = nullptr;
  void* W = nullptr;
  int c = 1;
  // queue
  bool has_gate = false;
  int gate_nq = 0, gate_q[2] = {0, 0}, gate_pid = -1;
  zc gate_U[16], gate_dU[16];
  bool gate_has_d = false;
  bool has_chan = false;
  int chan_q = 0, chan_K = 0;
  zc chan_M[4][4];
  double eps = 0.0;
  int solver = 0;  // 0 auto, 1 Jacobi, 2 tridiagonal, 3 cluster
  int eig_prec = LR_EIGP_REFINED;  // LR_C64: FP32 solve + FP64 refinement, FP32 only, or FP64 solve
  int eig_iters = 1;
  void* rf_work = nullptr;         // refinement workspace (allocated on first use)
  int last_m = 0;                  // size of the last eigenproblem (lr_last_eig)
  double* tlog = nullptr;          // per-truncation log (lr_set_trunc_log): records
  int64_t* tlog_n = nullptr;       // records written (device counter)
  int tlog_cap = 0;
  int path = 0;    // 0 structured truncation where it applies, 1 always expand V'
  double2* S = nullptr;   // pair Gram (2c x 2c)
  int* tc_status = nullptr;  // set by tensor-core kernels when a bounded wait gives up
  float* projB = nullptr;    // pre-split projection operand for the tensor-core projection
  // Trace anchoring of the tensor-core projection: its FP32 accumulation in tensor memory
  // shrinks the state by about 2e-7 per launch (measured), which would accumulate over a
  // deep circuit. The projection adds the squared norm of its output to proj_ssq; the
  // state is then s V with s = sqrt((1 - discarded mass so far) / |V|^2) (Tr rho = 1 -
  // discarded mass is exact for LRET with complete Kraus sets), and s is folded into the
  // next truncation's pair Gram (s^2) and projection (s), or applied to V before any other
  // use (scale_pending; expansions commute with it).
  double* proj_ssq = nullptr;  // [0] squared norm, [1] the scale s, [2 ..] per-block partials
  bool scale_pending = false;
  int use_tc = 1;
  double2* D = nullptr;   // pair projection (2c x 2k)
  // deferred pair projection: the state is [V_0 V_1] C on qubit pend_q, V holding
  // pend_cm materialised columns and h->c the state's columns; S holds the pair
  // Gram of the materialised V on pend_q
  bool pend = false;
  int pend_q = 0, pend_cm = 0;
  double2* pend_C = nullptr;   // 2 pend_cm x 2 c (row stride 2 c)
  double2* pend_C2 = nullptr;  // product scratch
  double2* S2 = nullptr;       // pair Gram of the deferred state (2c x 2c)
  double2* Ztmp = nullptr;     // C^dag S
  // workspaces
  double2* partials = nullptr;
  size_t partials_elems = 0;
  double2* G = nullptr;
  double* evals = nullptr;
  double2* evecs = nullptr;
  EigOut* eo = nullptr;
  void* eig_work = nullptr;
  double* acc = nullptr;       // [0] cumulative discarded, [1] last gap, [2] eig status, [3] compressions
  double* dscratch = nullptr;  // readout partials / small outputs
  size_t dscratch_elems = 0;
  double* samp = nullptr;      // measurement sampling: CDF, block sums and offsets, uniforms
  size_t samp_elems = 0;
  int64_t* samp_out = nullptr;
  int samp_shots = 0;
  void* gmat = nullptr;        // dense / diagonal gate operand (state precision)
  size_t gmat_bytes = 0;
  uint32_t* goff = nullptr;    // dense gate row offsets
  size_t goff_elems = 0;
  int goff_k = 0, goff_q[32] = {0};  // qubit list the offsets were built for
  uint64_t* d_xm = nullptr;
  uint64_t* d_zm = nullptr;
  double* d_coeff = nullptr;
  int masks_cap = 0;
  EigOut* h_eo = nullptr;  // pinned
  double* h_small = nullptr;  // pinned, 64 doubles
  int64_t ncomp = 0;
  // tape
  bool record = false;
  int ckpt_every = 0;
  std::vector<Stage> tape;
  // backward scratch
  void* vb[2] = {nullptr, nullptr};
  std::vector<void*> seg;
  double2 *bC = nullptr, *bFA = nullptr, *bT1 = nullptr, *bMcat = nullptr;
  double* bgrad = nullptr;
  int bgrad_cap = 0;
  double* bpart = nullptr;
  size_t bytes = 0;
  // per-kernel-class CUDA-event timing (lr_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  std::vector<std::pair<int, int>> ev_pending;  // (class, index of start event)
  int ev_next = 0;
  double kms[LR_NKCLASS] = {0};
  int64_t kcnt[LR_NKCLASS] = {0};
};

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      snprintf(g_errmsg, sizeof(g_errmsg), "%s: %s", #call, cudaGetErrorString(_e));   \
      return LR_ECUDA;                                                                 \
    }                                                                                  \
  } while (0)

namespace {

template <typename F>
cudaError_t by_dtype(int dtype, F f) {
  if (dtype == LR_C64) return f(float());
  return f(double());
}

int dmalloc(lr_ctx* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    snprintf(g_errmsg, sizeof(g_errmsg), "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LR_ENOMEM : LR_ECUDA;
  }
  h->bytes += bytes;
  return LR_OK;
}

void dfree(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

size_t slab_bytes(const lr_ctx* h) { return (size_t)h->N * h->cap * h->esz; }

void timer_drain(lr_ctx* h) {
  if (h->ev_pending.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto& pr : h->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[pr.second], h->ev[pr.second + 1]) == cudaSuccess) {
      h->kms[pr.first] += ms;
      h->kcnt[pr.first] += 1;
    }
  }
  h->ev_pending.clear();
  h->ev_next = 0;
}

// Returns the start-event index, or -1 when timing is off.
int tbeg(lr_ctx* h) {
  if (!h->timing) return -1;
  if (h->ev_next + 2 > (int)h->ev.size()) timer_drain(h);
  const int i = h->ev_next;
  h->ev_next += 2;
  cudaEventRecord(h->ev[i], h->stream);
  return i;
}

void tend(lr_ctx* h, int cls, int i) {
  if (i < 0) return;
  cudaEventRecord(h->ev[i + 1], h->stream);
  h->ev_pending.push_back({cls, i});
}

int check_unitary_like(const zc* U, int d) {
  for (int i = 0; i < d * d; ++i)
    if (!std::isfinite(U[i].real()) || !std::isfinite(U[i].imag())) return LR_EINVAL;
  return LR_OK;
}

// embed a one-qubit matrix K into the 4x4 basis (2*b(q0) + b(q1)); which = 0 -> acts on q0
void embed2(const zc K[4], int which, zc out[16]) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      const int a0 = a >> 1, a1 = a & 1, b0 = b >> 1, b1 = b & 1;
      zc v = 0;
      if (which == 0) v = (a1 == b1) ? K[a0 * 2 + b0] : zc(0);
      else v = (a0 == b0) ? K[a1 * 2 + b1] : zc(0);
      out[a * 4 + b] = v;
    }
}

void matmul(const zc* A, const zc* B, zc* C, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      zc s = 0;
      for (int l = 0; l < d; ++l) s += A[i * d + l] * B[l * d + j];
      C[i * d + j] = s;
    }
}

void put(double2& dst, zc v) { dst = make_double2(v.real(), v.imag()); }

// Build the group operator for the queued gate and/or channel.
void build_op(const lr_ctx* h, bool use_gate, bool use_chan, GroupOp* op, int* pid) {
  memset(op, 0, sizeof(GroupOp));
  *pid = -1;
  const bool grad = use_gate && h->gate_has_d && h->gate_pid >= 0;
  if (use_gate) {
    const int d = 1 << h->gate_nq;
    op->G = d;
    op->bits[0] = h->gate_q[0];
    op->bits[1] = h->gate_nq == 2 ? h->gate_q[1] : 0;
    if (use_chan) {
      op->K = h->chan_K;
      for (int al = 0; al < h->chan_K; ++al) {
        zc Kfull[16], M[16], dM[16];
        if (d == 2) {
          for (int i = 0; i < 4; ++i) Kfull[i] = h->chan_M[al][i];
        } else {
          embed2(h->chan_M[al], h->chan_q == h->gate_q[0] ? 0 : 1, Kfull);
        }
        matmul(Kfull, h->gate_U, M, d);
        if (grad) matmul(Kfull, h->gate_dU, dM, d);
        for (int a = 0; a < d; ++a)
          for (int g = 0; g < d; ++g) {
            put(op->M[al][a][g], M[a * d + g]);
            if (grad) put(op->dM[al][a][g], dM[a * d + g]);
          }
      }
    } else {
      op->K = 1;
      for (int a = 0; a < d; ++a)
        for (int g = 0; g < d; ++g) {
          put(op->M[0][a][g], h->gate_U[a * d + g]);
          if (grad) put(op->dM[0][a][g], h->gate_dU[a * d + g]);
        }
    }
    if (grad) {
      op->has_grad = 1;
      *pid = h->gate_pid;
    }
  } else {
    op->G = 2;
    op->bits[0] = h->chan_q;
    op->K = h->chan_K;
    for (int al = 0; al < h->chan_K; ++al)
      for (int a = 0; a < 2; ++a)
        for (int g = 0; g < 2; ++g) put(op->M[al][a][g], h->chan_M[al][a * 2 + g]);
  }
}

int snapshot(lr_ctx* h, Stage& st) {
  const bool at_ckpt = h->tape.empty() || (h->ckpt_every > 0 && (h->tape.size() % h->ckpt_every) == 0);
  if (!at_ckpt) return LR_OK;
  int rc = dmalloc(h, &st.ckpt, slab_bytes(h));
  if (rc) return rc;
  CK(cudaMemcpyAsync(st.ckpt, h->V, slab_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
  return LR_OK;
}

// A[i] *= s^power (complex128 small matrices)
__global__ void k_scale_c2(double2* __restrict__ A, int n, const double* __restrict__ s, int power) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double f = power == 2 ? s[0] * s[0] : s[0];
  A[i] = make_double2(A[i].x * f, A[i].y * f);
}

// |V|^2 = the projection blocks' partial squared norms ssq[2 ..], summed in a fixed order;
// s = sqrt((1 - discarded mass so far) / |V|^2) into ssq[1] (acc[0]: the discarded mass)
__global__ void __launch_bounds__(256) k_trace_scale(double* ssq, int nparts, const double* acc) {
  __shared__ double red[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) v += ssq[2 + i];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {  // fixed-order tree
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  v = red[0];
  if (threadIdx.x == 0) {
    const double t = 1.0 - acc[0];
    ssq[0] = v;
    ssq[1] = (v > 0.0 && t > 0.0) ? sqrt(t / v) : 1.0;
  }
}

// V[x][j] *= s for the c columns of a complex64 state
__global__ void k_scale_cols(float2* __restrict__ V, int64_t N, int c, int ld, const double* __restrict__ s) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N * c) return;
  const int64_t x = e / c;
  const int j = (int)(e - x * c);
  const float f = (float)s[0];
  float2& v = V[x * ld + j];
  v = make_float2(v.x * f, v.y * f);
}

// V <- [V_0 V_1] D on qubit q (D: 2c x 2k, row stride 2k), into W, then swap.
int run_pair_proj(lr_ctx* h, const double2* D, int c, int k, int q) {
  const int64_t N2 = h->N / 2;
  const int ld = h->cap;
  const int te = tbeg(h);
  if (h->dtype == LR_C64 && h->use_tc && proj_pair_tc_supported(c, k, N2)) {
    CK(launch_proj_pair_tc(h->V, ld, c, k, q, N2, D, h->projB, h->W, h->tc_status, h->proj_ssq + 2, h->stream));
    k_trace_scale<<<1, 256, 0, h->stream>>>(h->proj_ssq, proj_pair_tc_blocks(N2), h->acc);
    note_launches(1);
    h->scale_pending = true;
  } else {
    CK(by_dtype(h->dtype, [&](auto t) {
      return launch_rowmat<decltype(t)>(h->V, ld, 2 * c, D, 2 * k, nullptr, 0, 0, nullptr, 0, h->W, ld, 2 * k,
                                        N2, h->stream, q, c, k);
    }));
  }
  tend(h, LR_K_PROJECT, te);
  std::swap(h->V, h->W);
  return LR_OK;
}

// Apply a deferred pair projection, if any, so that V (up to a pending scale) holds the state.
int materialize_proj(lr_ctx* h) {
  if (!h->pend) return LR_OK;
  h->pend = false;
  return run_pair_proj(h, h->pend_C, h->pend_cm, h->c, h->pend_q);
}

// Apply a pending trace-anchoring scale to V.
int apply_scale(lr_ctx* h) {
  if (!h->scale_pending) return LR_OK;
  h->scale_pending = false;
  const int64_t n = h->N * (int64_t)h->c;  // only the complex64 tensor-core path sets a scale
  k_scale_cols<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>((float2*)h->V, h->N, h->c, h->cap,
                                                                    h->proj_ssq + 1);
  note_launches(1);
  CK(cudaGetLastError());
  return LR_OK;
}


// Run one expansion stage V -> W, swap. Queue flags are cleared by the caller.
int run_expand(lr_ctx* h, bool use_gate, bool use_chan) {
  {
    int rc = materialize_proj(h);  // a pending scale commutes with the expansion and stays pending
    if (rc) return rc;
  }
  GroupOp op;
  int pid;
  build_op(h, use_gate, use_chan, &op, &pid);
  const int c_out = h->c * op.K;
  if (c_out > h->cap) {
    snprintf(g_errmsg, sizeof(g_errmsg), "columns %d x %d exceed capacity %d", h->c, op.K, h->cap);
    return LR_ECAPACITY;
  }
  Stage st;
  if (h->record) {
    st.type = 0;
    st.c_in = h->c;
    st.c_out = c_out;
    st.op = op;
    st.param_id = pid;
    int rc = snapshot(h, st);
    if (rc) return rc;
  }
  const int64_t N = h->N;
  const int c = h->c, ld = h->cap;
  const int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_expand<decltype(t)>(h->V, h->W, N, c, ld, op, h->stream);
  }));
  tend(h, LR_K_EXPAND, te);
  std::swap(h->V, h->W);
  h->c = c_out;
  if (h->record) h->tape.push_back(st);
  return LR_OK;
}

int flush_gate(lr_ctx* h) {
  if (!h->has_gate) return LR_OK;
  int rc = run_expand(h, true, false);
  if (rc) return rc;
  h->has_gate = false;
  return LR_OK;
}

int flush_all(lr_ctx* h) {
  {
    int rc = materialize_proj(h);  // a pending scale commutes with gates and expansions
    if (rc) return rc;
  }
  if (h->has_chan) {
    int rc = run_expand(h, h->has_gate, true);
    if (rc) return rc;
    h->has_gate = false;
    h->has_chan = false;
    return LR_OK;
  }
  return flush_gate(h);
}

// Everything queued applied and any pending scale too: V holds the state (readouts).
int flush_state(lr_ctx* h) {
  int rc = flush_all(h);
  if (!rc) rc = apply_scale(h);
  return rc;
}

// Per-truncation accounting; with a log buffer (cap > 0) also one record per truncation:
// [m, k, lambda_1, lambda_k, lambda_{k+1}, discarded, trace, gap] (FP64).
// U[a][k + j] -= T[a][j] (a < m, j < m - k): the discarded columns of the eigenvector
// matrix made orthogonal to the kept ones (T = U_r (U_r^dag U_d))
__global__ void k_sub_cols(double2* __restrict__ U, int m, int k, const double2* __restrict__ T) {
  const int d = m - k;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * d) return;
  const int a = e / d, j = e % d;
  const double2 t = T[e];
  double2& u = U[(size_t)a * m + k + j];
  u = make_double2(u.x - t.x, u.y - t.y);
}

__global__ void k_accum(const EigOut* eo, const double* evals, int m, double* acc, double* log, int cap,
                        int64_t* nlog) {
  acc[0] += eo->dropped;
  acc[1] = eo->gap;
  if ((double)eo->status > acc[2]) acc[2] = (double)eo->status;
  acc[3] += 1.0;
  if (cap > 0) {
    const int64_t i = *nlog;
    if (i < cap) {
      const int k = eo->k;
      double* rec = log + i * LR_TRUNC_LOG_FIELDS;
      rec[0] = m;
      rec[1] = k;
      rec[2] = evals[0];
      rec[3] = k >= 1 ? evals[k - 1] : 0.0;
      rec[4] = k < m ? evals[k] : 0.0;
      rec[5] = eo->dropped;
      rec[6] = eo->trace;
      rec[7] = eo->gap;
    }
    *nlog = i + 1;
  }
}

int ensure_masks(lr_ctx* h, int T) {
  if (T <= h->masks_cap) return LR_OK;
  dfree((void*&)h->d_xm);
  dfree((void*&)h->d_zm);
  dfree((void*&)h->d_coeff);
  int cap = T < 64 ? 64 : T;
  int rc = dmalloc(h, (void**)&h->d_xm, sizeof(uint64_t) * cap);
  if (!rc) rc = dmalloc(h, (void**)&h->d_zm, sizeof(uint64_t) * cap);
  if (!rc) rc = dmalloc(h, (void**)&h->d_coeff, sizeof(double) * cap);
  if (rc) return rc;
  h->masks_cap = cap;
  return LR_OK;
}

int ensure_dscratch(lr_ctx* h, size_t elems) {
  if (elems <= h->dscratch_elems) return LR_OK;
  dfree((void*&)h->dscratch);
  int rc = dmalloc(h, (void**)&h->dscratch, sizeof(double) * elems);
  if (rc) return rc;
  h->dscratch_elems = elems;
  return LR_OK;
}

int upload_terms(lr_ctx* h, int T, const uint64_t* xm, const uint64_t* zm, const double* coeff) {
  const uint64_t lim = (h->n >= 64) ? ~0ull : ((1ull << h->n) - 1ull);
  for (int t = 0; t < T; ++t)
    if ((xm[t] & ~lim) || (zm[t] & ~lim)) return LR_EINVAL;
  int rc = ensure_masks(h, T);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->d_xm, xm, sizeof(uint64_t) * T, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_zm, zm, sizeof(uint64_t) * T, cudaMemcpyHostToDevice, h->stream));
  if (coeff) CK(cudaMemcpyAsync(h->d_coeff, coeff, sizeof(double) * T, cudaMemcpyHostToDevice, h->stream));
  return LR_OK;
}

// Eigensolve of the m x m Gram matrix in h->G (Sec. II.B), rank choice, FP64
// accounting; *k_out receives the kept count (synchronises only for the eps rule).
int run_eigh(lr_ctx* h, int m, int r_eff, double eps, int* k_out) {
  h->last_m = m;
  int te = tbeg(h);
  // arithmetic of the solver: FP64 for an FP64 state or when asked; the FP32 solve
  // of an FP32 state is followed by the FP64 refinement of the kept vectors unless
  // that is switched off
  const bool fp64 = h->dtype == LR_C128 || h->eig_prec == LR_EIGP_FP64;
  const int kmax = r_eff > 0 ? (r_eff < m ? r_eff : m) : m;
  const bool refine = !fp64 && h->eig_prec == LR_EIGP_REFINED && kmax < m;
  const int all_vecs = (h->record || refine) ? 1 : 0;
  const int sdt = fp64 ? LR_C128 : LR_C64;
  const bool small = m <= (fp64 ? 64 : 32);
  const bool use_cluster = h->solver == 3 || (h->solver == 0 && !small);
  const bool use_tri = h->solver == 2;
  if (use_cluster) {
    CK(by_dtype(sdt, [&](auto t) {
      return launch_eigh_cluster<decltype(t)>(h->G, m, h->eig_work, h->evals, h->evecs, h->eo, r_eff, eps,
                                              all_vecs, h->stream);
    }));
  } else if (use_tri) {
    CK(by_dtype(sdt, [&](auto t) {
      return launch_eigh_tri<decltype(t)>(h->G, m, h->eig_work, h->evals, h->evecs, h->eo, r_eff, eps, all_vecs,
                                          h->stream);
    }));
  } else {
    CK(by_dtype(sdt, [&](auto t) {
      return launch_eigh<decltype(t)>(h->G, m, h->eig_work, h->evals, h->evecs, h->eo, r_eff, eps, h->stream);
    }));
  }
  tend(h, LR_K_EIGH, te);
  if (refine && h->eig_iters > 0) {
    if (!h->rf_work) {
      int rc = dmalloc(h, &h->rf_work, eig_refine_work_bytes(256));
      if (rc) return rc;
    }
    te = tbeg(h);
    CK(launch_eig_refine(h->G, m, h->evals, h->evecs, h->eo, kmax, h->eig_iters, h->rf_work, h->stream));
    if (h->record) {
      // the adjoint (App. B derivative of the truncation) needs a complement basis
      // orthogonal to the refined kept vectors: the FP32 discarded vectors carry
      // components of about 2^-24 along them, which the 1 / (lambda_i - lambda_j) terms
      // would amplify (one classical Gram-Schmidt pass in FP64; the workspace is free)
      double2* W = (double2*)h->rf_work;
      double2* T = W + (size_t)m * m;
      const int d = m - kmax;
      CK(launch_zgemm_small(h->evecs, m, 1, h->evecs + kmax, m, W, d, kmax, d, m, h->stream));
      CK(launch_zgemm_small(h->evecs, m, 0, W, d, T, d, m, d, kmax, h->stream));
      k_sub_cols<<<(m * d + 255) / 256, 256, 0, h->stream>>>(h->evecs, m, kmax, T);
      note_launches(1);
    }
    tend(h, LR_K_EIGREFINE, te);
  }
  k_accum<<<1, 1, 0, h->stream>>>(h->eo, h->evals, m, h->acc, h->tlog, h->tlog_cap, h->tlog_n);
  note_launches(1);
  CK(cudaGetLastError());
  if (r_eff > 0) {
    *k_out = r_eff < m ? r_eff : m;
  } else {
    CK(cudaMemcpyAsync(h->h_eo, h->eo, sizeof(EigOut), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *k_out = h->h_eo->k;
  }
  return LR_OK;
}

// Truncation after a one-qubit channel without forming V' (the expansion is
// implicit): with M_a = Kt_a G (G the queued one-qubit gate on the channel's
// qubit, or I) and S = [V_0 V_1]^dag [V_0 V_1] (rows of V with the qubit's bit
// clear / set), the Gram of V' = [M_1 V, ..., M_K V] is
//   G'_ab = sum_{b,b'} (M_a^dag M_b)_{bb'} S_{bb'}              (blocks c x c),
// and the projection V' U_r acts on row pairs as [V_0 V_1] D with
//   D[(b,i)][(a,j)] = sum_al (M_al)_{ab} U[al c + i][j].
// The same rho results as expanding then truncating (Eq. 4, Sec. II.B).
int do_structured(lr_ctx* h, int r_eff, double eps, double* discarded_out) {
  const int c = h->c, K = h->chan_K, m = c * K, q = h->chan_q;
  const int64_t N2 = h->N / 2;
  const int ld = h->cap;
  PairQ pq;
  memset(&pq, 0, sizeof(pq));
  zc Gm[4] = {1, 0, 0, 1};
  if (h->has_gate) for (int i = 0; i < 4; ++i) Gm[i] = h->gate_U[i];
  zc M[4][4];
  for (int al = 0; al < K; ++al) {
    matmul(h->chan_M[al], Gm, M[al], 2);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) put(pq.M[al][a][b], M[al][a * 2 + b]);
  }
  for (int al = 0; al < K; ++al)
    for (int be = 0; be < K; ++be)
      for (int b = 0; b < 2; ++b)
        for (int bp = 0; bp < 2; ++bp) {
          zc acc = 0;
          for (int a = 0; a < 2; ++a) acc += std::conj(M[al][a * 2 + b]) * M[be][a * 2 + bp];
          put(pq.Q[al][be][b][bp], acc);
        }
  // A truncation on the qubit of a deferred projection continues it: with the
  // state [V_0 V_1] C, its pair Gram is C^dag S C (S the pair Gram of V), and the
  // new projection composes, C <- C D. Otherwise the deferred one is applied first.
  const bool fuse = h->pend && h->pend_q == q;
  if (h->pend && !fuse) {
    int rc = materialize_proj(h);  // a scale it leaves pending is folded in below
    if (rc) return rc;
  }
  // (a deferred projection never coexists with a pending scale: the scale is folded
  // into the projection matrix when the deferral starts)
  const bool fold_scale = h->scale_pending && !fuse;
  if (!h->pend_C) {
    const size_t big = sizeof(double2) * 512 * 512;
    int rc = dmalloc(h, (void**)&h->pend_C, big);
    if (!rc) rc = dmalloc(h, (void**)&h->pend_C2, big);
    if (!rc) rc = dmalloc(h, (void**)&h->S2, big);
    if (!rc) rc = dmalloc(h, (void**)&h->Ztmp, big);
    if (rc) return rc;
  }
  const int cm = fuse ? h->pend_cm : c;
  int te;
  if (fuse) {
    te = tbeg(h);
    CK(launch_zgemm_small(h->pend_C, 2 * c, 1, h->S, 2 * cm, h->Ztmp, 2 * cm, 2 * c, 2 * cm, 2 * cm, h->stream));
    CK(launch_zgemm_small(h->Ztmp, 2 * cm, 0, h->pend_C, 2 * c, h->S2, 2 * c, 2 * c, 2 * c, 2 * cm, h->stream));
    CK(launch_assemble_gram(h->S2, c, K, pq, h->G, h->stream));
    tend(h, LR_K_SMALL, te);
  } else {
    te = tbeg(h);
    const int splits = gram_splits(N2, 2 * c, 2 * c);
    if (h->dtype == LR_C64 && h->use_tc && gram_pair_tc_supported(c, N2)) {
      const int max_splits = (int)(h->partials_elems / ((size_t)4 * c * c));
      CK(launch_gram_pair_tc(h->V, ld, c, q, N2, h->partials, max_splits, h->S, h->tc_status, h->stream));
    } else {
      CK(by_dtype(h->dtype, [&](auto t) {
        return launch_gram<decltype(t)>(h->V, ld, 2 * c, h->V, ld, 2 * c, N2, true, h->partials, splits, h->S,
                                        h->stream, q, c);
      }));
    }
    tend(h, LR_K_GRAM, te);
    te = tbeg(h);
    if (fold_scale) {  // the state is s V: its pair Gram is s^2 S
      k_scale_c2<<<(4 * c * c + 255) / 256, 256, 0, h->stream>>>(h->S, 4 * c * c, h->proj_ssq + 1, 2);
      note_launches(1);
    }
    CK(launch_assemble_gram(h->S, c, K, pq, h->G, h->stream));
    tend(h, LR_K_SMALL, te);
  }
  int k;
  int rc = run_eigh(h, m, r_eff, eps, &k);
  if (rc) return rc;
  te = tbeg(h);
  CK(launch_build_proj(h->evecs, c, K, k, pq, h->D, h->stream));
  if (fuse) {
    CK(launch_zgemm_small(h->pend_C, 2 * c, 0, h->D, 2 * k, h->pend_C2, 2 * k, 2 * cm, 2 * k, 2 * c, h->stream));
    std::swap(h->pend_C, h->pend_C2);
  } else {
    CK(cudaMemcpyAsync(h->pend_C, h->D, sizeof(double2) * 4 * c * k, cudaMemcpyDeviceToDevice, h->stream));
    if (fold_scale) {  // and its projection s [V_0 V_1] D
      k_scale_c2<<<(4 * c * k + 255) / 256, 256, 0, h->stream>>>(h->pend_C, 4 * c * k, h->proj_ssq + 1, 1);
      note_launches(1);
      h->scale_pending = false;
    }
    h->pend_cm = c;
    h->pend_q = q;
  }
  tend(h, LR_K_SMALL, te);
  h->pend = true;  // the projection itself runs when the state is next needed
  h->c = k;
  h->ncomp++;
  h->has_gate = false;
  h->has_chan = false;
  if (discarded_out) {
    CK(cudaMemcpyAsync(h->h_eo, h->eo, sizeof(EigOut), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *discarded_out = h->h_eo->dropped;
  }
  return LR_OK;
}

int do_truncate(lr_ctx* h, int r_eff, double eps, double* discarded_out) {
  {
    int rc = apply_scale(h);  // (normally applied by flush_all already)
    if (rc) return rc;
  }
  const int m = h->c;
  const int64_t N = h->N;
  const int ld = h->cap;
  if (r_eff > 0 && m <= r_eff) {  // nothing to drop: rho unchanged, skip
    if (discarded_out) *discarded_out = 0.0;
    return LR_OK;
  }
  if (m > 256) {
    snprintf(g_errmsg, sizeof(g_errmsg), "truncation of %d columns exceeds the eigensolver limit 256", m);
    return LR_ECAPACITY;
  }
  Stage st;
  if (h->record) {
    st.type = 1;
    st.c_in = m;
    st.m = m;
    int rc = snapshot(h, st);
    if (rc) return rc;
  }
  const int splits = gram_splits(N, m, m);
  int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_gram<decltype(t)>(h->V, ld, m, h->V, ld, m, N, true, h->partials, splits, h->G, h->stream);
  }));
  tend(h, LR_K_GRAM, te);
  int k;
  int rc0 = run_eigh(h, m, r_eff, eps, &k);
  if (rc0) return rc0;
  te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_rowmat<decltype(t)>(h->V, ld, m, h->evecs, m, nullptr, 0, 0, nullptr, 0, h->W, ld, k, N,
                                      h->stream);
  }));
  tend(h, LR_K_PROJECT, te);
  std::swap(h->V, h->W);
  h->c = k;
  h->ncomp++;
  if (h->record) {
    st.k = k;
    st.c_out = k;
    int rc = dmalloc(h, (void**)&st.U, sizeof(double2) * m * m);
    if (!rc) rc = dmalloc(h, (void**)&st.lam, sizeof(double) * m);
    if (rc) return rc;
    CK(cudaMemcpyAsync(st.U, h->evecs, sizeof(double2) * m * m, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(st.lam, h->evals, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
    h->tape.push_back(st);
  }
  if (discarded_out) {
    CK(cudaMemcpyAsync(h->h_eo, h->eo, sizeof(EigOut), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *discarded_out = h->h_eo->dropped;
  }
  return LR_OK;
}

void clear_tape(lr_ctx* h) {
  for (auto& st : h->tape) {
    dfree(st.ckpt);
    dfree((void*&)st.U);
    dfree((void*&)st.lam);
    dfree(st.gmat);
    dfree((void*&)st.goff);
  }
  h->tape.clear();
}

// Copy `count` interleaved complex doubles to h->gmat in the state's precision
// (FP32 pairs for LR_C64), growing the buffer as needed.
int upload_gate_operand(lr_ctx* h, const double* src, size_t count) {
  const size_t bytes = count * h->esz;
  if (bytes > h->gmat_bytes) {
    dfree(h->gmat);
    h->gmat_bytes = 0;
    int rc = dmalloc(h, &h->gmat, bytes);
    if (rc) return rc;
    h->gmat_bytes = bytes;
  }
  CK(cudaStreamSynchronize(h->stream));  // the previous operand may still be in use
  if (h->dtype == LR_C64) {
    std::vector<float> tmp(2 * count);
    for (size_t i = 0; i < 2 * count; ++i) tmp[i] = (float)src[i];
    CK(cudaMemcpy(h->gmat, tmp.data(), bytes, cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(h->gmat, src, bytes, cudaMemcpyHostToDevice));
  }
  return LR_OK;
}

// Keep a private copy of a gate operand (and the current offsets) for the tape.
int tape_copy_operand(lr_ctx* h, Stage& st, const void* src, size_t count, int with_off, int D) {
  int rc = dmalloc(h, &st.gmat, count * h->esz);
  if (rc) return rc;
  CK(cudaMemcpyAsync(st.gmat, src, count * h->esz, cudaMemcpyDeviceToDevice, h->stream));
  if (with_off) {
    rc = dmalloc(h, (void**)&st.goff, sizeof(uint32_t) * D);
    if (rc) return rc;
    CK(cudaMemcpyAsync(st.goff, h->goff, sizeof(uint32_t) * D, cudaMemcpyDeviceToDevice, h->stream));
  }
  return LR_OK;
}

int set_initial_state(lr_ctx* h) {
  CK(cudaMemsetAsync(h->V, 0, slab_bytes(h), h->stream));
  // V[0][0] = 1
  if (h->dtype == LR_C64) {
    const float one[2] = {1.f, 0.f};
    CK(cudaMemcpyAsync(h->V, one, sizeof(one), cudaMemcpyHostToDevice, h->stream));
  } else {
    const double one[2] = {1.0, 0.0};
    CK(cudaMemcpyAsync(h->V, one, sizeof(one), cudaMemcpyHostToDevice, h->stream));
  }
  CK(cudaMemsetAsync(h->acc, 0, sizeof(double) * 8, h->stream));
  h->scale_pending = false;
  if (h->tlog_n) CK(cudaMemsetAsync(h->tlog_n, 0, sizeof(int64_t), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->c = 1;
  h->has_gate = h->has_chan = false;
  h->pend = false;
  h->ncomp = 0;
  clear_tape(h);
  return LR_OK;
}

// Dense k-qubit gate, 3 <= k <= LR_MAX_GATE_QUBITS: runs at once (not fused).
// The operand is either a host matrix of complex doubles (U_host, converted and
// uploaded here) or a caller-owned device matrix in the state's precision (U_dev).
int apply_dense(lr_ctx* h, int k, const int* qubits, const double* U_host, const void* U_dev) {
  const int D = 1 << k;
  const size_t cnt = (size_t)D * D;
  if (U_host)
    for (size_t i = 0; i < 2 * cnt; ++i)
      if (!std::isfinite(U_host[i])) return LR_EINVAL;
  int rc = flush_all(h);
  if (rc) return rc;
  DenseOp op{};
  op.k = k;
  for (int i = 0; i < k; ++i) op.pos[i] = qubits[i];
  std::sort(op.pos, op.pos + k);
  if (U_host) {
    rc = upload_gate_operand(h, U_host, cnt);  // synchronises
    if (rc) return rc;
  }
  // row offsets of the matrix indices; kept while the qubit list repeats
  bool same = h->goff && h->goff_k == k;
  for (int i = 0; same && i < k; ++i) same = h->goff_q[i] == qubits[i];
  if (!same) {
    std::vector<uint32_t> off(D);
    for (int a = 0; a < D; ++a) {
      uint32_t o = 0;
      for (int i = 0; i < k; ++i) o |= (uint32_t)((a >> (k - 1 - i)) & 1) << qubits[i];
      off[a] = o;
    }
    CK(cudaStreamSynchronize(h->stream));  // a previous gate may still read the table
    if ((size_t)D > h->goff_elems) {
      dfree((void*&)h->goff);
      h->goff_elems = 0;
      rc = dmalloc(h, (void**)&h->goff, sizeof(uint32_t) * D);
      if (rc) return rc;
      h->goff_elems = D;
    }
    CK(cudaMemcpy(h->goff, off.data(), sizeof(uint32_t) * D, cudaMemcpyHostToDevice));
    h->goff_k = k;
    for (int i = 0; i < k; ++i) h->goff_q[i] = qubits[i];
  }
  const void* G = U_host ? h->gmat : U_dev;
  Stage st;
  if (h->record) {
    st.type = 2;
    st.c_in = st.c_out = h->c;
    st.dop = op;
    rc = snapshot(h, st);
    if (!rc) rc = tape_copy_operand(h, st, G, cnt, 1, D);
    if (rc) return rc;
  }
  const int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_dense<decltype(t)>(h->V, h->W, h->N, h->c, h->cap, op, G, h->goff, 0, h->stream);
  }));
  tend(h, LR_K_EXPAND, te);
  std::swap(h->V, h->W);
  if (h->record) h->tape.push_back(st);
  return LR_OK;
}
}  // namespace

extern "C" {

const char* lr_status_string(int s) {
  switch (s) {
    case LR_OK: return "ok";
    case LR_EINVAL: return "invalid argument";
    case LR_EKRAUS: return "Kraus set is not complete (sum K^dag K != I)";
    case LR_ECAPACITY: return "column capacity exceeded";
    case LR_ENOMEM: return "device memory allocation failed";
    case LR_ETIMEOUT: return "bounded device wait timed out";
    case LR_ECUDA: return g_errmsg[0] ? g_errmsg : "CUDA error";
    case LR_ESTATE: return "call not valid in the current state";
    case LR_ENOCONV: return "eigensolver did not converge";
    default: return "unknown status";
  }
}

int lr_init_ex(int n, int r, int dtype, int capacity, void* stream, lr_handle* out) {
  if (!out) return LR_EINVAL;
  *out = nullptr;
  if (n < 1 || n > 30 || r < 1 || (dtype != LR_C64 && dtype != LR_C128)) return LR_EINVAL;
  if (capacity < r) return LR_EINVAL;
  lr_ctx* h = new lr_ctx();
  h->n = n;
  h->N = 1ll << n;
  h->r = r;
  h->dtype = dtype;
  h->cap = capacity + (capacity & 1);
  h->stream = (cudaStream_t)stream;
  h->esz = dtype == LR_C64 ? sizeof(float2) : sizeof(double2);
  const int m = h->cap < 256 ? h->cap : 256;
  // largest split-K workspace over every Gram shape a truncation or its adjoint can use
  size_t pe = 0;
  for (int ma = 1; ma <= m; ++ma) {
    const size_t a = (size_t)gram_splits(h->N, ma, ma) * ma * ma;
    if (a > pe) pe = a;
    for (int kb = 1; kb <= ma; kb += (kb < 8 ? 1 : 8)) {
      const size_t b = (size_t)gram_splits(h->N, ma, kb) * ma * kb;
      if (b > pe) pe = b;
    }
    const size_t b = (size_t)gram_splits(h->N, ma, ma) * ma * ma;
    if (b > pe) pe = b;
  }
  h->partials_elems = pe;
  int rc = dmalloc(h, &h->V, slab_bytes(h));
  if (!rc) rc = dmalloc(h, &h->W, slab_bytes(h));
  if (!rc) rc = dmalloc(h, (void**)&h->partials, sizeof(double2) * pe);
  if (!rc) rc = dmalloc(h, (void**)&h->G, sizeof(double2) * m * m);
  if (!rc) rc = dmalloc(h, (void**)&h->S, sizeof(double2) * m * m);
  if (!rc) rc = dmalloc(h, (void**)&h->tc_status, sizeof(int));
  if (!rc) rc = dmalloc(h, (void**)&h->proj_ssq, sizeof(double) * (2 + proj_pair_tc_blocks(h->N / 2)));
  if (!rc) rc = dmalloc(h, (void**)&h->projB, proj_pair_tc_scratch_bytes(64, 64));
  if (!rc && cudaMemset(h->tc_status, 0, sizeof(int)) != cudaSuccess) rc = LR_ECUDA;
  if (!rc) rc = dmalloc(h, (void**)&h->D, sizeof(double2) * m * m);
  if (!rc) rc = dmalloc(h, (void**)&h->evals, sizeof(double) * m);
  if (!rc) rc = dmalloc(h, (void**)&h->evecs, sizeof(double2) * m * m);
  if (!rc) rc = dmalloc(h, (void**)&h->eo, sizeof(EigOut));
  if (!rc) {
    // FP64 sizes for every dtype: the entropy readout runs the FP64 solvers
    size_t wb = eigh_work_bytes(m, true);
    const size_t wc = eigh_cluster_work_bytes(true);
    rc = dmalloc(h, &h->eig_work, wb > wc ? wb : wc);
  }
  if (!rc) rc = dmalloc(h, (void**)&h->acc, sizeof(double) * 8);
  if (!rc) rc = ensure_dscratch(h, 64 * 1024);
  if (!rc && cudaMallocHost((void**)&h->h_eo, sizeof(EigOut)) != cudaSuccess) rc = LR_ENOMEM;
  if (!rc && cudaMallocHost((void**)&h->h_small, sizeof(double) * 64) != cudaSuccess) rc = LR_ENOMEM;
  if (!rc) rc = set_initial_state(h);
  if (rc) {
    lr_free(h);
    return rc;
  }
  *out = h;
  return LR_OK;
}

int lr_init(int n, int r, int dtype, void* stream, lr_handle* out) {
  return lr_init_ex(n, r, dtype, 4 * r, stream, out);
}

int lr_free(lr_handle h) {
  if (!h) return LR_EINVAL;
  cudaStreamSynchronize(h->stream);
  clear_tape(h);
  dfree(h->V);
  dfree(h->W);
  dfree((void*&)h->partials);
  dfree((void*&)h->G);
  dfree((void*&)h->S);
  dfree((void*&)h->tc_status);
  dfree((void*&)h->proj_ssq);
  dfree((void*&)h->projB);
  dfree((void*&)h->D);
  dfree((void*&)h->pend_C);
  dfree((void*&)h->pend_C2);
  dfree((void*&)h->S2);
  dfree((void*&)h->Ztmp);
  dfree((void*&)h->evals);
  dfree((void*&)h->evecs);
  dfree((void*&)h->eo);
  dfree(h->eig_work);
  dfree(h->rf_work);
  dfree((void*&)h->tlog);
  dfree((void*&)h->tlog_n);
  dfree((void*&)h->acc);
  dfree((void*&)h->dscratch);
  dfree((void*&)h->samp);
  dfree((void*&)h->samp_out);
  dfree(h->gmat);
  dfree((void*&)h->goff);
  dfree((void*&)h->d_xm);
  dfree((void*&)h->d_zm);
  dfree((void*&)h->d_coeff);
  dfree(h->vb[0]);
  dfree(h->vb[1]);
  for (auto& p : h->seg) dfree(p);
  dfree((void*&)h->bC);
  dfree((void*&)h->bFA);
  dfree((void*&)h->bT1);
  dfree((void*&)h->bMcat);
  dfree((void*&)h->bgrad);
  dfree((void*&)h->bpart);
  for (auto e : h->ev) cudaEventDestroy(e);
  if (h->h_eo) cudaFreeHost(h->h_eo);
  if (h->h_small) cudaFreeHost(h->h_small);
  delete h;
  return LR_OK;
}

int lr_reset(lr_handle h) {
  if (!h) return LR_EINVAL;
  return set_initial_state(h);
}


int lr_apply_diagonal(lr_handle h, int nq, const int* qubits, const double* diag) {
  if (!h || !qubits || !diag || nq < 1 || nq > h->n || nq > 30) return LR_EINVAL;
  for (int i = 0; i < nq; ++i) {
    if (qubits[i] < 0 || qubits[i] >= h->n) return LR_EINVAL;
    for (int j = 0; j < i; ++j)
      if (qubits[j] == qubits[i]) return LR_EINVAL;
  }
  const size_t cnt = (size_t)1 << nq;
  for (size_t i = 0; i < 2 * cnt; ++i)
    if (!std::isfinite(diag[i])) return LR_EINVAL;
  int rc = flush_all(h);
  if (rc) return rc;
  DiagOp op{};
  op.k = nq;
  for (int i = 0; i < nq; ++i) op.q[i] = qubits[i];
  rc = upload_gate_operand(h, diag, cnt);
  if (rc) return rc;
  Stage st;
  if (h->record) {
    st.type = 3;
    st.c_in = st.c_out = h->c;
    st.gop = op;
    rc = snapshot(h, st);
    if (!rc) rc = tape_copy_operand(h, st, h->gmat, cnt, 0, 0);
    if (rc) return rc;
  }
  const int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_diag<decltype(t)>(h->V, h->V, h->N, h->c, h->cap, op, h->gmat, 0, h->stream);
  }));
  tend(h, LR_K_EXPAND, te);
  if (h->record) h->tape.push_back(st);
  return LR_OK;
}

int lr_apply_gate_device(lr_handle h, int nq, const int* qubits, const void* U_dev) {
  if (!h || !qubits || !U_dev || nq < 3 || nq > LR_MAX_GATE_QUBITS || nq > h->n) return LR_EINVAL;
  for (int i = 0; i < nq; ++i) {
    if (qubits[i] < 0 || qubits[i] >= h->n) return LR_EINVAL;
    for (int j = 0; j < i; ++j)
      if (qubits[j] == qubits[i]) return LR_EINVAL;
  }
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, U_dev) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return LR_EINVAL;
  }
  return apply_dense(h, nq, qubits, nullptr, U_dev);
}

int lr_apply_gate(lr_handle h, int nq, const int* qubits, const double* U, const double* dU, int param_id) {
  if (!h || !qubits || !U || nq < 1 || nq > LR_MAX_GATE_QUBITS || nq > h->n) return LR_EINVAL;
  if (nq >= 3) {
    for (int i = 0; i < nq; ++i) {
      if (qubits[i] < 0 || qubits[i] >= h->n) return LR_EINVAL;
      for (int j = 0; j < i; ++j)
        if (qubits[j] == qubits[i]) return LR_EINVAL;
    }
    if (param_id >= 0 || dU) return LR_EINVAL;  // dense gates are fixed
    return apply_dense(h, nq, qubits, U, nullptr);
  }
  for (int i = 0; i < nq; ++i)
    if (qubits[i] < 0 || qubits[i] >= h->n) return LR_EINVAL;
  if (nq == 2 && qubits[0] == qubits[1]) return LR_EINVAL;
  if (param_id >= 0 && !dU) return LR_EINVAL;
  const int d = 1 << nq;
  zc Uc[16], dUc[16];
  for (int i = 0; i < d * d; ++i) {
    Uc[i] = zc(U[2 * i], U[2 * i + 1]);
    dUc[i] = dU ? zc(dU[2 * i], dU[2 * i + 1]) : zc(0);
  }
  if (check_unitary_like(Uc, d)) return LR_EINVAL;
  // a queued channel or gate runs first; a deferred projection stays deferred for a
  // one-qubit gate on its qubit (the next truncation there can continue it)
  const bool keep = h->pend && !h->has_gate && !h->has_chan && nq == 1 && qubits[0] == h->pend_q;
  int rc = keep ? LR_OK : flush_all(h);
  if (rc) return rc;
  h->has_gate = true;
  h->gate_nq = nq;
  h->gate_q[0] = qubits[0];
  h->gate_q[1] = nq == 2 ? qubits[1] : 0;
  h->gate_pid = param_id;
  h->gate_has_d = (dU != nullptr) && param_id >= 0;
  for (int i = 0; i < 16; ++i) {
    h->gate_U[i] = i < d * d ? Uc[i] : zc(0);
    h->gate_dU[i] = i < d * d ? dUc[i] : zc(0);
  }
  return LR_OK;
}

int lr_apply_rotation(lr_handle h, int axis, int q, double theta, int param_id) {
  if (!h || axis < 0 || axis > 2) return LR_EINVAL;
  const zc I(0, 1);
  zc S[4];
  if (axis == 0) { S[0] = 0; S[1] = 1; S[2] = 1; S[3] = 0; }
  else if (axis == 1) { S[0] = 0; S[1] = -I; S[2] = I; S[3] = 0; }
  else { S[0] = 1; S[1] = 0; S[2] = 0; S[3] = -1; }
  const double cs = std::cos(theta / 2), sn = std::sin(theta / 2);
  zc U[4], dU[4];
  for (int i = 0; i < 4; ++i) U[i] = ((i == 0 || i == 3) ? cs : 0.0) - I * sn * S[i];
  // dU = -i/2 S U
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) dU[a * 2 + b] = -0.5 * I * (S[a * 2] * U[b] + S[a * 2 + 1] * U[2 + b]);
  double Ud[8], dUd[8];
  for (int i = 0; i < 4; ++i) {
    Ud[2 * i] = U[i].real(); Ud[2 * i + 1] = U[i].imag();
    dUd[2 * i] = dU[i].real(); dUd[2 * i + 1] = dU[i].imag();
  }
  return lr_apply_gate(h, 1, &q, Ud, dUd, param_id);
}

int lr_apply_kraus(lr_handle h, int q, int K, const double* kraus) {
  if (!h || !kraus || K < 1 || K > 4 || q < 0 || q >= h->n) return LR_EINVAL;
  zc M[4][4];
  for (int al = 0; al < K; ++al)
    for (int i = 0; i < 4; ++i) {
      M[al][i] = zc(kraus[al * 8 + 2 * i], kraus[al * 8 + 2 * i + 1]);
      if (!std::isfinite(M[al][i].real()) || !std::isfinite(M[al][i].imag())) return LR_EINVAL;
    }
  // completeness: sum_a K_a^dag K_a = I
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      zc s = 0;
      for (int al = 0; al < K; ++al)
        for (int l = 0; l < 2; ++l) s += std::conj(M[al][l * 2 + i]) * M[al][l * 2 + j];
      if (std::abs(s - zc(i == j ? 1.0 : 0.0)) > 1e-10) return LR_EKRAUS;
    }
  // a queued channel, or a gate that does not touch q, runs first
  if (h->has_chan) {
    int rc = flush_all(h);
    if (rc) return rc;
  }
  if (h->has_gate) {
    const bool touches = h->gate_q[0] == q || (h->gate_nq == 2 && h->gate_q[1] == q);
    if (!touches) {
      int rc = flush_gate(h);
      if (rc) return rc;
    }
  }
  if (h->c * K > h->cap) return LR_ECAPACITY;
  h->has_chan = true;
  h->chan_q = q;
  h->chan_K = K;
  for (int al = 0; al < 4; ++al)
    for (int i = 0; i < 4; ++i) h->chan_M[al][i] = al < K ? M[al][i] : zc(0);
  return LR_OK;
}

int lr_kraus_preset(int kind, double p, double* out, int* K_out) {
  if (!out || !K_out || !(p >= 0.0 && p <= 1.0)) return LR_EINVAL;
  for (int i = 0; i < 32; ++i) out[i] = 0.0;
  // out[al*8 + 2*(row*2 + col) + {0: re, 1: im}]
  auto set = [&](int al, int row, int col, double re, double im) {
    out[al * 8 + 2 * (row * 2 + col)] = re;
    out[al * 8 + 2 * (row * 2 + col) + 1] = im;
  };
  if (kind == LR_DEPOLARIZING) {
    const double a = std::sqrt(1.0 - p), b = std::sqrt(p / 3.0);
    set(0, 0, 0, a, 0); set(0, 1, 1, a, 0);            // sqrt(1-p) I
    set(1, 0, 1, b, 0); set(1, 1, 0, b, 0);            // sqrt(p/3) X
    set(2, 0, 1, 0, -b); set(2, 1, 0, 0, b);           // sqrt(p/3) Y
    set(3, 0, 0, b, 0); set(3, 1, 1, -b, 0);           // sqrt(p/3) Z
    *K_out = 4;
  } else if (kind == LR_AMPLITUDE_DAMPING) {
    set(0, 0, 0, 1.0, 0); set(0, 1, 1, std::sqrt(1.0 - p), 0);
    set(1, 0, 1, std::sqrt(p), 0);
    *K_out = 2;
  } else if (kind == LR_BIT_FLIP) {
    const double a = std::sqrt(1.0 - p), b = std::sqrt(p);
    set(0, 0, 0, a, 0); set(0, 1, 1, a, 0);
    set(1, 0, 1, b, 0); set(1, 1, 0, b, 0);
    *K_out = 2;
  } else {
    return LR_EINVAL;
  }
  return LR_OK;
}

int lr_set_eigensolver(lr_handle h, int which) {
  if (!h || which < 0 || which > 3) return LR_EINVAL;
  h->solver = which;
  return LR_OK;
}

int lr_set_eig_precision(lr_handle h, int mode, int iters) {
  if (!h || mode < LR_EIGP_REFINED || mode > LR_EIGP_FP64) return LR_EINVAL;
  h->eig_prec = mode;
  h->eig_iters = iters < 0 ? 0 : (iters > 4 ? 4 : iters);
  return LR_OK;
}

int lr_set_trunc_log(lr_handle h, int capacity) {
  if (!h || capacity < 0) return LR_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  dfree((void*&)h->tlog);
  dfree((void*&)h->tlog_n);
  h->tlog_cap = 0;
  if (capacity == 0) return LR_OK;
  int rc = dmalloc(h, (void**)&h->tlog, sizeof(double) * LR_TRUNC_LOG_FIELDS * (size_t)capacity);
  if (!rc) rc = dmalloc(h, (void**)&h->tlog_n, sizeof(int64_t));
  if (rc) return rc;
  CK(cudaMemsetAsync(h->tlog_n, 0, sizeof(int64_t), h->stream));
  h->tlog_cap = capacity;
  return LR_OK;
}

int lr_get_trunc_log(lr_handle h, double* out_host, int max_records, int64_t* count_out) {
  if (!h || !count_out || max_records < 0 || (max_records > 0 && !out_host)) return LR_EINVAL;
  if (h->tlog_cap == 0) {
    *count_out = 0;
    return LR_OK;
  }
  int rc = flush_all(h);
  if (rc) return rc;
  int64_t n = 0;
  CK(cudaMemcpyAsync(&n, h->tlog_n, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int64_t stored = n < h->tlog_cap ? n : h->tlog_cap;
  const int64_t copy = stored < max_records ? stored : max_records;
  if (copy > 0)
    CK(cudaMemcpy(out_host, h->tlog, sizeof(double) * LR_TRUNC_LOG_FIELDS * (size_t)copy, cudaMemcpyDeviceToHost));
  *count_out = n;
  return LR_OK;
}

int lr_set_eps(lr_handle h, double eps) {
  if (!h || !(eps < 1.0)) return LR_EINVAL;
  h->eps = eps > 0 ? eps : 0.0;
  return LR_OK;
}

int lr_compress(lr_handle h, int r, double* discarded_out) {
  if (!h) return LR_EINVAL;
  int r_eff = r;
  double eps = 0.0;
  if (r <= 0) {
    if (h->eps > 0) { r_eff = 0; eps = h->eps; }
    else r_eff = h->r;
  }
  int rc;
  if (h->has_chan && h->path == 0 && !h->record) {
    // a gate the structured form cannot absorb (two-qubit, or on another qubit) runs first
    if (h->has_gate && !(h->gate_nq == 1 && h->gate_q[0] == h->chan_q)) {
      rc = flush_gate(h);
      if (rc) return rc;
    }
    const int m = h->c * h->chan_K;
    const bool drops = !(r_eff > 0 && m <= r_eff);
    if (drops && m <= 256 && m <= h->cap && (h->N >= 2)) return do_structured(h, r_eff, eps, discarded_out);
  }
  rc = flush_all(h);
  if (rc) return rc;
  return do_truncate(h, r_eff, eps, discarded_out);
}

int lr_set_tensor_cores(lr_handle h, int on) {
  if (!h) return LR_EINVAL;
  h->use_tc = on != 0;
  return LR_OK;
}

int lr_set_path(lr_handle h, int which) {
  if (!h || which < 0 || which > 1) return LR_EINVAL;
  h->path = which;
  return LR_OK;
}

int lr_probs(lr_handle h, void* out_dev) {
  if (!h || !out_dev) return LR_EINVAL;
  int rc = flush_state(h);
  if (rc) return rc;
  const int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_probs<decltype(t)>(h->V, h->N, h->c, h->cap, out_dev, h->stream);
  }));
  tend(h, LR_K_READOUT, te);
  return LR_OK;
}

int lr_sample(lr_handle h, int shots, const double* uniforms, int64_t* out_host) {
  if (!h || shots < 0 || (shots > 0 && (!uniforms || !out_host))) return LR_EINVAL;
  for (int s = 0; s < shots; ++s)
    if (!(uniforms[s] >= 0.0 && uniforms[s] < 1.0)) return LR_EINVAL;
  if (shots == 0) return LR_OK;
  int rc = flush_state(h);
  if (rc) return rc;
  const int64_t nb = (h->N + SC_ROWS - 1) / SC_ROWS;
  const size_t need = (size_t)h->N + 2 * (size_t)nb + 1 + (size_t)shots;
  if (need > h->samp_elems) {
    dfree((void*&)h->samp);
    h->samp_elems = 0;
    rc = dmalloc(h, (void**)&h->samp, sizeof(double) * need);
    if (rc) return rc;
    h->samp_elems = need;
  }
  if (shots > h->samp_shots) {
    dfree((void*&)h->samp_out);
    h->samp_shots = 0;
    rc = dmalloc(h, (void**)&h->samp_out, sizeof(int64_t) * shots);
    if (rc) return rc;
    h->samp_shots = shots;
  }
  double* cdf = h->samp;
  double* bsum = cdf + h->N;
  double* boff = bsum + nb;  // nb + 1 values
  double* u = boff + nb + 1;
  CK(cudaMemcpyAsync(u, uniforms, sizeof(double) * shots, cudaMemcpyHostToDevice, h->stream));
  const int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_sample<decltype(t)>(h->V, h->N, h->c, h->cap, cdf, bsum, boff, u, shots, h->samp_out, h->stream);
  }));
  tend(h, LR_K_READOUT, te);
  CK(cudaMemcpyAsync(out_host, h->samp_out, sizeof(int64_t) * shots, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LR_OK;
}

int lr_entropy(lr_handle h, double* out_host) {
  if (!h || !out_host) return LR_EINVAL;
  int rc = flush_state(h);
  if (rc) return rc;
  const int c = h->c;
  if (c > 256) {
    snprintf(g_errmsg, sizeof(g_errmsg), "entropy of %d columns exceeds the eigensolver limit 256", c);
    return LR_ECAPACITY;
  }
  double* outd = h->dscratch;  // S, 2^S
  if (c == 1) {
    // one column: rho has rank one (pure up to normalisation)
    out_host[0] = 0.0;
    out_host[1] = 1.0;
    return LR_OK;
  }
  // spectrum of V^dag V in FP64 (Theorem 1): the FP64 solvers whatever the dtype
  const int splits = gram_splits(h->N, c, c);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_gram<decltype(t)>(h->V, h->cap, c, h->V, h->cap, c, h->N, true, h->partials, splits, h->G,
                                    h->stream);
  }));
  if (c <= 64) {
    CK(launch_eigh<double>(h->G, c, h->eig_work, h->evals, h->evecs, h->eo, c, 0.0, h->stream));
  } else {
    CK(launch_eigh_cluster<double>(h->G, c, h->eig_work, h->evals, h->evecs, h->eo, 1, 0.0, 0, h->stream));
  }
  CK(launch_entropy(h->evals, c, outd, h->stream));
  CK(cudaMemcpyAsync(h->h_small, outd, sizeof(double) * 2, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out_host[0] = h->h_small[0];
  out_host[1] = h->h_small[1];
  return LR_OK;
}

int lr_z_expect(lr_handle h, double* out_host) {
  if (!h || !out_host) return LR_EINVAL;
  int rc = flush_state(h);
  if (rc) return rc;
  double* outd = h->dscratch;              // n + 1 values
  double* part = h->dscratch + 64;         // <= 1024 * 32 partials
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_zexp<decltype(t)>(h->V, h->N, h->c, h->cap, h->n, part, outd, h->stream);
  }));
  CK(cudaMemcpyAsync(h->h_small, outd, sizeof(double) * (h->n + 1), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  memcpy(out_host, h->h_small, sizeof(double) * (h->n + 1));
  return LR_OK;
}

int lr_expect(lr_handle h, int T, const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
              double* out_host) {
  if (!h || T < 0 || !out_host || (T > 0 && (!xmask || !zmask || !coeff))) return LR_EINVAL;
  int rc = flush_state(h);
  if (rc) return rc;
  if (T == 0) { *out_host = 0.0; return LR_OK; }
  rc = upload_terms(h, T, xmask, zmask, coeff);
  if (rc) return rc;
  rc = ensure_dscratch(h, (size_t)T * 1025 + 64);
  if (rc) return rc;
  double* outd = h->dscratch;
  double* part = h->dscratch + T;
  const int te = tbeg(h);
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_pauli_expect<decltype(t)>(h->V, h->N, h->c, h->cap, T, h->d_xm, h->d_zm, part, outd,
                                            h->stream);
  }));
  tend(h, LR_K_PAULI, te);
  std::vector<double> vals(T);
  CK(cudaMemcpyAsync(vals.data(), outd, sizeof(double) * T, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  double s = 0.0;
  for (int t = 0; t < T; ++t) s += coeff[t] * vals[t];
  *out_host = s;
  return LR_OK;
}

int lr_set_record(lr_handle h, int on) {
  if (!h) return LR_EINVAL;
  if (on && !h->record && (h->c != 1 || h->ncomp != 0 || h->has_gate || h->has_chan)) {
    // recording must start from the initial state so the tape covers the circuit
    return LR_ESTATE;
  }
  h->record = on != 0;
  if (!h->record) clear_tape(h);
  return LR_OK;
}

int lr_set_checkpoint(lr_handle h, int every) {
  if (!h || every < 0) return LR_EINVAL;
  if (!h->tape.empty()) return LR_ESTATE;
  h->ckpt_every = every;
  return LR_OK;
}

int lr_backward(lr_handle h, int T, const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                int nparams, double* grad_out_host) {
  if (!h || T <= 0 || !xmask || !zmask || !coeff || nparams < 0 || (nparams > 0 && !grad_out_host))
    return LR_EINVAL;
  if (!h->record) return LR_ESTATE;
  int rc = flush_state(h);
  if (rc) return rc;
  for (auto& st : h->tape)
    if (st.type == 0 && st.param_id >= nparams) return LR_EINVAL;
  rc = upload_terms(h, T, xmask, zmask, coeff);
  if (rc) return rc;
  const int64_t N = h->N;
  const int ld = h->cap;
  const size_t sb = slab_bytes(h);
  // scratch
  for (int i = 0; i < 2; ++i)
    if (!h->vb[i]) { rc = dmalloc(h, &h->vb[i], sb); if (rc) return rc; }
  const int mmax = h->cap < 256 ? h->cap : 256;
  if (!h->bC) {
    rc = dmalloc(h, (void**)&h->bC, sizeof(double2) * mmax * mmax);
    if (!rc) rc = dmalloc(h, (void**)&h->bFA, sizeof(double2) * mmax * mmax);
    if (!rc) rc = dmalloc(h, (void**)&h->bT1, sizeof(double2) * mmax * mmax);
    if (!rc) rc = dmalloc(h, (void**)&h->bMcat, sizeof(double2) * 2 * mmax * mmax);
    if (!rc) rc = dmalloc(h, (void**)&h->bpart, sizeof(double) * 4096);
    if (rc) return rc;
  }
  if (nparams + 1 > h->bgrad_cap) {
    dfree((void*&)h->bgrad);
    rc = dmalloc(h, (void**)&h->bgrad, sizeof(double) * (nparams + 1));
    if (rc) return rc;
    h->bgrad_cap = nparams + 1;
  }
  CK(cudaMemsetAsync(h->bgrad, 0, sizeof(double) * (nparams + 1), h->stream));
  // seed: Vbar = H V
  int cur = 0;
  CK(by_dtype(h->dtype, [&](auto t) {
    return launch_pauli_apply<decltype(t)>(h->V, h->vb[cur], N, h->c, ld, T, h->d_xm, h->d_zm, h->d_coeff,
                                           h->stream);
  }));
  const int S = (int)h->tape.size();
  // segments start at stages that hold a snapshot
  int s1 = S;
  while (s1 > 0) {
    int s0 = s1 - 1;
    while (s0 > 0 && h->tape[s0].ckpt == nullptr) --s0;
    const int len = s1 - s0;
    while ((int)h->seg.size() < len) {
      void* p = nullptr;
      rc = dmalloc(h, &p, sb);
      if (rc) return rc;
      h->seg.push_back(p);
    }
    // recompute stage inputs seg[i] = input of stage s0 + i
    CK(cudaMemcpyAsync(h->seg[0], h->tape[s0].ckpt, sb, cudaMemcpyDeviceToDevice, h->stream));
    for (int s = s0; s < s1 - 1; ++s) {
      const Stage& st = h->tape[s];
      void* in = h->seg[s - s0];
      void* outp = h->seg[s - s0 + 1];
      if (st.type == 0) {
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_expand<decltype(t)>(in, outp, N, st.c_in, ld, st.op, h->stream);
        }));
      } else if (st.type == 2) {
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_dense<decltype(t)>(in, outp, N, st.c_in, ld, st.dop, st.gmat, st.goff, 0, h->stream);
        }));
      } else if (st.type == 3) {
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_diag<decltype(t)>(in, outp, N, st.c_in, ld, st.gop, st.gmat, 0, h->stream);
        }));
      } else {
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_rowmat<decltype(t)>(in, ld, st.m, st.U, st.m, nullptr, 0, 0, nullptr, 0, outp, ld, st.k,
                                            N, h->stream);
        }));
      }
    }
    // backward through the segment
    for (int s = s1 - 1; s >= s0; --s) {
      const Stage& st = h->tape[s];
      void* in = h->seg[s - s0];
      void* vbar = h->vb[cur];
      void* vbin = h->vb[cur ^ 1];
      if (st.type == 0) {
        int nb = 0;
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_expand_adj<decltype(t)>(vbar, in, vbin, N, st.c_in, ld, st.op, h->bpart, &nb,
                                                h->stream);
        }));
        if (st.op.has_grad && st.param_id >= 0)
          CK(launch_sum(h->bpart, nb, h->bgrad + st.param_id, 1, h->stream));
      } else if (st.type == 2) {
        // Vbar_in = G^dag Vbar_out
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_dense<decltype(t)>(vbar, vbin, N, st.c_in, ld, st.dop, st.gmat, st.goff, 1, h->stream);
        }));
      } else if (st.type == 3) {
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_diag<decltype(t)>(vbar, vbin, N, st.c_in, ld, st.gop, st.gmat, 1, h->stream);
        }));
      } else {
        const int m = st.m, k = st.k;
        const int splits = gram_splits(N, m, k);
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_gram<decltype(t)>(in, ld, m, vbar, ld, k, N, false, h->partials, splits, h->bC,
                                          h->stream);
        }));
        CK(launch_trunc_adj_small(h->bC, st.U, st.lam, m, k, h->bFA, h->bT1, h->bMcat, h->stream));
        CK(by_dtype(h->dtype, [&](auto t) {
          return launch_rowmat<decltype(t)>(vbar, ld, k, h->bMcat, m, in, ld, m, h->bMcat + (size_t)k * m, m,
                                            vbin, ld, m, N, h->stream);
        }));
      }
      cur ^= 1;
    }
    s1 = s0;
  }
  if (nparams > 0) {
    CK(cudaMemcpyAsync(grad_out_host, h->bgrad, sizeof(double) * nparams, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return LR_OK;
}

int lr_get_info(lr_handle h, lr_info* info) {
  if (!h || !info) return LR_EINVAL;
  int rc = flush_all(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->h_small, h->acc, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->stream));
  int tcs = 0;
  CK(cudaMemcpyAsync(&tcs, h->tc_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  info->n = h->n;
  info->columns = h->c;
  info->capacity = h->cap;
  info->dtype = h->dtype;
  info->compressions = h->ncomp;
  info->stages = (int64_t)h->tape.size();
  info->discarded = h->h_small[0];
  info->last_gap = h->h_small[1];
  if (tcs || h->h_small[2] >= 3) return LR_ETIMEOUT;  // eigensolver status 3: a bounded wait gave up
  return h->h_small[2] > 0 ? LR_ENOCONV : LR_OK;
}

int lr_get_state(lr_handle h, void* out_host) {
  if (!h || !out_host) return LR_EINVAL;
  int rc = flush_state(h);
  if (rc) return rc;
  CK(cudaMemcpy2DAsync(out_host, h->c * h->esz, h->V, h->cap * h->esz, h->c * h->esz, (size_t)h->N,
                       cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LR_OK;
}

int64_t lr_device_bytes(lr_handle h) { return h ? (int64_t)h->bytes : 0; }

int lr_last_eig(lr_handle h, int* m_out, int* k_out, double* G_out, double* evals_out, double* evecs_out) {
  if (!h || !m_out || !k_out) return LR_EINVAL;
  const int m = h->last_m;
  CK(cudaMemcpyAsync(h->h_eo, h->eo, sizeof(EigOut), cudaMemcpyDeviceToHost, h->stream));
  if (m > 0) {
    if (G_out) CK(cudaMemcpyAsync(G_out, h->G, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, h->stream));
    if (evals_out) CK(cudaMemcpyAsync(evals_out, h->evals, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream));
    if (evecs_out) CK(cudaMemcpyAsync(evecs_out, h->evecs, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  *m_out = m;
  *k_out = m > 0 ? h->h_eo->k : 0;
  return LR_OK;
}

int lr_last_eig_stats(lr_handle h, int* sweeps_out, long long* cycles_out) {
  if (!h || !sweeps_out || !cycles_out) return LR_EINVAL;
  CK(cudaMemcpyAsync(h->h_eo, h->eo, sizeof(EigOut), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *sweeps_out = h->h_eo->sweeps;
  for (int i = 0; i < 6; ++i) cycles_out[i] = h->h_eo->cycles[i];
  return LR_OK;
}

int lr_set_timing(lr_handle h, int on) {
  if (!h) return LR_EINVAL;
  if (on && h->ev.empty()) {
    h->ev.resize(4096);
    for (auto& e : h->ev) CK(cudaEventCreate(&e));
  }
  timer_drain(h);
  h->timing = on != 0;
  return LR_OK;
}

int lr_kernel_times(lr_handle h, double* ms_out, int64_t* counts_out) {
  if (!h || !ms_out || !counts_out) return LR_EINVAL;
  timer_drain(h);
  for (int i = 0; i < LR_NKCLASS; ++i) {
    ms_out[i] = h->kms[i];
    counts_out[i] = h->kcnt[i];
    h->kms[i] = 0.0;
    h->kcnt[i] = 0;
  }
  return LR_OK;
}

}  // extern "C"
