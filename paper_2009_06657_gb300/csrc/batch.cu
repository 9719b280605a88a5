// Batched execution of many independent noisy circuits (uneven n, r, depth).
//
// Each circuit is lowered once on the host into a list of stages with the
// same semantics as the single-circuit runtime (Alg. 1 with one-qubit Kraus
// groups, fixed rank): an expansion stage (a gate alone, or a channel whose
// expanded column count still fits the rank) or a truncation stage (a channel
// and, folded into it, a one-qubit gate on the same qubit; Gram of the row
// pairs, eigensolve, projection on the row pairs). Stage s of every circuit
// runs in the same batched launches: one expansion launch, then the truncation
// launches (pair Gram, split sums, assembly; the eigensolves: one CTA per circuit,
// or an 8-CTA cluster for the largest Gram matrices, the two in parallel graph
// branches; for a complex64 state the FP64 refinement; projection matrix,
// projection, accounting). The Gram and the projection of a complex64 circuit
// with enough rows run on the tensor cores. Per-step task tables and block-to-task
// prefix tables are built and uploaded once; the whole schedule is captured into
// one CUDA graph, so a run is a single graph launch.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "lret.h"

using namespace lret;
using zc = std::complex<double>;

namespace {

struct Circ {
  int n = 0, r = 0, cap = 0;
  int64_t N = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;   // buffer holding the state after the whole schedule
  int c = 1;     // columns after the whole schedule
  int splits = 1;
  double* acc = nullptr;
  double2 *partials = nullptr, *S = nullptr, *G = nullptr, *evecs = nullptr, *D = nullptr;
  double* evals = nullptr;
  EigOut* eo = nullptr;
  void* eigwork = nullptr;
  void* rfwork = nullptr;  // FP64 refinement workspace (refined eigensolve)
  int64_t tc_rows = 0;     // rows per split of the tensor-core Gram (0: not eligible)
  int tc_splits = 0;
  float* B = nullptr;      // tensor-core projection operand
  double* tcs = nullptr;   // trace anchoring: [unused, s, per-block squared norms]
  int64_t gates = 0, truncs = 0;
};

struct Step {
  int e_off = 0, e_cnt = 0, e_blocks = 0, eb_off = 0;
  int t_off = 0, t_cnt = 0, gram_blocks = 0, proj_blocks = 0, gb_off = 0, pb_off = 0, max_m2 = 0, max_d = 0;
  int max_m = 0, max_k = 0;  // largest Gram size and rank of the step's truncations
  int tg_off = 0, tg_blocks = 0;  // tensor-core Gram of the step's eligible truncations
  int tp_off = 0, tp_blocks = 0, max_nk = 0;  // tensor-core projection
  int tri_off = 0, tri_cnt = 0;  // step-local indices of the one-CTA solver's tasks
  int cl_off = 0, cl_cnt = 0;    // the cluster solver's tasks (in lr_batch::cl_tasks)
};



void rot(int axis, double th, zc U[4]) {
  const zc I(0, 1);
  zc S[4];
  if (axis == 0) { S[0] = 0; S[1] = 1; S[2] = 1; S[3] = 0; }
  else if (axis == 1) { S[0] = 0; S[1] = -I; S[2] = I; S[3] = 0; }
  else { S[0] = 1; S[1] = 0; S[2] = 0; S[3] = -1; }
  const double cs = std::cos(th / 2), sn = std::sin(th / 2);
  for (int i = 0; i < 4; ++i) U[i] = ((i == 0 || i == 3) ? cs : 0.0) - I * sn * S[i];
}

void mm2(const zc* A, const zc* B, zc* C) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) C[i * 2 + j] = A[i * 2] * B[j] + A[i * 2 + 1] * B[2 + j];
}

void put(double2& d, zc v) { d = make_double2(v.real(), v.imag()); }

}  // namespace

struct lr_batch {
  int count = 0, dtype = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // created here: the legacy default stream cannot be captured
  cudaStream_t side = nullptr;  // second branch of a step's eigensolves
  cudaEvent_t fork = nullptr, join = nullptr;
  int cluster_min_m = 0;
  std::vector<ClusterTask> cl_tasks;  // step-major
  size_t esz = 0;
  std::vector<Circ> circ;
  std::vector<Step> steps;
  int eig_prec = LR_EIGP_REFINED, eig_iters = 1;
  ExpandTask* d_et = nullptr;
  TruncTask* d_tt = nullptr;
  RefineTask* d_rt = nullptr;  // one per truncation task, same order (refined eigensolve)
  int* d_status = nullptr;     // set by a tensor-core kernel whose bounded wait gave up
  bool any_tc = false;
  bool any_cluster = false;
  int* d_bs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int use_graph = 1;
  long long graph_kernels = 0;  // kernels in the captured graph
  int64_t launches = 0, gates = 0, truncs = 0, expands = 0;
  size_t bytes = 0;
};

#define BCK(call)                                                                      \
  do {                                                                                 \
    cudaError_t _e = (call);                                                           \
    if (_e != cudaSuccess) {                                                           \
      lret::set_error("%s: %s", #call, cudaGetErrorString(_e));                        \
      return LR_ECUDA;                                                                 \
    }                                                                                  \
  } while (0)

namespace {

int bmalloc(lr_batch* b, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    return LR_ENOMEM;
  }
  b->bytes += bytes;
  return LR_OK;
}

template <typename F>
cudaError_t by_dt(int dtype, F f) {
  if (dtype == LR_C64) return f(float());
  return f(double());
}

// Lowered stage of one circuit.
struct HStage {
  int type;        // 0 expansion, 1 truncation
  int G, K, q;     // group rows; Kraus count; qubit (pair bit) for truncation
  int bits[2];
  int c_in, c_out;
  zc M[4][4][4];   // expansion: M[al][a][g]; truncation: M[al][a][b] (2x2)
};

int lower(const lr_circuit& cd, std::vector<HStage>& out, int64_t* gates) {
  const int n = cd.n, r = cd.r;
  int c = 1;
  bool pend = false;
  int pnq = 0, pq[2] = {0, 0};
  zc pU[16];
  *gates = 0;
  auto emit_gate = [&]() {
    HStage st{};
    st.type = 0;
    st.G = 1 << pnq;
    st.K = 1;
    st.bits[0] = pq[0];
    st.bits[1] = pnq == 2 ? pq[1] : 0;
    st.c_in = st.c_out = c;
    for (int a = 0; a < st.G; ++a)
      for (int g = 0; g < st.G; ++g) st.M[0][a][g] = pU[a * st.G + g];
    out.push_back(st);
    pend = false;
  };
  for (int i = 0; i < cd.nops; ++i) {
    const lr_op& o = cd.ops[i];
    if (o.kind <= LR_OP_CZ) {
      if (o.q0 < 0 || o.q0 >= n) return LR_EINVAL;
      if (o.kind >= LR_OP_CNOT && (o.q1 < 0 || o.q1 >= n || o.q1 == o.q0)) return LR_EINVAL;
      if (pend) emit_gate();
      ++*gates;
      if (o.kind <= LR_OP_RZ) {
        pnq = 1;
        pq[0] = o.q0;
        rot(o.kind - LR_OP_RX, o.theta, pU);
      } else {
        pnq = 2;
        pq[0] = o.q0;
        pq[1] = o.q1;
        for (int k = 0; k < 16; ++k) pU[k] = 0;
        if (o.kind == LR_OP_CNOT) { pU[0] = pU[5] = 1; pU[11] = pU[14] = 1; }
        else { pU[0] = pU[5] = pU[10] = 1; pU[15] = -1; }
      }
      pend = true;
    } else if (o.kind <= LR_OP_BF) {
      if (o.q0 < 0 || o.q0 >= n) return LR_EINVAL;
      double kr[32];
      int K = 0;
      const int kind = o.kind == LR_OP_DEP ? LR_DEPOLARIZING : (o.kind == LR_OP_AD ? LR_AMPLITUDE_DAMPING : LR_BIT_FLIP);
      if (lr_kraus_preset(kind, o.p, kr, &K) != LR_OK) return LR_EINVAL;
      const int q = o.q0;
      if (pend && !(pnq == 1 && pq[0] == q)) emit_gate();
      zc Gm[4] = {1, 0, 0, 1};
      if (pend) for (int k = 0; k < 4; ++k) Gm[k] = pU[k];
      HStage st{};
      st.K = K;
      st.q = q;
      st.G = 2;
      st.bits[0] = q;
      for (int al = 0; al < K; ++al) {
        zc Kd[4], M[4];
        for (int k = 0; k < 4; ++k) Kd[k] = zc(kr[al * 8 + 2 * k], kr[al * 8 + 2 * k + 1]);
        mm2(Kd, Gm, M);
        for (int a = 0; a < 2; ++a)
          for (int g = 0; g < 2; ++g) st.M[al][a][g] = M[a * 2 + g];
      }
      st.c_in = c;
      if (c * K <= r) {
        st.type = 0;
        st.c_out = c * K;
      } else {
        st.type = 1;
        st.c_out = r;
      }
      c = st.c_out;
      out.push_back(st);
      pend = false;
    } else {
      return LR_EINVAL;
    }
  }
  if (pend) emit_gate();
  return LR_OK;
}

// Prob(x) *= s^2 (complex64 batches: tensor-core circuits carry a trace scale s)
__global__ void k_scale_probs(float* __restrict__ p, int64_t N, const double* __restrict__ s) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x < N) p[x] = (float)((double)p[x] * s[0] * s[0]);
}

int init_states(lr_batch* b) {
  for (auto& C : b->circ) {
    BCK(cudaMemsetAsync(C.buf[0], 0, (size_t)C.N * C.cap * b->esz, b->stream));
    if (b->dtype == LR_C64) {
      const float one[2] = {1.f, 0.f};
      BCK(cudaMemcpyAsync(C.buf[0], one, sizeof(one), cudaMemcpyHostToDevice, b->stream));
    } else {
      const double one[2] = {1.0, 0.0};
      BCK(cudaMemcpyAsync(C.buf[0], one, sizeof(one), cudaMemcpyHostToDevice, b->stream));
    }
    BCK(cudaMemsetAsync(C.acc, 0, sizeof(double) * 8, b->stream));
    if (C.tcs) {
      const double one[2] = {0.0, 1.0};
      BCK(cudaMemcpyAsync(C.tcs, one, sizeof(one), cudaMemcpyHostToDevice, b->stream));
    }
  }
  BCK(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return LR_OK;
}

// the eigensolver's arithmetic: FP64 for a complex128 state or when asked for
bool solve_fp64(const lr_batch* b) { return b->dtype == LR_C128 || b->eig_prec == LR_EIGP_FP64; }

// whether an m x m Gram matrix goes to the cluster solver
bool uses_cluster(const lr_batch* b, int m) {
  return b->cluster_min_m > 0 && m >= b->cluster_min_m && m <= eigh_cluster_max_m() && m >= 2;
}

// The step's eigensolves: the large Gram matrices on the cluster solver (main stream),
// the others on the one-CTA solver (a forked branch when both kinds are present).
template <typename T>
cudaError_t solve_step(lr_batch* b, const Step& st, const TruncTask* tt, int all_vecs) {
  const int* tri_sel = b->d_bs + st.tri_off;
  const ClusterTask* cl = b->cl_tasks.data() + st.cl_off;
  if (!st.cl_cnt) return launch_eigh_tri_batch<T>(tt, tri_sel, st.tri_cnt, all_vecs, b->stream);
  if (!st.tri_cnt) return launch_eigh_cluster_batch<T>(cl, st.cl_cnt, all_vecs, b->stream);
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
  if (e == cudaSuccess) e = launch_eigh_tri_batch<T>(tt, tri_sel, st.tri_cnt, all_vecs, b->side);
  if (e == cudaSuccess) e = launch_eigh_cluster_batch<T>(cl, st.cl_cnt, all_vecs, b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->join, b->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
  return e;
}

int enqueue(lr_batch* b) {
  const int dt = b->dtype;
  for (const Step& st : b->steps) {
    if (st.e_cnt) {
      BCK(by_dt(dt, [&](auto t) {
        return launch_expand_batch<decltype(t)>(b->d_et + st.e_off, b->d_bs + st.eb_off, st.e_blocks, st.e_cnt,
                                                b->stream);
      }));
    }
    if (st.t_cnt) {
      const TruncTask* tt = b->d_tt + st.t_off;
      if (st.tg_blocks) BCK(launch_gram_pair_tc_batch(tt, b->d_bs + st.tg_off, st.tg_blocks, st.t_cnt, b->stream));
      BCK(by_dt(dt, [&](auto t) {
        return launch_trunc_batch_gemms<decltype(t)>(tt, b->d_bs + st.gb_off, st.gram_blocks, b->d_bs + st.pb_off,
                                                     st.proj_blocks, st.t_cnt, st.max_m2, st.max_d, 0, b->stream);
      }));
      const int refine = !solve_fp64(b) && b->eig_prec == LR_EIGP_REFINED;
      BCK(solve_fp64(b) ? solve_step<double>(b, st, tt, 0) : solve_step<float>(b, st, tt, refine));
      if (!solve_fp64(b)) {
        if (refine)
          BCK(launch_eig_refine_batch(b->d_rt + st.t_off, st.t_cnt, st.max_m, st.max_k, b->eig_iters, b->stream));
      }
      BCK(by_dt(dt, [&](auto t) {
        return launch_trunc_batch_gemms<decltype(t)>(tt, b->d_bs + st.gb_off, st.gram_blocks, b->d_bs + st.pb_off,
                                                     st.proj_blocks, st.t_cnt, st.max_m2, st.max_d, 1, b->stream);
      }));
      if (st.tp_blocks)
        BCK(launch_proj_pair_tc_batch(tt, b->d_bs + st.tp_off, st.tp_blocks, st.t_cnt, st.max_nk, b->stream));
    }
  }
  return LR_OK;
}

}  // namespace

extern "C" {

int lr_batch_free(lr_batch_handle b) {
  if (!b) return LR_EINVAL;
  cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& C : b->circ) {
    for (int i = 0; i < 2; ++i) if (C.buf[i]) cudaFree(C.buf[i]);
    void* ps[] = {C.acc, C.partials, C.S, C.G, C.evecs, C.D, C.evals, C.eo, C.eigwork, C.rfwork, C.B, C.tcs};
    for (void* p : ps) if (p) cudaFree(p);
  }
  if (b->d_et) cudaFree(b->d_et);
  if (b->d_tt) cudaFree(b->d_tt);
  if (b->d_rt) cudaFree(b->d_rt);
  if (b->d_status) cudaFree(b->d_status);
  if (b->d_bs) cudaFree(b->d_bs);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  delete b;
  return LR_OK;
}

void lr_batch_opts_default(lr_batch_opts* o) {
  if (!o) return;
  o->dtype = LR_C64;
  o->eig_precision = LR_EIGP_REFINED;
  o->eig_iters = 1;
  o->rows_per_split = 0;
  o->splits = nullptr;
  o->use_graph = 1;
  o->stream = nullptr;
  o->tensor_cores = 1;
  o->cluster_min_m = 256;
}

int lr_batch_create(const lr_circuit* circuits, int count, int dtype, int rows_per_split, int use_graph,
                    void* stream, lr_batch_handle* out) {
  lr_batch_opts o;
  lr_batch_opts_default(&o);
  o.dtype = dtype;
  o.rows_per_split = rows_per_split;
  o.use_graph = use_graph;
  o.stream = stream;
  return lr_batch_create_ex(circuits, count, &o, out);
}

int lr_batch_create_ex(const lr_circuit* circuits, int count, const lr_batch_opts* opts, lr_batch_handle* out) {
  if (!out || !opts) return LR_EINVAL;
  *out = nullptr;
  const int dtype = opts->dtype, use_graph = opts->use_graph;
  int rows_per_split = opts->rows_per_split;
  void* stream = opts->stream;
  if (!circuits || count < 1 || (dtype != LR_C64 && dtype != LR_C128)) return LR_EINVAL;
  if (opts->eig_precision < LR_EIGP_REFINED || opts->eig_precision > LR_EIGP_FP64) return LR_EINVAL;
  if (opts->eig_precision == LR_EIGP_REFINED && (opts->eig_iters < 1 || opts->eig_iters > 4)) return LR_EINVAL;
  if (opts->cluster_min_m < 0) return LR_EINVAL;
  if (rows_per_split <= 0) rows_per_split = 4096;
  lr_batch* b = new lr_batch();
  b->count = count;
  b->dtype = dtype;
  b->eig_prec = dtype == LR_C128 ? LR_EIGP_FP64 : opts->eig_precision;
  b->eig_iters = opts->eig_iters;
  b->cluster_min_m = opts->cluster_min_m;
  b->stream = (cudaStream_t)stream;
  if (!b->stream && use_graph) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return LR_ECUDA;
    }
    b->own_stream = true;
  }
  b->esz = dtype == LR_C64 ? sizeof(float2) : sizeof(double2);
  b->use_graph = use_graph;
  b->circ.resize(count);
  if (bmalloc(b, (void**)&b->d_status, sizeof(int)) != LR_OK) {
    lr_batch_free(b);
    return LR_ENOMEM;
  }
  std::vector<std::vector<HStage>> stages(count);
  size_t max_stages = 0;
  int rc = LR_OK;
  for (int i = 0; i < count && !rc; ++i) {
    const lr_circuit& cd = circuits[i];
    if (cd.n < 2 || cd.n > 30 || cd.r < 1 || 4 * cd.r > 256 || cd.nops < 0 || (cd.nops > 0 && !cd.ops)) {
      rc = LR_EINVAL;
      break;
    }
    Circ& C = b->circ[i];
    C.n = cd.n;
    C.r = cd.r;
    C.cap = 4 * cd.r + ((4 * cd.r) & 1);
    C.N = 1ll << cd.n;
    rc = lower(cd, stages[i], &C.gates);
    if (rc) break;
    b->gates += C.gates;
    max_stages = std::max(max_stages, stages[i].size());
    const int64_t N2 = C.N / 2;
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, N2 / rows_per_split));
    if (opts->splits && opts->splits[i] > 0)
      splits = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)64, N2, (int64_t)opts->splits[i]}));
    C.splits = splits;
    const int m = 4 * cd.r, c2 = 2 * cd.r;
    // tensor-core Gram for a complex64 state with at least 2^12 row pairs
    // (per truncation the column counts must also suit them): splits of at least 2048
    // row pairs, at most 64 of them
    size_t part_bytes = sizeof(double2) * (size_t)splits * c2 * c2;
    if (dtype == LR_C64 && opts->tensor_cores && gram_pair_tc_supported(8, N2)) {
      int64_t rows = std::max<int64_t>(2048, (N2 + 63) / 64);
      rows = ((rows + 31) / 32) * 32;
      C.tc_rows = rows;
      C.tc_splits = (int)((N2 + rows - 1) / rows);
      part_bytes = std::max(part_bytes, sizeof(float2) * (size_t)C.tc_splits * c2 * c2);
    }
    const size_t slab = (size_t)C.N * C.cap * b->esz;
    rc = bmalloc(b, &C.buf[0], slab);
    if (!rc) rc = bmalloc(b, &C.buf[1], slab);
    if (!rc) rc = bmalloc(b, (void**)&C.acc, sizeof(double) * 8);
    if (!rc) rc = bmalloc(b, (void**)&C.partials, part_bytes);
    // (scratch of the largest supported shape, c = k = 64)
    if (!rc && C.tc_rows) rc = bmalloc(b, (void**)&C.B, proj_pair_tc_scratch_bytes(64, 64));
    if (!rc && C.tc_rows) rc = bmalloc(b, (void**)&C.tcs, sizeof(double) * (2 + proj_pair_tc_blocks(N2)));

    if (!rc) rc = bmalloc(b, (void**)&C.G, sizeof(double2) * (size_t)m * m);
    if (!rc) rc = bmalloc(b, (void**)&C.evecs, sizeof(double2) * (size_t)m * m);
    if (!rc) rc = bmalloc(b, (void**)&C.D, sizeof(double2) * (size_t)c2 * c2);
    if (!rc) rc = bmalloc(b, (void**)&C.S, sizeof(double2) * (size_t)c2 * c2);
    if (!rc) rc = bmalloc(b, (void**)&C.evals, sizeof(double) * m);
    if (!rc) rc = bmalloc(b, (void**)&C.eo, sizeof(EigOut));
    size_t ew = eigh_work_bytes(m, solve_fp64(b));
    if (uses_cluster(b, m)) ew = std::max(ew, eigh_cluster_work_bytes(solve_fp64(b)));
    if (!rc) rc = bmalloc(b, &C.eigwork, ew);
    if (!rc && !solve_fp64(b) && b->eig_prec == LR_EIGP_REFINED) rc = bmalloc(b, &C.rfwork, eig_refine_work_bytes(m));
  }
  if (rc) {
    lr_batch_free(b);
    return rc;
  }
  // step-major task tables
  std::vector<ExpandTask> et;
  std::vector<TruncTask> tt;
  std::vector<RefineTask> rt;
  std::vector<int> bs;
  b->steps.resize(max_stages);
  for (size_t s = 0; s < max_stages; ++s) {
    Step& S = b->steps[s];
    S.e_off = (int)et.size();
    S.t_off = (int)tt.size();
    std::vector<int> eblocks, gblocks, pblocks, tgblocks, tpblocks, tri_sel;
    S.cl_off = (int)b->cl_tasks.size();
    for (int i = 0; i < count; ++i) {
      if (s >= stages[i].size()) continue;
      const HStage& h = stages[i][s];
      Circ& C = b->circ[i];
      if (h.type == 0) {
        ExpandTask e{};
        e.V = C.buf[C.cur];
        e.W = C.buf[C.cur ^ 1];
        e.total = (C.N / h.G) * (int64_t)h.c_in;
        e.c = h.c_in;
        e.ld = C.cap;
        e.G = h.G;
        e.K = h.K;
        e.bits[0] = h.bits[0];
        e.bits[1] = h.bits[1];
        for (int al = 0; al < h.K; ++al)
          for (int a = 0; a < h.G; ++a)
            for (int g = 0; g < h.G; ++g) put(e.M[(al * h.G + a) * h.G + g], h.M[al][a][g]);
        et.push_back(e);
        eblocks.push_back(expand_blocks(e.total));
        ++b->expands;
      } else {
        TruncTask t{};
        t.V = C.buf[C.cur];
        t.W = C.buf[C.cur ^ 1];
        t.N2 = C.N / 2;
        t.splits = C.splits;
        t.chunk = trunc_chunk(t.N2, C.splits);
        t.c = h.c_in;
        t.ld = C.cap;
        t.K = h.K;
        t.k = h.c_out;
        t.q = h.q;
        t.tiles = trunc_tiles(h.c_in);
        t.m = h.K * h.c_in;
        for (int al = 0; al < h.K; ++al)
          for (int a = 0; a < 2; ++a)
            for (int g = 0; g < 2; ++g) put(t.M[al][a][g], h.M[al][a][g]);
        t.partials = C.partials;
        t.S = C.S;
        t.G = C.G;
        t.evals = C.evals;
        t.evecs = C.evecs;
        t.eo = C.eo;
        t.eigwork = C.eigwork;
        t.D = C.D;
        t.acc = C.acc;
        t.status = b->d_status;
        t.tc = C.tc_rows > 0 && gram_pair_tc_supported(t.c, t.N2);
        t.tcp = C.tc_rows > 0 && proj_pair_tc_supported(t.c, t.k, t.N2);
        t.tcs = C.tcs;
        t.B = C.B;
        if (t.tc) {
          t.tc_rows = C.tc_rows;
          t.splits = C.tc_splits;
          b->any_tc = true;
        }
        if (uses_cluster(b, t.m))
          b->cl_tasks.push_back(ClusterTask{C.G, C.eigwork, C.evals, C.evecs, C.eo, t.m, t.k});
        else
          tri_sel.push_back((int)tt.size() - S.t_off);
        tt.push_back(t);
        rt.push_back(RefineTask{C.G, t.m, t.k, C.evals, C.evecs, C.eo, C.rfwork});
        S.max_m = std::max(S.max_m, t.m);
        S.max_k = std::max(S.max_k, t.k);
        // tensor-core Gram and projection where they apply (the projection's output
        // anchored to the exact trace through tcs, as in the single-circuit runtime)
        gblocks.push_back(t.tc ? 0 : t.tiles * t.splits);
        pblocks.push_back(t.tcp ? 0 : trunc_proj_blocks(t.N2, t.k));
        tgblocks.push_back(t.tc ? t.splits : 0);
        tpblocks.push_back(t.tcp ? proj_pair_tc_blocks(t.N2) : 0);
        if (t.tcp) S.max_nk = std::max(S.max_nk, 16 * t.c * t.k);
        S.max_m2 = std::max({S.max_m2, t.m * t.m, 4 * t.c * t.c});
        S.max_d = std::max(S.max_d, 4 * t.c * t.k);
        ++C.truncs;
        ++b->truncs;
      }
      C.cur ^= 1;
      C.c = h.c_out;
    }
    S.e_cnt = (int)et.size() - S.e_off;
    S.t_cnt = (int)tt.size() - S.t_off;
    auto prefix = [&](const std::vector<int>& v, int* off, int* total) {
      *off = (int)bs.size();
      int acc = 0;
      for (int x : v) { bs.push_back(acc); acc += x; }
      bs.push_back(acc);
      *total = acc;
    };
    if (S.e_cnt) prefix(eblocks, &S.eb_off, &S.e_blocks);
    if (S.t_cnt) {
      prefix(gblocks, &S.gb_off, &S.gram_blocks);
      prefix(pblocks, &S.pb_off, &S.proj_blocks);
      prefix(tgblocks, &S.tg_off, &S.tg_blocks);
      prefix(tpblocks, &S.tp_off, &S.tp_blocks);
      S.tri_off = (int)bs.size();
      S.tri_cnt = (int)tri_sel.size();
      bs.insert(bs.end(), tri_sel.begin(), tri_sel.end());
      S.cl_cnt = (int)b->cl_tasks.size() - S.cl_off;
      if (S.cl_cnt) b->any_cluster = true;
    }
  }
  rc = bmalloc(b, (void**)&b->d_et, sizeof(ExpandTask) * std::max<size_t>(1, et.size()));
  if (!rc) rc = bmalloc(b, (void**)&b->d_tt, sizeof(TruncTask) * std::max<size_t>(1, tt.size()));
  if (!rc) rc = bmalloc(b, (void**)&b->d_rt, sizeof(RefineTask) * std::max<size_t>(1, rt.size()));
  if (!rc) rc = bmalloc(b, (void**)&b->d_bs, sizeof(int) * std::max<size_t>(1, bs.size()));
  if (rc) {
    lr_batch_free(b);
    return rc;
  }
  cudaError_t e = cudaSuccess;
  if (!et.empty()) e = cudaMemcpy(b->d_et, et.data(), sizeof(ExpandTask) * et.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tt.empty())
    e = cudaMemcpy(b->d_tt, tt.data(), sizeof(TruncTask) * tt.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !rt.empty())
    e = cudaMemcpy(b->d_rt, rt.data(), sizeof(RefineTask) * rt.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !bs.empty()) e = cudaMemcpy(b->d_bs, bs.data(), sizeof(int) * bs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = solve_fp64(b) ? prepare_eigh_tri_batch<double>() : prepare_eigh_tri_batch<float>();
  if (e == cudaSuccess && b->any_cluster)
    e = solve_fp64(b) ? prepare_eigh_cluster_batch<double>() : prepare_eigh_cluster_batch<float>();
  if (e == cudaSuccess && b->any_cluster) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && b->any_cluster) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess && b->any_cluster) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e == cudaSuccess && b->any_tc) e = prepare_gram_tc_batch();
  if (e == cudaSuccess && b->any_tc) e = prepare_proj_tc_batch();
  if (e != cudaSuccess) {
    lret::set_error("%s: %s", "batch setup", cudaGetErrorString(e));
    lr_batch_free(b);
    return LR_ECUDA;
  }
  rc = init_states(b);
  if (!rc && use_graph) {
    // the whole schedule becomes one graph
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const long long before = lret::launches_total();
      rc = enqueue(b);
      // captured launches run on each replay, not now
      b->graph_kernels = lret::launches_total() - before;
      b->launches = b->graph_kernels;
      lret::note_launches(-b->graph_kernels);
      cudaGraph_t g = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (!rc && e2 == cudaSuccess) {
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
      } else if (!rc) {
        e = e2;
      }
    }
    if (!rc && e != cudaSuccess) {
      lret::set_error("%s: %s", "graph capture", cudaGetErrorString(e));
      rc = LR_ECUDA;
    }
  }
  if (rc) {
    lr_batch_free(b);
    return rc;
  }
  *out = b;
  return LR_OK;
}

int lr_batch_run(lr_batch_handle b) {
  if (!b) return LR_EINVAL;
  if (b->exec) {
    BCK(cudaGraphLaunch(b->exec, b->stream));
    lret::note_launches(b->graph_kernels);
    return LR_OK;
  }
  const long long before = lret::launches_total();
  const int rc = enqueue(b);
  b->launches = lret::launches_total() - before;
  return rc;
}

int lr_batch_reset(lr_batch_handle b) {
  if (!b) return LR_EINVAL;
  return init_states(b);
}

int lr_batch_info(lr_batch_handle b, int i, lr_info* info) {
  if (!b || !info || i < 0 || i >= b->count) return LR_EINVAL;
  const Circ& C = b->circ[i];
  double acc[8];
  int st = 0;
  BCK(cudaMemcpyAsync(acc, C.acc, sizeof(acc), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  info->n = C.n;
  info->columns = C.c;
  info->capacity = C.cap;
  info->dtype = b->dtype;
  info->compressions = (int64_t)acc[3];
  info->stages = C.truncs;
  info->discarded = acc[0];
  info->last_gap = acc[1];
  if (st) {
    lret::set_error("%s: %s", "lr_batch_info", "a bounded wait of a tensor-core kernel gave up");
    return LR_ETIMEOUT;
  }
  return acc[2] > 0 ? LR_ENOCONV : LR_OK;
}

int lr_batch_probs(lr_batch_handle b, int i, void* out_dev) {
  if (!b || !out_dev || i < 0 || i >= b->count) return LR_EINVAL;
  const Circ& C = b->circ[i];
  BCK(by_dt(b->dtype, [&](auto t) {
    return launch_probs<decltype(t)>(C.buf[C.cur], C.N, C.c, C.cap, out_dev, b->stream);
  }));
  if (C.tcs) {  // the state is s V
    k_scale_probs<<<(unsigned)((C.N + 255) / 256), 256, 0, b->stream>>>((float*)out_dev, C.N, C.tcs + 1);
    lret::note_launches(1);
    BCK(cudaGetLastError());
  }
  BCK(cudaStreamSynchronize(b->stream));
  return LR_OK;
}

int lr_batch_stats(lr_batch_handle b, int64_t* gates, int64_t* truncations, int64_t* steps, int64_t* launches) {
  if (!b || !gates || !truncations || !steps || !launches) return LR_EINVAL;
  *gates = b->gates;
  *truncations = b->truncs;
  *steps = (int64_t)b->steps.size();
  *launches = b->launches;
  return LR_OK;
}

}  // extern "C"
