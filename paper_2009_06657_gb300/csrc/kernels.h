// Internal launch interface between the host runtime (runtime.cu) and the
// kernels. Not part of the public C ABI (include/lret.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lret {

// Last error text of this thread (read back by lr_status_string).
void set_error(const char* fmt, const char* a, const char* b);

// A row-group operator: G = 2 (one qubit) or 4 (two qubits) rows of V are
// mixed by K matrices M[alpha] (G x G). The matrix index of a row is
// 2*b(bits[0]) + b(bits[1]) for G = 4 and b(bits[0]) for G = 2.
struct GroupOp {
  int G;
  int bits[2];
  int K;
  double2 M[4][4][4];   // M[alpha][a][g]
  double2 dM[4][4][4];  // derivative blocks for the adjoint (same layout)
  int has_grad;
};

// Result block written by the eigensolver (device memory).
// Process-wide count of kernels this library has launched (graph replays add
// the kernels of the graph); read through lr_launch_count.
void note_launches(long long n);
long long launches_total();

struct EigOut {
  int k;            // kept columns
  int sweeps;       // Jacobi sweeps used
  int status;       // 0 = converged, 1 = sweep limit
  int pad;
  double dropped;   // sum of discarded eigenvalues (clamped at 0), FP64
  double kept;      // sum of kept eigenvalues, FP64
  double gap;       // (lambda_k - lambda_{k+1}) / lambda_1, inf if nothing dropped
  double trace;     // trace of the Gram matrix (FP64 sum of its diagonal)
  long long cycles[6];  // SM clock cycles per solver phase (diagnostics)
};

// ---- expansion (Eqs. 3-4): W[x_a][alpha*c + j] = sum_g M[alpha][a][g] V[x_g][j]
template <typename T>
cudaError_t launch_expand(const void* V, void* W, int64_t N, int c, int ld, const GroupOp& op,
                          cudaStream_t s);

// ---- dense k-qubit gate (3 <= k <= 13): W[base(g) + off[a]][j] = sum_b G[a][b] V[base(g) + off[b]][j]
// pos = the k target qubits in ascending order; G is D x D row-major (D = 2^k) in the
// state's precision; off[a] = the target bits of matrix index a placed at their qubits.
// adjoint = 1 applies G^dag.
struct DenseOp {
  int k;
  int pos[32];
};
template <typename T>
cudaError_t launch_dense(const void* V, void* W, int64_t N, int c, int ld, const DenseOp& op, const void* G,
                         const uint32_t* off, int adjoint, cudaStream_t s);

// ---- diagonal k-qubit gate: W[x][j] = d[i(x)] V[x][j], i(x) = sum_t b(q[t]) 2^(k-1-t);
// conj = 1 applies conj(d). V == W allowed.
struct DiagOp {
  int k;
  int q[32];
};
template <typename T>
cudaError_t launch_diag(const void* V, void* W, int64_t N, int c, int ld, const DiagOp& op, const void* d,
                        int conj, cudaStream_t s);

// ---- adjoint of the expansion: Vbar[x_g][j] = sum_{alpha,a} conj(M[alpha][a][g]) Wbar[x_a][alpha c + j]
// and grad_partials[block] = 2 Re sum conj(Wbar) (dM V). Returns the grid size used.
template <typename T>
cudaError_t launch_expand_adj(const void* Wbar, const void* Vin, void* Vbar, int64_t N, int c, int ld,
                              const GroupOp& op, double* grad_partials, int* nblocks_out,
                              cudaStream_t s);

// ---- out = sum_t coeff_t P_t V (Pauli sum applied to the rows of V)
template <typename T>
cudaError_t launch_pauli_apply(const void* V, void* out, int64_t N, int c, int ld, int T_terms,
                               const uint64_t* xm, const uint64_t* zm, const double* coeff,
                               cudaStream_t s);

// ---- Gram: out[i][j] = sum_x conj(A[x][i]) B[x][j], FP64 result (ma x mb, row-major).
// partials: workspace of splits * ma * mb double2. hermitian => A == B, ma == mb.
// pairbit >= 0: the operand is the pair matrix Z = [V_0 V_1] (N/2 logical rows,
// 2*chalf logical columns) formed from V without copying; N is then N/2.
template <typename T>
cudaError_t launch_gram(const void* A, int lda, int ma, const void* B, int ldb, int mb, int64_t N,
                        bool hermitian, double2* partials, int splits, double2* out, cudaStream_t s,
                        int pairbit = -1, int chalf = 0);
int gram_splits(int64_t N, int ma, int mb);
// sum split partials of a Hermitian m x m Gram (upper 64-tiles computed) into out
cudaError_t launch_gram_reduce_herm(const double2* partials, int splits, int m, double2* out, cudaStream_t s);
// the same from FP32 partials (summed in FP64)
cudaError_t launch_gram_reduce_herm_f32(const float2* partials, int splits, int m, double2* out, cudaStream_t s);
// tensor-core (tcgen05, 3xTF32) pair Gram for the FP32 state; status: device int set on a wait timeout
bool gram_pair_tc_supported(int c, int64_t N2);
cudaError_t launch_gram_pair_tc(const void* V, int ld, int c, int pairbit, int64_t N2, double2* partials,
                                int max_splits, double2* out, int* status, cudaStream_t s);

// Small matrices of the structured truncation: M[al] = Kt_al G (2x2) and
// Q[al][be] = M[al]^dag M[be].
struct PairQ {
  double2 M[4][2][2];
  double2 Q[4][4][2][2];
};
// G' (K c x K c) from the pair Gram S (2c x 2c)
cudaError_t launch_assemble_gram(const double2* S, int c, int K, const PairQ& q, double2* Gp, cudaStream_t s);
// C (M x N) = op(A) B, op(A) = A (adj = 0, A is M x K) or A^dag (adj = 1, A is K x M); FP64
cudaError_t launch_zgemm_small(const double2* A, int lda, int adj, const double2* B, int ldb, double2* C, int ldc,
                               int M, int N, int K, cudaStream_t s);
// D (2c x 2k) = pair-projection matrix from the leading k eigenvectors U (m x m)
cudaError_t launch_build_proj(const double2* U, int c, int K, int k, const PairQ& q, double2* D, cudaStream_t s);

// ---- batched structured truncation: one task per circuit ------------------------
struct TruncTask {
  const void* V;      // state (N x ld), pairs on bit q
  void* W;            // output slab
  int64_t N2;         // number of row pairs (N / 2)
  int64_t chunk;      // Gram rows per split
  int c, ld, K, k, q, splits, tiles, m;
  double2 M[4][2][2]; // Kt_a G
  double2* partials;  // splits x (2c)^2
  double2* S;         // (2c)^2: the partials summed over splits
  double2* G;         // m x m Gram of the implicit V'
  double* evals;
  double2* evecs;
  EigOut* eo;
  void* eigwork;
  double2* D;         // 2c x 2k
  double* acc;        // per-circuit accounting [discarded, gap, status, truncations]
  // tensor-core Gram (complex64 state, shapes the tcgen05 kernel takes): FP32 partials
  // (splits of tc_rows row pairs, the upper triangle by 64-row blocks of the 2c x 2c
  // result) into `partials`
  int tc;
  int64_t tc_rows;
  int* status;        // set when a bounded wait of a tcgen05 kernel gave up
  // tensor-core projection (tcp != 0) with the trace anchoring of the single-circuit
  // runtime: B the pre-split operand; tcs (per circuit, or null) = [unused, s, per-block
  // squared norms of the last tensor-core projection]: the circuit's state is s V, s
  // folded into the next truncation's Gram (s^2) and projection matrix (s)
  int tcp;
  float* B;
  double* tcs;
};
// phase 0: pair Gram, split sums, assembly of G'; phase 1: projection matrix, pair projection,
// accounting. max_m2: the largest m^2 or (2c)^2 of the tasks.
template <typename T>
cudaError_t launch_trunc_batch_gemms(const TruncTask* tasks, const int* gram_bstart, int gram_blocks,
                                     const int* proj_bstart, int proj_blocks, int ntasks, int max_m2,
                                     int max_d, int phase, cudaStream_t s);
int trunc_tiles(int c);
// Batched tcgen05 Gram of the tasks with tc != 0: blocks map to tasks through a prefix
// table (one block per split). prepare_gram_tc_batch() sets the kernel's shared-memory
// limit (not a stream operation: call it before any graph capture).
cudaError_t prepare_gram_tc_batch();
cudaError_t launch_gram_pair_tc_batch(const TruncTask* tasks, const int* bstart, int nblocks, int ntasks,
                                      cudaStream_t s);
// Batched tcgen05 projection of the tasks with tcp != 0 (one block per 256 pair rows,
// blocks mapped to tasks through a prefix table), then each such task's new scale
// s = sqrt((1 - discarded mass so far) / |V|^2) into tcs[1]. max_nk: the largest 16 c k.
cudaError_t prepare_proj_tc_batch();
cudaError_t launch_proj_pair_tc_batch(const TruncTask* tasks, const int* bstart, int nblocks, int ntasks,
                                      int max_nk, cudaStream_t s);
int64_t trunc_chunk(int64_t N2, int splits);
int trunc_proj_blocks(int64_t N2, int k);
// T = the solver's arithmetic (float or double, independent of the state's type);
// all_vecs != 0 returns every eigenvector (for a refinement that follows); one block per
// task tasks[sel[i]], i < nsel
template <typename T>
cudaError_t launch_eigh_tri_batch(const TruncTask* tasks, const int* sel, int nsel, int all_vecs, cudaStream_t s);
template <typename T>
cudaError_t prepare_eigh_tri_batch();

struct ExpandTask {
  const void* V;
  void* W;
  int64_t total;  // groups x c
  int c, ld, G, K;
  int bits[2];
  double2 M[16];  // M[(al * G + a) * G + g]
};
template <typename T>
cudaError_t launch_expand_batch(const ExpandTask* tasks, const int* bstart, int nblocks, int ntasks,
                                cudaStream_t s);
int expand_blocks(int64_t total);

// tensor-core (tcgen05, 3xTF32) pair projection for the FP32 state: W (pairs) = V (pairs) x D,
// D: 2c x 2k complex128 (device); Bscratch: proj_pair_tc_scratch_bytes(c, k) bytes
bool proj_pair_tc_supported(int c, int k, int64_t N2);
int proj_pair_tc_blocks(int64_t N2);  // blocks of one projection launch
size_t proj_pair_tc_scratch_bytes(int c, int k);
// ssq (nullable, device): ssq[b] receives the squared Frobenius norm of what block b of
// the projection wrote (ceil(N2 / 256) blocks).
cudaError_t launch_proj_pair_tc(const void* V, int ld, int c, int k, int pairbit, int64_t N2, const double2* D,
                                float* Bscratch, void* W, int* status, double* ssq, cudaStream_t s);

// ---- Y[x][j] = sum_i A1[x][i] M1[i][j] + sum_i A2[x][i] M2[i][j]  (j < p)
// M1, M2: complex128 device matrices with leading dimensions ldm1, ldm2. A2 may be null.
// pairbit >= 0: A1 and Y are read/written as pair matrices (A1: 2*chalf logical
// columns, Y: p = 2*phalf), N is the number of pairs; A2 must be null.
template <typename T>
cudaError_t launch_rowmat(const void* A1, int lda1, int k1, const double2* M1, int ldm1,
                          const void* A2, int lda2, int k2, const double2* M2, int ldm2,
                          void* Y, int ldy, int p, int64_t N, cudaStream_t s, int pairbit = -1,
                          int chalf = 0, int phalf = 0);

// ---- Hermitian eigensolver (Jacobi, arithmetic in T): evals descending, evecs
// columns in the same order (m x m complex128, row-major), rank choice and FP64
// accounting into *out. r > 0: k = min(r, m); else threshold eps.
template <typename T>
cudaError_t launch_eigh(const double2* G, int m, void* work, double* evals, double2* evecs,
                        EigOut* out, int r, double eps, cudaStream_t s);
size_t eigh_work_bytes(int m, bool fp64);

// ---- Hermitian eigensolver, Householder tridiagonal + bisection + inverse
// iteration (arithmetic in T). Same outputs as launch_eigh; all_vecs = 0 only
// fills the kept columns of evecs.
template <typename T>
cudaError_t launch_eigh_tri(const double2* G, int m, void* work, double* evals, double2* evecs, EigOut* out,
                            int r, double eps, int all_vecs, cudaStream_t s);

// ---- the same eigensolver on a cluster of 8 CTAs (distributed shared memory);
// work: eigh_cluster_work_bytes(fp64) bytes
template <typename T>
cudaError_t launch_eigh_cluster(const double2* G, int m, void* work, double* evals, double2* evecs, EigOut* out,
                                int r, double eps, int all_vecs, cudaStream_t s);
size_t eigh_cluster_work_bytes(bool fp64);
int eigh_cluster_max_m();
// Batched cluster solve: one 8-CTA cluster per task (work: eigh_cluster_work_bytes;
// r = the kept count; the task list is copied into the launch's parameters,
// CL_BATCH_MAX tasks per launch). prepare_eigh_cluster_batch<T>() sets the
// shared-memory limit (not a stream operation: call it before any graph capture).
struct ClusterTask {
  const double2* G;
  void* work;
  double* evals;
  double2* evecs;
  EigOut* out;
  int m, r;
};
constexpr int CL_BATCH_MAX = 64;
template <typename T>
cudaError_t prepare_eigh_cluster_batch();
template <typename T>
cudaError_t launch_eigh_cluster_batch(const ClusterTask* tasks, int n, int all_vecs, cudaStream_t s);

// ---- FP64 refinement of the kept eigenvectors after an FP32 solve that returned
// all m eigenvectors (evecs m x m, columns descending; evals m): `iters` steps on
// the FP64 Gram matrix G, in place on the kept columns (k = eo->k <= kmax), kept
// eigenvalues and the accounting in *eo rewritten in FP64. work: eig_refine_work_bytes(m).
cudaError_t launch_eig_refine(const double2* G, int m, double* evals, double2* evecs, EigOut* eo, int kmax,
                              int iters, void* work, cudaStream_t s);
size_t eig_refine_work_bytes(int m);
// The same for many truncations in the same launches (one task each; the grids are
// sized for the largest m_max and kmax_max of the tasks).
struct RefineTask {
  const double2* G;
  int m, kmax;
  double* evals;
  double2* evecs;
  EigOut* eo;
  void* work;  // eig_refine_work_bytes(m)
};
cudaError_t launch_eig_refine_batch(const RefineTask* tasks, int ntasks, int m_max, int kmax_max, int iters,
                                    cudaStream_t s);

// ---- adjoint of a truncation: builds Mcat ((k+m) x m complex128) =
// [U_r^dag ; B + B^dag] with B = U_d (F o (U_d^dag C)) U_r^dag, F_ji = 1/(lam_i - lam_j).
cudaError_t launch_trunc_adj_small(const double2* C, const double2* U, const double* lam, int m,
                                   int k, double2* FA, double2* T1, double2* Mcat, cudaStream_t s);

// ---- measurement sampling (Sec. II.D): FP64 CDF of Prob(x) (N doubles in cdf,
// block sums in bsum[ceil(N / SC_ROWS)], offsets and the total in
// boff[ceil(N / SC_ROWS) + 1]) and one inverse-CDF search per shot
constexpr int SC_ROWS = 1024;
template <typename T>
cudaError_t launch_sample(const void* V, int64_t N, int c, int ld, double* cdf, double* bsum, double* boff,
                          const double* u, int shots, int64_t* out, cudaStream_t s);
// ---- von Neumann entropy (App. A) of m eigenvalues: out[0] = S (bits), out[1] = 2^S
cudaError_t launch_entropy(const double* lam, int m, double* out, cudaStream_t s);

// ---- readouts (grids never exceed kReadoutMaxBlocks blocks)
constexpr int kReadoutMaxBlocks = 1024;
template <typename T>
cudaError_t launch_probs(const void* V, int64_t N, int c, int ld, void* out, cudaStream_t s);
// out[0..n-1] = <Z_q>, out[n] = trace; partials: workspace of (n+1) * 1024 doubles
template <typename T>
cudaError_t launch_zexp(const void* V, int64_t N, int c, int ld, int n, double* partials,
                        double* out, cudaStream_t s);
// out[t] = Re Tr(V^dag P_t V); partials: workspace of T * 1024 doubles
template <typename T>
cudaError_t launch_pauli_expect(const void* V, int64_t N, int c, int ld, int T_terms,
                                const uint64_t* xm, const uint64_t* zm, double* partials,
                                double* out, cudaStream_t s);

// out[0] = sum of in[0..count-1] in index order (deterministic), optionally scaled/accumulated.
cudaError_t launch_sum(const double* in, int count, double* out, int accumulate, cudaStream_t s);

}  // namespace lret
