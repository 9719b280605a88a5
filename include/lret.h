/*
 * lret.h -- C ABI of liblret, low-rank noisy-circuit evolution on one GB300.
 *
 * Method: Chen, Farquhar, Parrish, "Low Rank Density Matrix Evolution for
 * Noisy Quantum Circuits" (arXiv:2009.06657). The density matrix is held as
 * rho = V V^dag with V a 2^n x c complex matrix (Eq. 2). A gate maps
 * V <- G V (Eq. 3); a Kraus channel maps V <- [Kt_1 V, ..., Kt_K V] (Eq. 4);
 * a compression keeps the leading eigenvectors of rho, found from the small
 * Gram matrix V^dag V (Sec. II.B and Theorem 1 of App. B); readouts are
 * Prob(x) = sum_v |V_xv|^2 (Eq. 9) and <O> = Tr(V^dag O V) (Sec. II.D).
 *
 * Conventions
 *   - Qubit q is bit q of the basis index x (little-endian).
 *   - Complex numbers are interleaved (re, im) pairs of double in every host
 *     array of this interface; matrices are row-major.
 *   - A two-qubit matrix on qubits (q0, q1) is indexed by 2*b(q0) + b(q1).
 *   - Kraus matrices carry their probability: Kt_a = sqrt(p_a) K_a (Eq. 1).
 *   - Pauli strings are (xmask, zmask) pairs: bit q of xmask set and zmask
 *     clear = X on q, zmask only = Z, both = Y. With that encoding
 *     P|x> = i^{#Y} (-1)^{popcount(x & zmask)} |x ^ xmask>.
 *
 * State and memory
 *   - A handle owns all device memory of one simulation (allocated with
 *     cudaMalloc in lr_init, released by lr_free). Work is queued on the CUDA
 *     stream given to lr_init. Host arrays passed in are copied during the
 *     call; the caller keeps ownership. Device output buffers belong to the
 *     caller.
 *   - Gates and channels are queued lazily and fused: a gate followed by a
 *     channel on one of its qubits runs as one expansion kernel.
 *   - Calls that return host values synchronise the handle's stream.
 *   - One host thread per handle.
 *
 * Errors: every call returns LR_OK (0) or a negative status. After an error
 * the handle's state is unchanged unless the status is LR_ECUDA.
 */
#ifndef LRET_H
#define LRET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LR_OK 0
#define LR_EINVAL -1     /* bad argument: qubit out of range, n > 30, ... */
#define LR_EKRAUS -2     /* || sum_a Kt_a^dag Kt_a - I ||_max > 1e-10 */
#define LR_ECAPACITY -3  /* columns would exceed the allocated capacity */
#define LR_ENOMEM -4     /* device allocation failed */
#define LR_ETIMEOUT -5   /* a bounded device-side wait gave up */
#define LR_ECUDA -6      /* a CUDA call failed */
#define LR_ESTATE -7     /* call not valid in the current state */
#define LR_ENOCONV -8    /* eigensolver reached its sweep limit */

#define LR_C64 0   /* complex64 state; FP32 arithmetic with FP64 sums */
#define LR_C128 1  /* complex128 state; FP64 throughout */

typedef struct lr_ctx* lr_handle;

/* Create a simulation of n qubits (1..30) in |0...0> (V = e_0, c = 1,
 * Algorithm 1 initial state). r is the default rank for lr_compress(r <= 0 ->
 * this r) and sets the column capacity to 4*r (a one-qubit channel with up to
 * four Kraus matrices). dtype is LR_C64 or LR_C128. stream is a cudaStream_t
 * (NULL = the legacy default stream). */
int lr_init(int n, int r, int dtype, void* stream, lr_handle* out);

/* Like lr_init with an explicit column capacity (>= r). */
int lr_init_ex(int n, int r, int dtype, int capacity, void* stream, lr_handle* out);

int lr_free(lr_handle h);

/* Return to |0...0>, clear the discarded mass, the tape and the queue. */
int lr_reset(lr_handle h);

/* Gate G on nq qubits, Eq. (3): V <- G V. U is 2^nq x 2^nq complex, row-major,
 * indexed by sum_i b(qubits[i]) 2^(nq-1-i) (the first listed qubit is the most
 * significant bit; for nq = 2 this is 2*b(q0) + b(q1)).
 * nq = 1 or 2: the gate is queued and fused with a following channel on one of
 *   its qubits. dU (nullable) is dG/dtheta for parameter param_id (>= 0 makes
 *   the gate differentiable; -1 = fixed).
 * 3 <= nq <= LR_MAX_GATE_QUBITS (and nq <= n): a dense multi-qubit unitary
 *   (Sec. II.C's k-qubit operators; the Grover iterates of Sec. III.D as one
 *   unitary). Queued work runs first, then the gate runs at once on the
 *   device in the state's precision; it must be fixed (dU = NULL,
 *   param_id = -1). Recording keeps a device copy of U for lr_backward.
 * Errors: LR_EINVAL for repeated or out-of-range qubits or non-finite entries.
 * U is not checked for unitarity. */
#define LR_MAX_GATE_QUBITS 13
int lr_apply_gate(lr_handle h, int nq, const int* qubits, const double* U,
                  const double* dU, int param_id);

/* Dense gate as lr_apply_gate with 3 <= nq <= LR_MAX_GATE_QUBITS, the matrix
 * given as a caller-owned DEVICE buffer U_dev of 2^nq x 2^nq complex numbers in
 * the state's precision (float2 pairs for LR_C64, double2 for LR_C128),
 * row-major, on the handle's device. It is read on the handle's stream and
 * must stay valid until that work has run; no copy is made (except the tape's
 * copy while recording). For gates applied many times (Grover iterates) this
 * skips the host conversion and upload. LR_EINVAL if U_dev is not device memory. */
int lr_apply_gate_device(lr_handle h, int nq, const int* qubits, const void* U_dev);

/* Diagonal gate on nq (1..n) qubits: row x of V is multiplied by
 * diag[sum_i b(qubits[i]) 2^(nq-1-i)] (Eq. 3 with a diagonal G, e.g. a phase
 * oracle). diag holds 2^nq complex entries (interleaved doubles). Queued work
 * runs first; the gate runs at once, in place. Errors as for lr_apply_gate. */
int lr_apply_diagonal(lr_handle h, int nq, const int* qubits, const double* diag);

/* Queue R_axis(theta) = exp(-i theta sigma_axis / 2) on qubit q; axis 0/1/2 =
 * X/Y/Z. The derivative is built natively. */
int lr_apply_rotation(lr_handle h, int axis, int q, double theta, int param_id);

/* Queue a one-qubit channel: K (1..4) Kraus matrices Kt_a (2x2 complex each,
 * probability folded in), Eq. (4). Completeness is checked (LR_EKRAUS).
 * Channels applied one after another with no lr_compress between them form
 * one Kraus group of M channels (Sec. II.C, Eq. 7): the columns multiply
 * (c -> c K_1 K_2 ... K_M) and the next lr_compress truncates the group at
 * once. LR_ECAPACITY if the columns would exceed the capacity (lr_init_ex). */
int lr_apply_kraus(lr_handle h, int q, int K, const double* kraus);

/* Kraus sets of the paper's channels with the probability folded in, written
 * as K x (2x2 complex) into out (room for 4 matrices, 32 doubles); *K_out
 * receives K. kind: LR_DEPOLARIZING (Sec. III.A.1: {sqrt(1-p) I, sqrt(p/3) X,
 * sqrt(p/3) Y, sqrt(p/3) Z}), LR_AMPLITUDE_DAMPING (Sec. III.A.3, p = gamma:
 * E0 = [[1,0],[0,sqrt(1-g)]], E1 = [[0,sqrt(g)],[0,0]]), LR_BIT_FLIP
 * (Sec. III.A.3: {sqrt(1-p) I, sqrt(p) X}). p must lie in [0, 1]. */
#define LR_DEPOLARIZING 0
#define LR_AMPLITUDE_DAMPING 1
#define LR_BIT_FLIP 2
int lr_kraus_preset(int kind, double p, double* out, int* K_out);

/* Run queued work, then truncate to the leading eigenvectors of V V^dag via
 * the Gram matrix (Sec. II.B, Theorem 1). r > 0 keeps min(r, columns); r <= 0
 * uses the threshold set by lr_set_eps if one is set, else the rank of
 * lr_init. discarded_out (nullable) receives the discarded eigenvalue mass of
 * this truncation (synchronises). */
int lr_compress(lr_handle h, int r, double* discarded_out);

/* Truncation path. LR_PATH_AUTO (default): a one-qubit channel followed by a
 * truncation is applied without forming V' -- the Gram of V' is assembled from
 * the 2c x 2c Gram of the row pairs [V_0 V_1] of the channel's qubit and the
 * projection V' U_r acts on those row pairs (same rho as Eq. 4 then Sec. II.B);
 * a queued one-qubit gate on the same qubit is folded in. Recording for
 * lr_backward uses the expanded form. LR_PATH_EXPAND always forms V'. */
#define LR_PATH_AUTO 0
#define LR_PATH_EXPAND 1
int lr_set_path(lr_handle h, int which);

/* Tensor cores for the FP32 state's Gram of the row pairs and projection on
 * the row pairs (tcgen05, 3xTF32 products, FP32 accumulation; Gram split
 * partials summed in FP64): on = 1 (default) where the shape allows it, 0 =
 * the SIMT kernels everywhere. The tensor core's FP32 accumulation shrinks a
 * projected state by about 2e-7 per projection; with tensor cores on, each
 * projected state is rescaled so that Tr rho = 1 - the discarded mass so far
 * (exact for LRET with complete Kraus sets), the scale folded into the next
 * truncation or applied before any other use of the state.
 * lr_get_info returns LR_ETIMEOUT if a bounded wait in a tensor-core kernel or
 * in the cluster eigensolver gave up. */
int lr_set_tensor_cores(lr_handle h, int on);

/* Threshold rule of Sec. II.B: keep the smallest k with
 * sum_{i<=k} lambda_i >= (1 - eps) * sum_i lambda_i. eps <= 0 disables it. */
int lr_set_eps(lr_handle h, double eps);

/* Per-truncation log (the rank history of Sec. II.B-C, from which the intermediate
 * rank V_I of Eq. 8 follows): capacity > 0 allocates room for that many records and
 * starts a new log (0 switches it off and frees it); lr_reset clears it. Every
 * truncation then appends, on the device, LR_TRUNC_LOG_FIELDS doubles:
 *   [0] m   columns before the truncation (the Gram matrix size)
 *   [1] k   columns kept
 *   [2] lambda_1, [3] lambda_k, [4] lambda_{k+1} (0 when nothing is dropped)
 *   [5] discarded eigenvalue mass, [6] trace of the Gram matrix,
 *   [7] (lambda_k - lambda_{k+1}) / lambda_1 (infinite when nothing is dropped).
 * Truncations skipped because nothing would be dropped (m <= r) write no record.
 * lr_get_trunc_log copies up to max_records records (row-major) into out_host and
 * the number of truncations logged (possibly above the capacity: later ones are
 * counted, not stored) into *count_out. It flushes queued work and synchronises. */
#define LR_TRUNC_LOG_FIELDS 8
int lr_set_trunc_log(lr_handle h, int capacity);
int lr_get_trunc_log(lr_handle h, double* out_host, int max_records, int64_t* count_out);

/* Eigensolver of the truncation: LR_EIG_AUTO (default: two-sided Jacobi for
 * small Gram matrices, the cluster tridiagonal solver above 32 columns (FP32
 * state) or 64 columns (FP64 state)), LR_EIG_JACOBI, LR_EIG_TRIDIAG
 * (Householder tridiagonal + bisection + inverse iteration, one thread block)
 * or LR_EIG_CLUSTER (the same on a cluster of 8 thread blocks). */
#define LR_EIG_AUTO 0
#define LR_EIG_JACOBI 1
#define LR_EIG_TRIDIAG 2
#define LR_EIG_CLUSTER 3
int lr_set_eigensolver(lr_handle h, int which);

/* Arithmetic of the truncation's eigensolve (Sec. II.B) for an LR_C64 state
 * (an LR_C128 state always solves in FP64 and ignores this setting).
 * LR_EIGP_REFINED (default): the solver runs in FP32 and returns every
 * eigenvector, then `iters` steps of an FP64 refinement of the kept ones on the
 * FP64 Gram matrix (residual G X - X diag(mu) in FP64, mu the FP64 Rayleigh
 * quotients; its components along the FP32 discarded eigenvectors divided by
 * the eigenvalue differences; first-order re-orthonormalisation of the kept
 * set), then two FP64 orthonormalisation steps of the kept set. The kept
 * eigenvalues become the FP64 Rayleigh quotients and the discarded mass
 * trace(G) minus their sum. iters: 0..4 (1 by default; values outside are
 * clamped); 0 returns the FP32 solve with every eigenvector and no refinement
 * (for inspection).
 * LR_EIGP_FP32: the FP32 solve alone (kept vectors and eigenvalues to FP32
 * accuracy). LR_EIGP_FP64: the solver itself in FP64 arithmetic. */
#define LR_EIGP_REFINED 0
#define LR_EIGP_FP32 1
#define LR_EIGP_FP64 2
int lr_set_eig_precision(lr_handle h, int mode, int iters);

/* Prob(x) = sum_v |V_xv|^2 (Eq. 9) into a caller-owned device buffer of 2^n
 * floats (LR_C64) or doubles (LR_C128). Asynchronous. */
int lr_probs(lr_handle h, void* out_dev);

/* <H> = sum_t coeff_t Tr(V^dag P_t V) (Sec. II.D) for T Pauli strings.
 * out_host receives one double. Synchronises. */
int lr_expect(lr_handle h, int T, const uint64_t* xmask, const uint64_t* zmask,
              const double* coeff, double* out_host);

/* <Z_q> for every qubit and the trace, into out_host[0..n] (n + 1 doubles,
 * the trace last). Synchronises. */
int lr_z_expect(lr_handle h, double* out_host);

/* Record the tape (gates, channels, truncation eigenvectors and eigenvalues,
 * state checkpoints) needed by lr_backward. Off by default. */
int lr_set_record(lr_handle h, int on);

/* Keep a state checkpoint every `every` recorded stages (a stage is one
 * expansion or one truncation); 0 = only the initial state. The backward pass
 * recomputes the states in between from the stored eigenvectors. */
int lr_set_checkpoint(lr_handle h, int every);

/* Gradient of <H> = sum_t coeff_t <P_t> with respect to every parameter id
 * used in the recorded circuit: adjoint pass through truncations, channels
 * and gates. grad_out_host has nparams doubles (ids >= nparams are an error).
 * Synchronises. */
int lr_backward(lr_handle h, int T, const uint64_t* xmask, const uint64_t* zmask,
                const double* coeff, int nparams, double* grad_out_host);

typedef struct lr_info {
  int n;               /* qubits */
  int columns;         /* current column count c of V (queued work flushed) */
  int capacity;        /* allocated columns */
  int dtype;
  int64_t compressions;/* truncations performed */
  int64_t stages;      /* recorded stages */
  double discarded;    /* cumulative discarded eigenvalue mass (FP64) */
  double last_gap;     /* (lambda_k - lambda_{k+1}) / lambda_1 at the last cut */
} lr_info;

/* Flush queued work and report the state. Synchronises. */
int lr_get_info(lr_handle h, lr_info* info);

/* Copy V (2^n x c, row-major, interleaved complex in the handle's precision)
 * into a caller-owned host buffer of 2^n * c complex elements. Flushes
 * queued work and synchronises. */
int lr_get_state(lr_handle h, void* out_host);

/* Diagnostics of the last eigensolve: Jacobi sweeps (0 for the tridiagonal
 * solver) and SM clock cycles spent in its phases (tridiagonal solver:
 * reduction, bisection, sort/accounting, inverse iteration, back-transform;
 * six entries, unused ones 0). Synchronises. */
int lr_last_eig_stats(lr_handle h, int* sweeps_out, long long* cycles_out);

/* The last truncation's eigenproblem, for inspection: *m_out receives the Gram
 * matrix size m (0 before the first truncation) and *k_out the kept count; G_out
 * (m x m complex, row-major), evals_out (m doubles, descending) and evecs_out
 * (m x m complex, row-major, column i = eigenvector i) receive the FP64 Gram
 * matrix the eigensolver read and its output (after any refinement; with
 * LR_EIGP_REFINED the kept columns and eigenvalues are refined, the others are
 * the FP32 solver's). Each array pointer may be NULL; host buffers of at least
 * 256 x 256 complex (evals: 256) always suffice. Synchronises. */
int lr_last_eig(lr_handle h, int* m_out, int* k_out, double* G_out, double* evals_out, double* evecs_out);

/* Upper bound on the device bytes the handle holds (for capacity planning). */
int64_t lr_device_bytes(lr_handle h);

/* Allocation-free <H> for callers that cannot allocate device memory when they
 * read out (a server that reserved all device memory for its own pool up front,
 * or a thread that must not take the device-wide synchronisation that
 * cudaMalloc/cudaFree imply). The paper has no counterpart: this is an interface variant of
 * lr_expect that computes the same sum_t coeff_t Tr(V^dag P_t V).
 *
 * V_dev: caller-owned device state, 2^n x c complex (row-major, leading
 * dimension ld >= c elements, interleaved complex64 for LR_C64 or complex128 for
 * LR_C128). xmask/zmask/coeff: T host values (Pauli encoding as above).
 * out_host: one double. stream: cudaStream_t (NULL = legacy default stream).
 *
 * Scratch (term masks and partial sums, about 2 MB) lives in one fixed device
 * array of this library, held by every GPU that loads it until the process
 * exits; the call allocates and frees nothing (the first call on a device looks
 * up that array's device address). All calls share the array, and the last call's contents
 * stay in it (every value a call reads is written by that call first): calls
 * that overlap on the GPU, from different streams or threads, race and must be
 * serialised by the caller. T > LR_STATIC_MAX_TERMS returns LR_ECAPACITY.
 * Synchronises the stream, so it is not a call to make on a stream that is
 * capturing a graph (nor on NULL while any global-mode capture is open); the
 * first call on a device, which does the one-time address lookup, belongs
 * before any stream capture the process starts. */
#define LR_STATIC_MAX_TERMS 256
int lr_expect_static(const void* V_dev, int n, int c, int ld, int dtype, int T,
                     const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                     double* out_host, void* stream);

/* ---- Batched execution of many independent circuits -------------------------
 * Not in the paper: many circuits of uneven n, r and depth advance together,
 * stage s of every circuit in the same launches, the whole schedule captured
 * in one CUDA graph. Semantics per circuit are those of the single-circuit
 * calls with a truncation to rank r after every channel (fixed rank). */
#define LR_OP_RX 0
#define LR_OP_RY 1
#define LR_OP_RZ 2
#define LR_OP_CNOT 3   /* q0 = control, q1 = target */
#define LR_OP_CZ 4
#define LR_OP_DEP 5    /* p = depolarizing probability */
#define LR_OP_AD 6     /* p = amplitude-damping gamma */
#define LR_OP_BF 7     /* p = bit-flip probability */
typedef struct lr_op {
  int kind;
  int q0, q1;
  double theta;  /* rotation angle */
  double p;      /* channel strength */
} lr_op;
typedef struct lr_circuit {
  int n;         /* qubits, 2..30 */
  int r;         /* rank, 4r <= 256 */
  int nops;
  const lr_op* ops;
} lr_circuit;
typedef struct lr_batch* lr_batch_handle;

/* Lower, allocate, upload the task tables and (use_graph != 0) capture the
 * schedule into one CUDA graph. rows_per_split sets the Gram split size
 * (<= 0: 4096). Every circuit starts in |0...0>. The eigensolve of an LR_C64
 * batch is the refined one (lr_batch_create_ex chooses otherwise). A NULL stream with
 * use_graph != 0 gets a stream of the batch's own (the legacy default stream
 * cannot be captured); the batch calls synchronise it. */
int lr_batch_create(const lr_circuit* circuits, int count, int dtype, int rows_per_split, int use_graph,
                    void* stream, lr_batch_handle* out);
/* Options of lr_batch_create_ex (lr_batch_opts_default fills the defaults).
 * dtype: LR_C64 or LR_C128. eig_precision (LR_C64 only; LR_C128 always solves in
 * FP64): LR_EIGP_REFINED (default: FP32 solve of every eigenvector, then `eig_iters`
 * steps of the FP64 refinement of the kept ones, as lr_set_eig_precision describes),
 * LR_EIGP_FP32 or LR_EIGP_FP64 (the solver in FP64 arithmetic). rows_per_split: Gram
 * split size of a circuit without its own entry in `splits` (<= 0: 4096). splits:
 * NULL or one Gram split count per circuit (0 = from rows_per_split, else clamped to
 * 1..64 and to the circuit's row pairs), for example from an autotuned table.
 * use_graph, stream: as lr_batch_create. */
typedef struct lr_batch_opts {
  int dtype;
  int eig_precision;
  int eig_iters;
  int rows_per_split;
  const int* splits;
  int use_graph;
  void* stream;
  int tensor_cores;  /* LR_C64: tcgen05 Gram and projection for truncations they suit
                        (default 1); a circuit so projected is rescaled to
                        Tr rho = 1 - discarded mass after each projection, as in
                        lr_set_tensor_cores (the scale is kept per circuit and taken
                        into its next truncation and lr_batch_probs) */
  int cluster_min_m; /* truncations whose Gram matrix has at least this many rows are
                        solved by the 8-CTA cluster eigensolver, the others by the
                        one-CTA solver, the two launches running side by side within a
                        step; 0 = every truncation on the one-CTA solver (default 256) */
} lr_batch_opts;
void lr_batch_opts_default(lr_batch_opts* o);
int lr_batch_create_ex(const lr_circuit* circuits, int count, const lr_batch_opts* opts, lr_batch_handle* out);
/* Run the whole schedule once (one graph launch). Asynchronous. */
int lr_batch_run(lr_batch_handle b);
/* Put every circuit back into |0...0> with zero discarded mass. Synchronises. */
int lr_batch_reset(lr_batch_handle b);
/* Per-circuit state after a run (columns, discarded mass, truncations). Synchronises. */
int lr_batch_info(lr_batch_handle b, int i, lr_info* info);
/* Prob(x) of circuit i into a caller-owned device buffer (float for LR_C64).
 * Synchronises the batch's stream. */
int lr_batch_probs(lr_batch_handle b, int i, void* out_dev);
/* Totals: gates, truncations, schedule steps, and kernel launches per run (those
 * captured in the graph; without a graph, those of the last lr_batch_run, 0 before). */
int lr_batch_stats(lr_batch_handle b, int64_t* gates, int64_t* truncations, int64_t* steps, int64_t* launches);
int lr_batch_free(lr_batch_handle b);

/* Kernel classes for lr_kernel_times. */
#define LR_K_EXPAND 0   /* gate + Kraus expansion (Eqs. 3-4) */
#define LR_K_GRAM 1     /* Gram matrix V'^dag V' */
#define LR_K_EIGH 2     /* Hermitian eigensolve + rank choice */
#define LR_K_PROJECT 3  /* V <- V' U_r */
#define LR_K_READOUT 4  /* Prob(x) */
#define LR_K_PAULI 5    /* Pauli expectations */
#define LR_K_SMALL 6    /* small dense products of a truncation: Gram assembly from the
                           pair Gram, pair projection coefficients, deferred-projection
                           products */
#define LR_K_EIGREFINE 7 /* FP64 refinement of the kept eigenvectors (LR_EIGP_REFINED) */
#define LR_NKCLASS 8

/* Bracket every forward kernel launch with CUDA events on the handle's stream
 * (on = 1) or stop (on = 0). Adds a small per-launch cost; for measurement. */
int lr_set_timing(lr_handle h, int on);

/* Device time (ms) and launch count per kernel class since the last call;
 * ms_out and counts_out have LR_NKCLASS entries. Synchronises and resets. */
int lr_kernel_times(lr_handle h, double* ms_out, int64_t* counts_out);

/* Measurement sampling (Sec. II.D: the counts of a computational-basis
 * measurement are drawn from Prob(x), Eq. 9, without forming rho). Shot s is the
 * smallest basis index x with CDF(x) > uniforms[s] * CDF(2^n - 1), CDF(x) the
 * running sum of Prob(x) over indices 0..x (inverse-transform sampling), clamped
 * to 2^n - 1. Prob(x) is formed as lr_probs forms it; the CDF is summed in FP64
 * in a fixed order, so equal states and draws give equal shots.
 *   shots    number of shots (>= 0)
 *   uniforms host array of `shots` draws in [0, 1), owned by the caller (the
 *            library draws no random numbers); any value outside -> LR_EINVAL
 *   out_host host array of `shots` int64 basis indices, written by the call
 * Flushes queued gates and channels, allocates its CDF buffer (2^n doubles) on
 * the first call or when more shots are asked, and synchronises. */
int lr_sample(lr_handle h, int shots, const double* uniforms, int64_t* out_host);

/* Von Neumann entropy of the normalised state (App. A): S = -sum_i mu_i log2 mu_i,
 * mu the eigenvalues of rho / Tr rho, obtained from the Gram matrix V^dag V
 * (whose nonzero eigenvalues are those of rho = V V^dag, Theorem 1) with the FP64
 * eigensolvers whatever the dtype; out_host[0] = S in bits, out_host[1] = 2^S (the
 * effective rank). More than 256 columns -> LR_ECAPACITY. Synchronises. */
int lr_entropy(lr_handle h, double* out_host);

/* Diagnostics, not in the paper: runs one kernel that waits on a shared-memory
 * mbarrier with the same bounded wait (at most `polls` polls) that the tensor-core
 * kernels and the cluster eigensolver use; `arrive` != 0 lets another thread arrive
 * first, 0 leaves the barrier unsignalled so that the wait runs out. Returns LR_OK
 * when the wait completed and LR_ETIMEOUT when it gave up (the kernel returns and the
 * context stays usable), LR_EINVAL for polls < 1. Allocates and frees one int of device
 * memory; synchronises `stream` (a cudaStream_t, NULL = the legacy default stream). */
int lr_selftest_wait(long long polls, int arrive, void* stream);

const char* lr_status_string(int status);

/* Number of GPU kernels this library has launched in this process, over all
 * handles and batches (a replay of a batch's CUDA graph adds the kernels in
 * the graph). For counting launches inside a measured region: read it before
 * and after. Never fails. */
int64_t lr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* LRET_H */
