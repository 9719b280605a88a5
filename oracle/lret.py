"""CPU oracle for low-rank noisy-circuit evolution (LRET), arXiv:2009.06657.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The product path (the
CUDA library and its Python binding) never calls it and shares no code with it.

Plain NumPy in complex128 / float64. Every routine follows the paper's
definitions directly, without blocking or fusion:

* ``FDMState``  -- full density-matrix evolution, Eq. (1) (Sec. II.A):
  rho <- sum_a p_a K_a rho K_a^dag, gates rho <- G rho G^dag.
* ``SVState``   -- noiseless statevector, used for the zero-noise pin.
* ``LRETState`` -- Algorithm 1 (Sec. II.D) with Kraus groups of M one-qubit
  channels (Sec. II.C, Eq. 7; M = 1 truncates after every channel):
  L <- G L (Eq. 3), G a dense k-qubit or diagonal unitary as well;
  L <- [sqrt(p_1) K_1 L, ...] (Eq. 4);
  eigenvalue truncation through the small Gram matrix L^dag L (Sec. II.B,
  Theorem 1 of App. B); readouts Prob(x) (Eq. 9) and Tr(L^dag O L) (Sec. II.D),
  the von Neumann entropy of App. A from the spectrum of L^dag L.
* ``sample_inverse_cdf`` -- measurement counts drawn from Prob(x) (Sec. II.D)
  with caller-supplied uniforms.

Conventions (the paper fixes none of them):

* Qubit q is bit q of the basis index x (little-endian).
* A two-qubit matrix acting on qubits (q0, q1) is indexed by 2*b(q0) + b(q1),
  b(q) being the bit of qubit q. CNOT(q0 -> q1) flips q1 when q0 is 1.
* Rotations: R_s(theta) = exp(-i theta s / 2) for s in {X, Y, Z}.
* Kraus matrices are passed with the probability folded in: Kt_a = sqrt(p_a) K_a.
  Depolarizing (Sec. III.A.1): {sqrt(1-p) I, sqrt(p/3) X, sqrt(p/3) Y, sqrt(p/3) Z}.
  Amplitude damping (Sec. III.A.3): E0 = [[1,0],[0,sqrt(1-g)]], E1 = [[0,sqrt(g)],[0,0]].
  Bit flip (Sec. III.A.3): {sqrt(1-p) I, sqrt(p) X}.
* A k-qubit matrix on qubits (q_0, ..., q_{k-1}) is indexed by
  sum_i b(q_i) 2^(k-1-i): the first listed qubit is the most significant bit.
  A diagonal gate lists its 2^k diagonal entries in the same order.
* Kraus groups (Sec. II.C): a truncation follows every M-th channel of the
  circuit, and the last channels of a circuit get one of their own.
* Truncation keeps k = min(r, m) columns for a fixed rank r, or, for a
  threshold eps, the smallest k whose eigenvalue sum reaches (1 - eps) of the
  current trace (the crossing eigenvalue is kept). No renormalisation, so
  Tr rho = 1 - (cumulative discarded eigenvalue mass).
"""
from __future__ import annotations

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": I2, "X": SX, "Y": SY, "Z": SZ}


# --------------------------------------------------------------------------
# Gates and channels
# --------------------------------------------------------------------------

def rotation(axis, theta):
    """R_axis(theta) = exp(-i theta sigma / 2) = cos(theta/2) I - i sin(theta/2) sigma."""
    s = PAULI[axis.upper()]
    return np.cos(theta / 2.0) * I2 - 1j * np.sin(theta / 2.0) * s


def rotation_derivative(axis, theta):
    """d/dtheta of rotation(axis, theta) = -i/2 sigma R(theta)."""
    s = PAULI[axis.upper()]
    return -0.5j * s @ rotation(axis, theta)


def cnot():
    """CNOT in the (2*b(control) + b(target)) basis."""
    U = np.zeros((4, 4), dtype=np.complex128)
    U[0, 0] = U[1, 1] = 1.0
    U[2, 3] = U[3, 2] = 1.0
    return U


def cz():
    return np.diag([1.0, 1.0, 1.0, -1.0]).astype(np.complex128)


def depolarizing(p):
    """Kraus set of (1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z), Sec. III.A.1."""
    return [np.sqrt(1.0 - p) * I2, np.sqrt(p / 3.0) * SX,
            np.sqrt(p / 3.0) * SY, np.sqrt(p / 3.0) * SZ]


def amplitude_damping(g):
    """E0, E1 of the amplitude-damping channel, Sec. III.A.3 (p -> gamma)."""
    E0 = np.array([[1.0, 0.0], [0.0, np.sqrt(1.0 - g)]], dtype=np.complex128)
    E1 = np.array([[0.0, np.sqrt(g)], [0.0, 0.0]], dtype=np.complex128)
    return [E0, E1]


def bit_flip(p):
    """(1-p) rho + p X rho X, Sec. III.A.3."""
    return [np.sqrt(1.0 - p) * I2, np.sqrt(p) * SX]


def channel_kraus(op):
    if op["op"] == "dep":
        return depolarizing(op["p"])
    if op["op"] == "ad":
        return amplitude_damping(op["gamma"])
    if op["op"] == "bf":
        return bit_flip(op["p"])
    raise ValueError(op)


def swap():
    """Exchanges the two qubits: |b0 b1> -> |b1 b0> in the basis 2 b(q0) + b(q1)."""
    M = np.zeros((4, 4), dtype=np.complex128)
    for b0 in range(2):
        for b1 in range(2):
            M[2 * b1 + b0, 2 * b0 + b1] = 1.0
    return M


# fixed one-qubit gates of the randomized-benchmarking set (Sec. III, random circuits)
FIXED_1Q = {
    "x": SX,
    "y": SY,
    "z": SZ,
    "s": np.diag([1.0, 1.0j]).astype(np.complex128),
    "t": np.diag([1.0, np.exp(0.25j * np.pi)]).astype(np.complex128),
    "h": np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0),
}


def gate_matrix(op):
    """(qubits, matrix) for a gate op of the shared op-list format."""
    name = op["op"]
    if name in ("rx", "ry", "rz"):
        return [op["q"]], rotation(name[1], op["theta"])
    if name in FIXED_1Q:
        return [op["q"]], FIXED_1Q[name]
    if name == "cnot":
        return list(op["q"]), cnot()
    if name == "cz":
        return list(op["q"]), cz()
    if name == "swap":
        return list(op["q"]), swap()
    if name == "unitary":
        return list(op["q"]), np.asarray(op["U"], dtype=np.complex128)
    if name == "diag":
        return list(op["q"]), np.diag(np.asarray(op["d"], dtype=np.complex128))
    raise ValueError(op)


def is_gate(op):
    return op["op"] in ("rx", "ry", "rz", "cnot", "cz", "swap", "unitary", "diag") or op["op"] in FIXED_1Q


def is_channel(op):
    return op["op"] in ("dep", "ad", "bf")


# --------------------------------------------------------------------------
# Applying a k-qubit matrix to the row index of a (2^n x c) array
# --------------------------------------------------------------------------

def apply_rows(n, A, qubits, M):
    """Return (M on `qubits`) @ A for A of shape (2^n, c).

    Rows are viewed as an n-way tensor; qubit q is tensor axis n-1-q because
    the basis index is little-endian. M is indexed by the bits of `qubits`
    in the given order, the first qubit being the most significant.
    """
    k = len(qubits)
    c = A.shape[1]
    T = A.reshape((2,) * n + (c,))
    axes = [n - 1 - q for q in qubits]
    Mt = M.reshape((2,) * (2 * k))
    # contract M's input indices with the selected axes of T
    out = np.tensordot(Mt, T, axes=(list(range(k, 2 * k)), axes))
    # tensordot puts M's output indices first; move them back into place
    out = np.moveaxis(out, list(range(k)), axes)
    return out.reshape(2 ** n, c)


def diag_index(n, qubits):
    """For every basis index x, sum_i b(q_i) 2^(k-1-i) (first qubit most significant)."""
    x = np.arange(2 ** n, dtype=np.int64)
    k = len(qubits)
    idx = np.zeros(2 ** n, dtype=np.int64)
    for i, q in enumerate(qubits):
        idx |= ((x >> q) & 1) << (k - 1 - i)
    return idx


def apply_diag_rows(n, A, qubits, d):
    """Return (diag(d) on `qubits`) @ A: row x scaled by d[diag_index(x)]."""
    d = np.asarray(d, dtype=np.complex128)
    return d[diag_index(n, qubits)][:, None] * A


def pauli_string_matrix_apply(n, A, term):
    """Apply the Pauli string `term` = [(q, 'X'|'Y'|'Z'), ...] to the rows of A."""
    out = A
    for q, s in term:
        out = apply_rows(n, out, [q], PAULI[s])
    return out


def pauli_sum_apply(n, A, terms):
    """(sum_t c_t P_t) A for terms = [(c_t, string_t), ...]."""
    out = np.zeros_like(A)
    for c, term in terms:
        out += c * pauli_string_matrix_apply(n, A, term)
    return out


# --------------------------------------------------------------------------
# Full density matrix (Eq. 1) and statevector
# --------------------------------------------------------------------------

class FDMState:
    """Exact density-matrix evolution, Eq. (1)."""

    def __init__(self, n):
        self.n = n
        self.rho = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
        self.rho[0, 0] = 1.0

    def _conj_apply(self, qubits, M):
        # rho <- M rho M^dag: apply M to the rows, then to the rows of the adjoint
        X = apply_rows(self.n, self.rho, qubits, M)
        return apply_rows(self.n, X.conj().T, qubits, M).conj().T

    def gate(self, qubits, U):
        self.rho = self._conj_apply(qubits, U)

    def diag(self, qubits, d):
        # rho <- D rho D^dag: rho[x, y] d[x] conj(d[y])
        dx = np.asarray(d, dtype=np.complex128)[diag_index(self.n, qubits)]
        self.rho = dx[:, None] * self.rho * dx.conj()[None, :]

    def channel(self, q, kraus):
        acc = np.zeros_like(self.rho)
        for K in kraus:
            acc += self._conj_apply([q], K)
        self.rho = acc

    def probs(self):
        return np.real(np.diag(self.rho)).copy()

    def expect(self, terms):
        # Tr(rho H) with H applied column-block by column-block
        Hrho = pauli_sum_apply(self.n, self.rho, terms)
        return float(np.real(np.trace(Hrho)))


class SVState:
    """Noiseless statevector |psi>, used for the zero-noise pin."""

    def __init__(self, n):
        self.n = n
        self.psi = np.zeros((2 ** n, 1), dtype=np.complex128)
        self.psi[0, 0] = 1.0

    def gate(self, qubits, U):
        self.psi = apply_rows(self.n, self.psi, qubits, U)

    def diag(self, qubits, d):
        self.psi = apply_diag_rows(self.n, self.psi, qubits, d)

    def probs(self):
        return np.abs(self.psi[:, 0]) ** 2

    def expect(self, terms):
        Hpsi = pauli_sum_apply(self.n, self.psi, terms)
        return float(np.real(np.vdot(self.psi[:, 0], Hpsi[:, 0])))


# --------------------------------------------------------------------------
# Low-rank evolution with eigenvalue truncation (Algorithm 1)
# --------------------------------------------------------------------------

def gram_eigh(G):
    """Eigenpairs of the Hermitian Gram matrix of a truncation (Sec. II.B), FP64,
    eigenvalues descending with the eigenvectors (columns) in the same order."""
    G = 0.5 * (G + G.conj().T)
    lam, U = np.linalg.eigh(G)
    return lam[::-1].copy(), U[:, ::-1].copy()


def choose_rank(lam, r=None, eps=None):
    """Number k of leading eigenvalues kept (Sec. II.B).

    lam: eigenvalues sorted descending. Fixed rank: k = min(r, m). Threshold:
    smallest k with sum(lam[:k]) >= (1 - eps) * sum(lam), at least 1.
    """
    m = len(lam)
    if r is not None and r > 0:
        return min(int(r), m)
    if eps is None:
        raise ValueError("need r or eps")
    lp = np.clip(lam, 0.0, None)
    total = lp.sum()
    csum = np.cumsum(lp)
    k = int(np.searchsorted(csum, (1.0 - eps) * total, side="left")) + 1
    return max(1, min(k, m))


class LRETState:
    """L (2^n x c) with rho = L L^dag, Eq. (2). Starts from |0...0>."""

    def __init__(self, n):
        self.n = n
        self.L = np.zeros((2 ** n, 1), dtype=np.complex128)
        self.L[0, 0] = 1.0
        self.discarded = 0.0
        self.log = []  # one dict per truncation

    # Eq. (3): L <- G L
    def gate(self, qubits, U):
        self.L = apply_rows(self.n, self.L, qubits, U)

    # Eq. (3) with a diagonal G
    def diag(self, qubits, d):
        self.L = apply_diag_rows(self.n, self.L, qubits, d)

    # Eq. (4): L <- [sqrt(p_1) K_1 L, ..., sqrt(p_A) K_A L]  (alpha-major blocks)
    def channel(self, q, kraus):
        self.L = np.hstack([apply_rows(self.n, self.L, [q], K) for K in kraus])

    # Sec. II.B with Theorem 1: eigenpairs of L L^dag from the Gram L^dag L
    def compress(self, r=None, eps=None):
        L = self.L
        G = L.conj().T @ L
        lam, U = gram_eigh(G)
        k = choose_rank(lam, r=r, eps=eps)
        dropped = float(np.clip(lam[k:], 0.0, None).sum())
        self.L = L @ U[:, :k]
        self.discarded += dropped
        lam1 = max(float(lam[0]), 1e-300)
        gap = float((lam[k - 1] - lam[k]) / lam1) if k < len(lam) else np.inf
        self.log.append({"m": len(lam), "k": k, "dropped": dropped, "gap": gap,
                         "lam": lam.copy()})
        return dropped

    def rho(self):
        return self.L @ self.L.conj().T

    # Eq. (9): Prob(x) = sum_v |L_xv|^2
    def probs(self):
        return np.sum(np.abs(self.L) ** 2, axis=1)

    # Sec. II.D: <O> = Tr(L^dag O L)
    def expect(self, terms):
        HL = pauli_sum_apply(self.n, self.L, terms)
        return float(np.real(np.trace(self.L.conj().T @ HL)))

    def z_expect(self):
        p = self.probs()
        x = np.arange(2 ** self.n)
        return np.array([np.sum(p * (1.0 - 2.0 * ((x >> q) & 1))) for q in range(self.n)])

    def trace(self):
        return float(np.real(np.sum(np.abs(self.L) ** 2)))

    # App. A: S = -Tr(rho log2 rho) of the normalised state. The nonzero
    # eigenvalues of rho = L L^dag are those of L^dag L (Theorem 1).
    def entropy(self):
        G = self.L.conj().T @ self.L
        return entropy_from_eigenvalues(np.linalg.eigvalsh(0.5 * (G + G.conj().T)))


def entropy_from_eigenvalues(lam):
    """S = -sum_i mu_i log2 mu_i with mu = max(lam, 0) / sum(max(lam, 0)) (App. A:
    von Neumann entropy in bits of the normalised state; zero terms omitted).
    The effective rank of App. A is then 2**S."""
    lp = np.clip(np.asarray(lam, dtype=np.float64), 0.0, None)
    mu = lp / lp.sum()
    mu = mu[mu > 0]
    return float(-np.sum(mu * np.log2(mu)))


def entropy_dense(rho):
    """The same entropy from the full density matrix (2^n x 2^n), for pins."""
    return entropy_from_eigenvalues(np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)))


def sample_inverse_cdf(probs, uniforms):
    """Measurement sampling from Prob(x) (Sec. II.D): shot s is the smallest x
    with CDF(x) > u_s * CDF(last), CDF the running sum of Prob(x) in index order,
    clamped to the last index. ``uniforms`` are the caller's draws in [0, 1)."""
    cdf = np.cumsum(np.asarray(probs, dtype=np.float64))
    t = np.asarray(uniforms, dtype=np.float64) * cdf[-1]
    idx = np.searchsorted(cdf, t, side="right")
    return np.minimum(idx, len(cdf) - 1).astype(np.int64)


# --------------------------------------------------------------------------
# Circuit runners over the shared op-list format
# --------------------------------------------------------------------------

def with_thetas(ops, thetas):
    """Copy of ops with parameter pid set to thetas[pid]."""
    out = []
    for o in ops:
        o2 = dict(o)
        if o.get("pid", -1) >= 0:
            o2["theta"] = float(thetas[o["pid"]])
        out.append(o2)
    return out


def _apply_gate_op(st, o):
    if o["op"] == "diag":
        st.diag(list(o["q"]), o["d"])
    else:
        qs, U = gate_matrix(o)
        st.gate(qs, U)


def run_lret(n, ops, r=None, eps=None, compress=True, group=1):
    """Algorithm 1: gates (Eq. 3), channels concatenated (Eq. 4), and a
    truncation after every `group`-th channel (Kraus groups, Sec. II.C) plus one
    after the circuit's last channels if they have not been truncated yet."""
    st = LRETState(n)
    pending = 0
    for o in ops:
        if is_gate(o):
            _apply_gate_op(st, o)
        elif is_channel(o):
            st.channel(o["q"], channel_kraus(o))
            pending += 1
            if compress and pending == group:
                st.compress(r=r, eps=eps)
                pending = 0
        else:
            raise ValueError(o)
    if compress and pending:
        st.compress(r=r, eps=eps)
    return st


def run_fdm(n, ops):
    st = FDMState(n)
    for o in ops:
        if is_gate(o):
            _apply_gate_op(st, o)
        elif is_channel(o):
            st.channel(o["q"], channel_kraus(o))
    return st


def run_sv(n, ops):
    st = SVState(n)
    for o in ops:
        if is_gate(o):
            _apply_gate_op(st, o)
    return st


# --------------------------------------------------------------------------
# Metrics (Sec. III, Eq. 10) and gradients
# --------------------------------------------------------------------------

def variational_distance(pa, pb):
    """T(rho_A, rho_B) = sum_i |rho_A,ii - rho_B,ii| (Sec. III, no factor 1/2)."""
    return float(np.sum(np.abs(np.asarray(pa) - np.asarray(pb))))


def distortion(p_lret, p_exact, p_noiseless):
    """Eq. (10): T(rho_LRET, rho_exact) / T(rho_exact, rho_noiseless)."""
    return variational_distance(p_lret, p_exact) / variational_distance(p_exact, p_noiseless)


def trace_distance_lowrank(LA, LB):
    """0.5 * || LA LA^dag - LB LB^dag ||_1 without forming 2^n x 2^n matrices.

    With the thin QR factorisation [LA LB] = Q [RA RB], the difference is
    Q (RA RA^dag - RB RB^dag) Q^dag with Q orthonormal, so its nonzero eigenvalues
    are those of the small Hermitian matrix RA RA^dag - RB RB^dag. Both steps are
    backward stable, so nearly equal states keep an absolute error at the level of
    the unit roundoff (the eigenvalues of the non-Hermitian S X^dag X, S = diag(I, -I),
    are equal in exact arithmetic but nearly defective when LA ~ LB, which leaves an
    error of order sqrt(unit roundoff)).
    """
    ra = LA.shape[1]
    _, R = np.linalg.qr(np.hstack([LA, LB]), mode="reduced")
    RA, RB = R[:, :ra], R[:, ra:]
    D = RA @ RA.conj().T - RB @ RB.conj().T
    return 0.5 * float(np.sum(np.abs(np.linalg.eigvalsh(0.5 * (D + D.conj().T)))))


def expect_lret(n, ops, thetas, terms, r=None, eps=None):
    return run_lret(n, with_thetas(ops, thetas), r=r, eps=eps).expect(terms)


def expect_fdm(n, ops, thetas, terms):
    return run_fdm(n, with_thetas(ops, thetas)).expect(terms)


def gradient_fd_lret(n, ops, thetas, terms, r=None, eps=None, h=1e-4, pids=None):
    """Central finite differences of <H> through Algorithm 1 (FP64)."""
    thetas = np.asarray(thetas, dtype=np.float64)
    pids = range(len(thetas)) if pids is None else pids
    g = np.zeros(len(thetas))
    for i in pids:
        tp = thetas.copy(); tp[i] += h
        tm = thetas.copy(); tm[i] -= h
        g[i] = (expect_lret(n, ops, tp, terms, r, eps) - expect_lret(n, ops, tm, terms, r, eps)) / (2 * h)
    return g


def gradient_param_shift_fdm(n, ops, thetas, terms, pids=None):
    """Parameter-shift rule on exact evolution: (f(t + pi/2) - f(t - pi/2)) / 2.

    Exact for gates exp(-i theta P / 2) with parameter-independent channels.
    """
    thetas = np.asarray(thetas, dtype=np.float64)
    pids = range(len(thetas)) if pids is None else pids
    g = np.zeros(len(thetas))
    for i in pids:
        tp = thetas.copy(); tp[i] += np.pi / 2
        tm = thetas.copy(); tm[i] -= np.pi / 2
        g[i] = 0.5 * (expect_fdm(n, ops, tp, terms) - expect_fdm(n, ops, tm, terms))
    return g
