"""Pins for the CPU oracle: closed forms, invariants and exact identities.

Each test ties the oracle to something other than itself: a value the paper's
definitions fix in closed form, a textbook identity, or an independent
construction (dense Kronecker products, the exact density matrix, the
statevector). A plausible slip anywhere in the oracle (a dropped Kraus term, a
wrong sign or qubit index, a transposed factor) fails at least one of them.
"""
import numpy as np
import pytest

from oracle import lret as O
from workloads import random_layered, random_pauli_sum, hea


def kron_pauli(n, term):
    """Dense 2^n x 2^n Pauli string built by Kronecker products (independent of apply_rows)."""
    mats = [O.I2] * n
    for q, s in term:
        mats[q] = O.PAULI[s]
    out = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):  # most significant qubit first
        out = np.kron(out, mats[q])
    return out


# ---- channels (Sec. III.A) -------------------------------------------------

@pytest.mark.parametrize("p", [0.0, 1e-3, 0.0033, 0.2, 0.75])
def test_kraus_completeness(p):
    for ks in (O.depolarizing(p), O.amplitude_damping(p), O.bit_flip(p)):
        S = sum(K.conj().T @ K for K in ks)
        assert np.max(np.abs(S - np.eye(2))) < 1e-15


def test_depolarizing_on_zero_closed_form():
    p = 0.03
    st = O.LRETState(1)
    st.channel(0, O.depolarizing(p))
    pr = st.probs()
    # (1-p)|0><0| + p/3 (|1><1| + |1><1| + |0><0|)
    assert np.allclose(pr, [1 - 2 * p / 3, 2 * p / 3], atol=1e-15)


def test_amplitude_damping_on_one_closed_form():
    g = 0.07
    st = O.LRETState(1)
    st.gate([0], O.PAULI["X"])
    st.channel(0, O.amplitude_damping(g))
    assert np.allclose(st.probs(), [g, 1 - g], atol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 5])
def test_ry_then_depolarizing_z_closed_form(k):
    # Ry(t)|0> has <Z> = cos t, <X> = sin t; each depolarizing scales the Bloch vector by 1 - 4p/3
    t, p = 0.7, 0.02
    st = O.LRETState(1)
    st.gate([0], O.rotation("Y", t))
    for _ in range(k):
        st.channel(0, O.depolarizing(p))
    f = (1 - 4 * p / 3) ** k
    assert abs(st.expect([(1.0, [(0, "Z")])]) - f * np.cos(t)) < 1e-14
    assert abs(st.expect([(1.0, [(0, "X")])]) - f * np.sin(t)) < 1e-14


def test_rotation_sign_conventions():
    # Ry(pi/2)|0> = |+>; Rz(phi) then gives <X> = cos phi, <Y> = sin phi
    phi = 0.4
    st = O.SVState(1)
    st.gate([0], O.rotation("Y", np.pi / 2))
    st.gate([0], O.rotation("Z", phi))
    assert abs(st.expect([(1.0, [(0, "X")])]) - np.cos(phi)) < 1e-14
    assert abs(st.expect([(1.0, [(0, "Y")])]) - np.sin(phi)) < 1e-14
    # Rx(t)|0>: <Y> = -sin t
    st = O.SVState(1)
    st.gate([0], O.rotation("X", 0.3))
    assert abs(st.expect([(1.0, [(0, "Y")])]) + np.sin(0.3)) < 1e-14


def test_rotation_derivative_matches_fd():
    for ax in "XYZ":
        t, h = 0.37, 1e-6
        fd = (O.rotation(ax, t + h) - O.rotation(ax, t - h)) / (2 * h)
        assert np.max(np.abs(fd - O.rotation_derivative(ax, t))) < 1e-9


def test_cnot_and_qubit_order():
    # |x> with x = 1 (qubit 0 set). CNOT(0 -> 2) must give x = 1 + 4 = 5.
    n = 3
    st = O.SVState(n)
    st.gate([0], O.PAULI["X"])
    st.gate([0, 2], O.cnot())
    assert abs(st.probs()[5] - 1.0) < 1e-15
    # CNOT(2 -> 0) on the same state does nothing (control qubit 2 is 0)
    st2 = O.SVState(n)
    st2.gate([0], O.PAULI["X"])
    st2.gate([2, 0], O.cnot())
    assert abs(st2.probs()[1] - 1.0) < 1e-15
    # CZ phase: |11> on qubits (1,2) picks up -1; check via <X_1> after H-like prep
    st3 = O.SVState(3)
    st3.gate([1], O.rotation("Y", np.pi / 2))
    st3.gate([2], O.PAULI["X"])
    st3.gate([1, 2], O.cz())
    assert abs(st3.expect([(1.0, [(1, "X")])]) + 1.0) < 1e-14


def test_apply_rows_matches_kron():
    rng = np.random.default_rng(1)
    n = 4
    A = rng.normal(size=(2 ** n, 3)) + 1j * rng.normal(size=(2 ** n, 3))
    U = np.linalg.qr(rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)))[0]
    # dense operator for U on qubits (3, 1): basis index of U = 2*b3 + b1
    D = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for x in range(2 ** n):
        b3, b1 = (x >> 3) & 1, (x >> 1) & 1
        for o in range(4):
            y = x & ~(1 << 3) & ~(1 << 1)
            y |= ((o >> 1) & 1) << 3
            y |= (o & 1) << 1
            D[y, x] += U[o, 2 * b3 + b1]
    assert np.allclose(O.apply_rows(n, A, [3, 1], U), D @ A, atol=1e-13)


def test_pauli_expectation_matches_dense_kron():
    rng = np.random.default_rng(2)
    n = 5
    L = rng.normal(size=(2 ** n, 4)) + 1j * rng.normal(size=(2 ** n, 4))
    terms = random_pauli_sum(n, 12, seed=7)
    st = O.LRETState(n)
    st.L = L
    H = sum(c * kron_pauli(n, t) for c, t in terms)
    ref = np.real(np.trace(H @ (L @ L.conj().T)))
    assert abs(st.expect(terms) - ref) < 1e-11
    # Y on (|0> + i|1>)/sqrt2 is +1
    s = O.SVState(1)
    s.psi = np.array([[1.0], [1j]]) / np.sqrt(2)
    assert abs(s.expect([(1.0, [(0, "Y")])]) - 1.0) < 1e-15


def test_z_expect_matches_dense_kron_on_every_qubit():
    # <Z_q> from Prob(x) (Eq. 9 weighted by (-1)^{x_q}) against Tr(Z_q rho) with Z_q a
    # dense Kronecker product, on a random unnormalised low-rank state
    rng = np.random.default_rng(21)
    n = 5
    L = rng.normal(size=(2 ** n, 3)) + 1j * rng.normal(size=(2 ** n, 3))
    st = O.LRETState(n)
    st.L = L
    rho = L @ L.conj().T
    z = st.z_expect()
    assert z.shape == (n,)
    for q in range(n):
        ref = np.real(np.trace(kron_pauli(n, [(q, "Z")]) @ rho))
        assert abs(z[q] - ref) < 1e-11
        assert abs(z[q] - st.expect([(1.0, [(q, "Z")])])) < 1e-11
    assert abs(st.trace() - np.real(np.trace(rho))) < 1e-11


def test_z_expect_closed_forms_on_product_states():
    # Ry(t_q) on every qubit, a depolarizing channel on qubit 1 and amplitude damping on
    # the top qubit: <Z_q> = cos t_q, (1 - 4p/3) cos t_1 on qubit 1, and for the damped
    # qubit (1 - g) (cos t - 1) + 1 = cos t + g (1 - cos t). An X on qubit 2 flips its
    # sign. A wrong bit index or sign in the readout fails one of these.
    n, p, g = 4, 0.05, 0.3
    t = np.array([0.3, 1.1, 2.0, 0.8])
    st = O.LRETState(n)
    for q in range(n):
        st.gate([q], O.rotation("Y", t[q]))
    st.gate([2], O.PAULI["X"])
    st.channel(1, O.depolarizing(p))
    st.channel(n - 1, O.amplitude_damping(g))
    expect = np.cos(t)
    expect[1] *= 1 - 4 * p / 3
    expect[2] *= -1.0
    expect[n - 1] = np.cos(t[n - 1]) + g * (1 - np.cos(t[n - 1]))
    assert np.max(np.abs(st.z_expect() - expect)) < 1e-14
    assert abs(st.trace() - 1.0) < 1e-14


# ---- exact evolution (Eq. 1) ----------------------------------------------

def test_fdm_trace_positivity_and_sv():
    n = 4
    ops = random_layered(n, 3, seed=11, noise=("mixed", 0.05, 0.08))
    st = O.run_fdm(n, ops)
    assert abs(np.trace(st.rho).real - 1) < 1e-13
    assert np.min(np.linalg.eigvalsh(st.rho)) > -1e-13
    ops0 = random_layered(n, 3, seed=11, noise=None)
    fd0 = O.run_fdm(n, ops0)
    sv = O.run_sv(n, ops0)
    assert np.max(np.abs(fd0.rho - sv.psi @ sv.psi.conj().T)) < 1e-13


# ---- low rank vs exact -----------------------------------------------------

def test_lret_full_rank_equals_fdm():
    # 6 qubits, r = 64 >= rank: Algorithm 1 reproduces Eq. (1) to 1e-12
    n = 6
    ops = random_layered(n, 4, seed=1001, noise=("mixed", 0.01, 0.02))
    lr = O.run_lret(n, ops, r=2 ** n)
    fd = O.run_fdm(n, ops)
    assert np.max(np.abs(lr.rho() - fd.rho)) < 1e-12
    assert lr.discarded < 1e-12
    terms = random_pauli_sum(n, 20, seed=5)
    assert abs(lr.expect(terms) - fd.expect(terms)) < 1e-12


def test_lret_zero_noise_equals_statevector():
    n = 5
    ops = random_layered(n, 5, seed=3, noise=("dep", 0.0))
    lr = O.run_lret(n, ops, r=1)
    sv = O.run_sv(n, ops)
    assert np.max(np.abs(lr.probs() - sv.probs())) < 1e-13
    assert abs(lr.trace() - 1.0) < 1e-13


def test_theorem1_gram_spectrum():
    # App. B: B^dag B and B B^dag share the m nonzero eigenvalues; B u are eigenvectors
    rng = np.random.default_rng(4)
    B = rng.normal(size=(40, 7)) + 1j * rng.normal(size=(40, 7))
    lm, U = np.linalg.eigh(B.conj().T @ B)
    lD = np.linalg.eigvalsh(B @ B.conj().T)
    assert np.allclose(np.sort(lD)[-7:], lm, rtol=1e-12, atol=1e-10)
    D = B @ B.conj().T
    for i in range(7):
        v = B @ U[:, i]
        assert np.allclose(D @ v, lm[i] * v, atol=1e-9)


def test_truncation_error_equals_discarded_mass():
    # Eckart-Young (Sec. II.B): || rho' - rho_trunc ||_1 = sum of dropped eigenvalues
    n = 4
    ops = random_layered(n, 1, seed=8, noise=("dep", 0.05))
    chans = [i for i, o in enumerate(ops) if O.is_channel(o)]
    ops = [o for i, o in enumerate(ops) if not O.is_channel(o) or i in chans[:3]]
    st = O.run_lret(n, ops, compress=False)  # untruncated L, 4^3 columns
    rho_full = st.rho()
    d = st.compress(r=3)
    diff = np.linalg.eigvalsh(rho_full - st.rho())
    assert abs(np.sum(np.abs(diff)) - d) < 1e-13
    assert d > 1e-4
    # trace bookkeeping: Tr rho = 1 - cumulative discarded mass
    assert abs(st.trace() - (1 - d)) < 1e-13


def test_product_state_spectrum_closed_form():
    # depolarizing on each of 3 qubits of |000>: eigenvalues are products of (1-2p/3, 2p/3)
    n, p = 3, 0.1
    st = O.LRETState(n)
    for q in range(n):
        st.channel(q, O.depolarizing(p))
    a, b = 1 - 2 * p / 3, 2 * p / 3
    from math import comb
    expect = sorted([a ** (n - k) * b ** k for k in range(n + 1) for _ in range(comb(n, k))], reverse=True)
    d = st.compress(r=4)
    lam = st.log[-1]["lam"]
    assert np.allclose(lam[:8], expect, atol=1e-14)
    assert abs(d - sum(expect[4:])) < 1e-14


def test_eps_rule_reading():
    lam = np.array([0.6, 0.3, 0.05, 0.03, 0.02])
    # cumulative 0.6, 0.9, 0.95, 0.98, 1.0; eps = 0.05 -> reach 0.95 with k = 3 (crossing kept)
    assert O.choose_rank(lam, eps=0.05) == 3
    assert O.choose_rank(lam, eps=0.049) == 4
    assert O.choose_rank(lam, eps=0.5) == 1
    assert O.choose_rank(lam, r=2) == 2
    assert O.choose_rank(lam, r=9) == 5


def test_lowrank_trace_distance_matches_dense():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(32, 3)) + 1j * rng.normal(size=(32, 3))
    B = rng.normal(size=(32, 5)) + 1j * rng.normal(size=(32, 5))
    dense = 0.5 * np.sum(np.abs(np.linalg.eigvalsh(A @ A.conj().T - B @ B.conj().T)))
    assert abs(O.trace_distance_lowrank(A, B) - dense) < 1e-10


def test_lowrank_trace_distance_of_nearly_equal_states():
    """Two states with the same eigenvectors and eigenvalues that differ by 1e-12:
    the trace distance is half the sum of the eigenvalue differences exactly, a
    case where a nearly defective eigenproblem would leave an error near 1e-8."""
    rng = np.random.default_rng(10)
    Q, _ = np.linalg.qr(rng.normal(size=(256, 8)) + 1j * rng.normal(size=(256, 8)))
    lam = np.sort(rng.uniform(size=8))[::-1]
    lam /= lam.sum()
    dl = 1e-12 * rng.choice([-1.0, 1.0], size=8)
    A = Q * np.sqrt(lam)
    B = (Q * np.sqrt(lam + dl)) @ np.linalg.qr(rng.normal(size=(8, 8)))[0]  # other gauge
    assert abs(O.trace_distance_lowrank(A, B) - 0.5 * np.sum(np.abs(dl))) < 1e-14
    assert O.trace_distance_lowrank(A, A) < 1e-15


# ---- gradients -------------------------------------------------------------

def test_gradient_fd_full_rank_matches_parameter_shift():
    # r = 2^n LRET is exact, so its FD gradient equals the parameter-shift gradient of Eq. (1)
    n = 3
    ops, th = hea(n, 2, seed=4000, noise=("dep", 0.02))
    terms = random_pauli_sum(n, 6, seed=41)
    g_fd = O.gradient_fd_lret(n, ops, th, terms, r=2 ** n, h=1e-4)
    g_ps = O.gradient_param_shift_fdm(n, ops, th, terms)
    assert np.max(np.abs(g_fd - g_ps)) < 1e-8
    assert np.max(np.abs(g_ps)) > 1e-2


def test_distortion_definition():
    pe = np.array([0.5, 0.3, 0.2])
    pn = np.array([0.6, 0.3, 0.1])
    pl = np.array([0.52, 0.29, 0.19])
    assert abs(O.distortion(pl, pe, pn) - (0.04 / 0.2)) < 1e-15


# ---- von Neumann entropy (App. A) and measurement sampling (Sec. II.D) -----

def _h2(x):
    return -x * np.log2(x) - (1 - x) * np.log2(1 - x)


def test_entropy_pure_state_is_zero():
    st = O.LRETState(3)
    for q in range(3):
        st.gate([q], O.rotation("Y", 0.3 + q))
    st.gate([0, 1], O.cnot())
    assert abs(st.entropy()) < 1e-12


@pytest.mark.parametrize("p", [1e-3, 0.05, 0.75])
def test_entropy_of_depolarized_product_state_closed_form(p):
    # each qubit of |0..0> after its own depolarizing channel has spectrum
    # (1 - 2p/3, 2p/3), so S = n * H2(2p/3) bits; p = 3/4 gives I/2 per qubit, S = n
    n = 3
    st, fdm = O.LRETState(n), O.FDMState(n)
    for q in range(n):
        st.channel(q, O.depolarizing(p))
        fdm.channel(q, O.depolarizing(p))
    want = n * _h2(2 * p / 3)
    assert abs(st.entropy() - want) < 1e-12
    assert abs(O.entropy_dense(fdm.rho) - want) < 1e-12
    if p == 0.75:
        assert abs(st.entropy() - n) < 1e-12


def test_entropy_lowrank_matches_dense_after_truncation():
    # the Gram-spectrum route (Theorem 1) against the eigenvalues of the dense
    # L L^dag, on a truncated state (trace below 1: both normalise)
    n = 5
    ops = random_layered(n, 4, seed=77, noise=("dep", 0.02))
    st = O.run_lret(n, ops, r=6)
    assert st.trace() < 1.0
    assert abs(st.entropy() - O.entropy_dense(st.rho())) < 1e-10
    # normalisation: a scaled spectrum has the same entropy, two equal weights give 1 bit
    assert abs(O.entropy_from_eigenvalues([0.2, 0.2]) - 1.0) < 1e-15
    lam = np.array([0.5, 0.3, 0.2, 0.0, -1e-17])
    assert abs(O.entropy_from_eigenvalues(3.7 * lam) - O.entropy_from_eigenvalues(lam)) < 1e-15


def test_entropy_full_rank_lret_matches_fdm():
    n = 4
    ops = random_layered(n, 3, seed=78, noise=("mixed", 0.02, 0.05))
    lret, fdm = O.run_lret(n, ops, r=2 ** n), O.run_fdm(n, ops)
    assert abs(lret.entropy() - O.entropy_dense(fdm.rho)) < 1e-10


def test_sampling_uniform_distribution_closed_form():
    # Ry(pi/2) on every qubit gives Prob(x) = 2^-n: shot u lands on floor(u 2^n)
    n = 4
    sv = O.SVState(n)
    for q in range(n):
        sv.gate([q], O.rotation("Y", np.pi / 2))
    k = np.arange(2 ** n)
    u = (k + 0.5) / 2 ** n
    assert np.array_equal(O.sample_inverse_cdf(sv.probs(), u), k)


def test_sampling_matches_brute_force_definition():
    rng = np.random.default_rng(5)
    p = rng.random(7)
    p[[1, 4]] = 0.0  # zero-probability outcomes are never drawn
    u = rng.random(500)
    got = O.sample_inverse_cdf(p, u)
    tot = sum(p)
    for s, us in zip(got, u):
        acc, want = 0.0, len(p) - 1
        for x in range(len(p)):
            acc += p[x]
            if acc > us * tot:
                want = x
                break
        assert s == want
        assert p[s] > 0


# ---- randomized-benchmarking gate set and bit flip (Sec. III) ----------------

def test_fixed_one_qubit_gate_identities():
    S, T, X, Y, Z = (O.FIXED_1Q[k] for k in ("s", "t", "x", "y", "z"))
    assert np.allclose(S @ S, Z, atol=1e-15)
    assert np.allclose(T @ T, S, atol=1e-15)
    assert np.allclose(np.linalg.matrix_power(T, 8), np.eye(2), atol=1e-15)
    assert np.allclose(X @ Y, 1j * Z, atol=1e-15)  # Pauli algebra fixes the signs of Y
    # S maps <X> to <Y> on |+>: Ry(pi/2)|0> = |+>, then S
    sv = O.SVState(1)
    sv.gate([0], O.rotation("Y", np.pi / 2))
    sv.gate([0], S)
    assert abs(sv.expect([(1.0, [(0, "Y")])]) - 1.0) < 1e-14


def test_swap_is_three_cnots_and_moves_a_flip():
    C01 = O.cnot()  # control q0, target q1 in the basis 2 b(q0) + b(q1)
    # CNOT with control q1, target q0 in the same basis
    C10 = np.zeros((4, 4), dtype=np.complex128)
    for b0 in range(2):
        for b1 in range(2):
            C10[2 * (b0 ^ b1) + b1, 2 * b0 + b1] = 1.0
    assert np.allclose(C01 @ C10 @ C01, O.swap(), atol=1e-15)
    st = O.SVState(3)
    st.gate([0], O.FIXED_1Q["x"])          # |001>: qubit 0 set
    st.gate([0, 2], O.swap())              # qubit 2 set -> index 4
    assert abs(st.probs()[4] - 1.0) < 1e-15


def test_bit_flip_on_zero_closed_form():
    p = 0.07
    st = O.LRETState(2)
    st.channel(1, O.bit_flip(p))
    assert np.allclose(st.probs(), [1 - p, 0, p, 0], atol=1e-15)


def test_rb_circuit_lret_full_rank_equals_fdm():
    from workloads import random_rb
    n = 4
    ops = random_rb(n, 4, seed=91, noise=("mixed3", 0.02, 0.05, 0.03))
    names = {o["op"] for o in ops}
    assert {"swap", "cz", "cnot"} & names and {"x", "s", "t", "rx"} & names and "bf" in names
    lret, fdm = O.run_lret(n, ops, r=2 ** n), O.run_fdm(n, ops)
    assert np.max(np.abs(lret.rho() - fdm.rho)) < 1e-12


# ---- dense k-qubit and diagonal gates, Kraus groups, Grover (Sec. II.C, III.D) --

def _rand_unitary(rng, d):
    Z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))[None, :]


def test_dense_gate_is_kron_of_its_factors_first_qubit_most_significant():
    rng = np.random.default_rng(11)
    n = 5
    A = rng.normal(size=(2 ** n, 3)) + 1j * rng.normal(size=(2 ** n, 3))
    qs = [3, 0, 4]
    F = [_rand_unitary(rng, 2) for _ in qs]
    seq = A
    for q, M in zip(qs, F):
        seq = O.apply_rows(n, seq, [q], M)
    dense = O.apply_rows(n, A, qs, np.kron(np.kron(F[0], F[1]), F[2]))
    assert np.max(np.abs(dense - seq)) < 1e-13


def test_dense_permutation_moves_basis_state_by_hand():
    # 3-qubit cyclic shift i -> i + 1 (mod 8) on qubits (q0, q1, q2) = (1, 4, 2):
    # index i = 4 b(1) + 2 b(4) + b(2)
    n = 5
    P = np.zeros((8, 8), dtype=np.complex128)
    for i in range(8):
        P[(i + 1) % 8, i] = 1.0
    # |x> with b(1) = 0, b(4) = 1, b(2) = 1 -> i = 3 -> 4 = (b(1)=1, b(4)=0, b(2)=0)
    x = (1 << 4) | (1 << 2) | (1 << 0)  # qubit 0 set as a spectator
    st = O.SVState(n)
    st.psi[:] = 0
    st.psi[x, 0] = 1.0
    st.gate([1, 4, 2], P)
    y = (1 << 1) | (1 << 0)
    assert abs(st.probs()[y] - 1.0) < 1e-15


def test_diagonal_gate_matches_dense_and_bitwise_definition():
    rng = np.random.default_rng(12)
    n = 6
    qs = [2, 5, 0, 3]
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, size=16))
    A = rng.normal(size=(2 ** n, 4)) + 1j * rng.normal(size=(2 ** n, 4))
    got = O.apply_diag_rows(n, A, qs, d)
    assert np.max(np.abs(got - O.apply_rows(n, A, qs, np.diag(d)))) < 1e-13
    for x in range(2 ** n):  # index from the binary string, most significant qubit first
        bits = format(x, f"0{n}b")[::-1]
        i = int("".join(bits[q] for q in qs), 2)
        assert np.max(np.abs(got[x] - d[i] * A[x])) < 1e-14


@pytest.mark.parametrize("n", [5, 6, 7])
@pytest.mark.parametrize("dense", [True, False])
def test_grover_noiseless_success_closed_form(n, dense):
    from workloads import grover, grover_good
    ops, t = grover(n, p=0.0, dense=dense)
    good = grover_good(n)
    theta = np.arcsin(np.sqrt(good.sum() / 2 ** n))
    pg = O.run_sv(n, ops).probs()[good].sum()
    assert abs(pg - np.sin((2 * t + 1) * theta) ** 2) < 1e-12
    assert t == int(np.floor(np.pi / 4 * np.sqrt(2 ** n / good.sum())))


def test_grover_dense_and_decomposed_iterates_agree_under_noise():
    from workloads import grover
    n = 4
    a, _ = grover(n, p=0.02, dense=True)
    b, _ = grover(n, p=0.02, dense=False)
    ra, rb = O.run_fdm(n, a).rho, O.run_fdm(n, b).rho
    assert np.max(np.abs(ra - rb)) < 1e-13


def test_grover_lret_full_rank_equals_fdm():
    from workloads import grover
    n = 4
    ops, _ = grover(n, p=0.03, dense=False)
    lret, fdm = O.run_lret(n, ops, r=2 ** n), O.run_fdm(n, ops)
    assert np.max(np.abs(lret.rho() - fdm.rho)) < 1e-12


def test_kraus_groups_truncate_after_every_mth_channel():
    from workloads import random_rb
    ops = random_rb(4, 3, seed=93, noise=("dep", 0.01))
    nch = sum(1 for o in ops if O.is_channel(o))
    for M in (1, 2, 3):
        st = O.run_lret(4, ops, r=16, group=M)
        assert len(st.log) == -(-nch // M)
        assert np.max(np.abs(st.rho() - O.run_fdm(4, ops).rho)) < 1e-12


def test_kraus_group_truncation_is_the_best_rank_r_approximation():
    # from an exact state, one group of M = 2 channels then one truncation keeps
    # the top-r spectral part of the exact density matrix (Eckart-Young, Sec. II.B)
    from workloads import random_layered
    n, r = 4, 5
    pre = random_layered(n, 2, seed=94, noise=None)
    ops = pre + [{"op": "dep", "q": 1, "p": 0.2}, {"op": "ad", "q": 3, "gamma": 0.3}]
    st = O.run_lret(n, ops, r=r, group=2)
    assert len(st.log) == 1 and st.log[0]["m"] == 4 * 2  # one column, then K = 4 and K = 2
    rho = O.run_fdm(n, ops).rho
    w, U = np.linalg.eigh(rho)
    top = (U[:, -r:] * w[-r:]) @ U[:, -r:].conj().T
    assert np.max(np.abs(st.rho() - top)) < 1e-12
    assert abs(st.discarded - w[:-r].sum()) < 1e-12


# ---- printed values (tests/golden) -----------------------------------------

def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_app_a_effective_rank_growth_printed_values():
    """App. A prints gamma_bit ~ 0.008 and gamma_dep ~ 0.009 at p = 0.1 %: the oracle's
    entropy of one bit flip on |0> and of a depolarizing channel on half of a Bell
    pair (where the entropy bound is attained) gives 2^S - 1 that rounds to them."""
    g = _golden("app_a_effective_rank.txt")
    p = g["p"]
    st = O.LRETState(1)
    st.channel(0, O.bit_flip(p))
    gamma_bit = 2.0 ** st.entropy() - 1.0
    bell = O.LRETState(2)
    bell.gate([0], O.FIXED_1Q["h"])
    bell.gate([0, 1], O.cnot())
    bell.channel(0, O.depolarizing(p))
    gamma_dep = 2.0 ** bell.entropy() - 1.0
    assert round(gamma_bit, 3) == g["gamma_bit"]
    assert round(gamma_dep, 3) == g["gamma_dep"]
    # and they equal the bound -sum p_a log2 p_a itself
    assert abs(bell.entropy() - (-(1 - p) * np.log2(1 - p) - p * np.log2(p / 3))) < 1e-12
    assert abs(st.entropy() - (-(1 - p) * np.log2(1 - p) - p * np.log2(p))) < 1e-12
