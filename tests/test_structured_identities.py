"""Exact identities behind the truncation that never forms V' (CPU, NumPy).

The GPU path truncates a channel on qubit q from the row pairs of V: rows with
bit q = 0 (V_0) and bit q = 1 (V_1). With A_alpha = K_alpha G (Kraus matrix
times the one-qubit gate folded into it) the expanded state V' = [A_1 V, ...,
A_K V] (Eq. 4) has the Gram matrix (Theorem 1)

    G'_{alpha beta} = sum_{b, b'} (A_alpha^dag A_beta)[b, b'] V_b^dag V_b'

and the projection V' U onto kept eigenvectors U is, on the rows with bit q = a,
sum_b V_b C_ab with C_ab = sum_alpha A_alpha[a, b] U^(alpha). These tests build
V' explicitly and check both identities, the composition rule of a deferred
projection (the pair Gram of [V_0 V_1] C is C^dag S C), and the two-qubit form
(the pair Gram on a second qubit from the quad Gram of V). Independent of the
CUDA path and of the oracle's own state classes.
"""
import numpy as np
import pytest

from oracle import lret as O


def _rand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _rows_with_bit(n, q, b):
    x = np.arange(2 ** n)
    return x[((x >> q) & 1) == b]


def _apply_one_qubit(n, V, q, A):
    """(A on qubit q) V, written out row by row: out[x] = sum_b A[bit_q(x), b] V[x with bit q = b]."""
    out = np.zeros_like(V)
    for x in range(2 ** n):
        a = (x >> q) & 1
        for b in (0, 1):
            out[x] += A[a, b] * V[(x & ~(1 << q)) | (b << q)]
    return out


def _kraus_with_gate(kind, seed):
    rng = np.random.default_rng(seed)
    G = np.linalg.qr(_rand(rng, 2, 2))[0]  # a random one-qubit unitary folded into the channel
    ks = O.depolarizing(0.07) if kind == "dep" else O.amplitude_damping(0.3)
    return [K @ G for K in ks]


@pytest.mark.parametrize("kind", ["dep", "ad"])
@pytest.mark.parametrize("n,q,c", [(4, 0, 3), (5, 2, 4), (5, 4, 2)])
def test_pair_gram_assembly_equals_expanded_gram(kind, n, q, c):
    rng = np.random.default_rng(100 + n + q)
    V = _rand(rng, 2 ** n, c)
    A = _kraus_with_gate(kind, n * 7 + q)
    Vx = np.hstack([_apply_one_qubit(n, V, q, Aa) for Aa in A])
    G_direct = Vx.conj().T @ Vx
    Vb = [V[_rows_with_bit(n, q, b)] for b in (0, 1)]
    S = {(b, bb): Vb[b].conj().T @ Vb[bb] for b in (0, 1) for bb in (0, 1)}
    K = len(A)
    G_pair = np.zeros((K * c, K * c), dtype=complex)
    for al in range(K):
        for be in range(K):
            M = A[al].conj().T @ A[be]
            G_pair[al * c:(al + 1) * c, be * c:(be + 1) * c] = sum(M[b, bb] * S[b, bb] for b in (0, 1) for bb in (0, 1))
    assert np.max(np.abs(G_pair - G_direct)) < 1e-12 * np.max(np.abs(G_direct))


@pytest.mark.parametrize("kind", ["dep", "ad"])
def test_pair_projection_equals_expanded_projection(kind):
    n, q, c, k = 5, 1, 4, 3
    rng = np.random.default_rng(7)
    V = _rand(rng, 2 ** n, c)
    A = _kraus_with_gate(kind, 11)
    Vx = np.hstack([_apply_one_qubit(n, V, q, Aa) for Aa in A])
    lam, U = np.linalg.eigh(Vx.conj().T @ Vx)
    Ur = U[:, ::-1][:, :k]
    direct = Vx @ Ur
    Vb = [V[_rows_with_bit(n, q, b)] for b in (0, 1)]
    for a in (0, 1):
        C = [sum(A[al][a, b] * Ur[al * c:(al + 1) * c] for al in range(len(A))) for b in (0, 1)]
        pair = Vb[0] @ C[0] + Vb[1] @ C[1]
        assert np.max(np.abs(pair - direct[_rows_with_bit(n, q, a)])) < 1e-12


def test_deferred_projection_pair_gram_is_c_dag_s_c():
    """W_a = sum_b V_b C_ab on the same qubit: [W_0 W_1] = [V_0 V_1] Cb with block
    (b, a) of Cb equal to C_ab, so the pair Gram of W is Cb^dag S Cb."""
    n, q, c, k = 5, 3, 4, 3
    rng = np.random.default_rng(21)
    V = _rand(rng, 2 ** n, c)
    C = {(a, b): _rand(rng, c, k) for a in (0, 1) for b in (0, 1)}
    rows = [_rows_with_bit(n, q, b) for b in (0, 1)]
    Vb = [V[rows[b]] for b in (0, 1)]
    W = np.zeros((2 ** n, k), dtype=complex)
    for a in (0, 1):
        W[rows[a]] = Vb[0] @ C[a, 0] + Vb[1] @ C[a, 1]
    P = np.hstack(Vb)
    S = P.conj().T @ P
    Cb = np.block([[C[0, 0], C[1, 0]], [C[0, 1], C[1, 1]]])
    Wp = np.hstack([W[rows[0]], W[rows[1]]])
    assert np.max(np.abs(Wp.conj().T @ Wp - Cb.conj().T @ S @ Cb)) < 1e-11


@pytest.mark.parametrize("q,q2", [(1, 3), (3, 1), (0, 4)])
def test_pair_gram_on_second_qubit_from_quad_gram(q, q2):
    """A state pending on qubit q (W_a = sum_b V_b C_ab) has, on another qubit q2,
    the pair Gram S'_{d d'} = sum_a sum_{b, b'} C_ab^dag Q_{(b, d), (b', d')} C_ab',
    Q being the Gram of the four row blocks of V split on bits q and q2."""
    n, c, k = 5, 3, 2
    rng = np.random.default_rng(31 + q + q2)
    V = _rand(rng, 2 ** n, c)
    C = {(a, b): _rand(rng, c, k) for a in (0, 1) for b in (0, 1)}
    x = np.arange(2 ** n)
    W = np.zeros((2 ** n, k), dtype=complex)
    for xi in x:  # W[x] = sum_b V[x with bit q = b] C_{bit_q(x), b}
        a = (xi >> q) & 1
        for b in (0, 1):
            W[xi] += V[(xi & ~(1 << q)) | (b << q)] @ C[a, b]

    def block(M, bq, bq2):  # rows with bit q = bq and bit q2 = bq2, in ascending order of x
        sel = x[(((x >> q) & 1) == bq) & (((x >> q2) & 1) == bq2)]
        return M[sel]

    Q = {(b, d, bb, dd): block(V, b, d).conj().T @ block(V, bb, dd)
         for b in (0, 1) for d in (0, 1) for bb in (0, 1) for dd in (0, 1)}
    for d in (0, 1):
        for dd in (0, 1):
            # direct: rows of W with bit q2 = d against rows with bit q2 = dd, paired by the other bits
            direct = sum(block(W, a, d).conj().T @ block(W, a, dd) for a in (0, 1))
            quad = sum(C[a, b].conj().T @ Q[b, d, bb, dd] @ C[a, bb]
                       for a in (0, 1) for b in (0, 1) for bb in (0, 1))
            assert np.max(np.abs(direct - quad)) < 1e-11
