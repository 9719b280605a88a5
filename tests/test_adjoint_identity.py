"""The adjoint formulas the GPU backward pass implements, checked against central
finite differences in FP64 on the CPU (no GPU, no CUDA code).

Loss L = Tr(V^dag H V) (real, H Hermitian); Vbar = dL/dconj(V) = H V and
dL = 2 Re <Vbar, dV>. Backward through one truncation V = V' U_r, where U_r holds
the k leading eigenvectors of V'^dag V' = U Lambda U^dag (Theorem 1):

    A = U_d^dag (V'^dag Vbar),  F_ji = 1 / (lambda_i - lambda_j)  (j discarded, i kept)
    B = U_d (F o A) U_r^dag,    Vbar' = Vbar U_r^dag + V' (B + B^dag)

Backward through a gate and channel V' = [Kt_a G(theta) V] (Eq. 4):
Vbar = sum_a (Kt_a G)^dag Vbar'_a and dL/dtheta = 2 Re sum_a <Vbar'_a, Kt_a G'(theta) V>.
"""
import numpy as np
import pytest

from oracle import lret as O


def _rand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _herm(rng, N):
    X = _rand(rng, N, N)
    return (X + X.conj().T) / 2


def _truncate(Vp, k):
    lam, U = np.linalg.eigh(Vp.conj().T @ Vp)
    lam, U = lam[::-1], U[:, ::-1]
    return Vp @ U[:, :k], lam, U


def _loss(V, H):
    return float(np.real(np.trace(V.conj().T @ H @ V)))


def _truncation_adjoint(Vp, Vbar, k):
    lam, U = np.linalg.eigh(Vp.conj().T @ Vp)
    lam, U = lam[::-1], U[:, ::-1]
    Ur, Ud = U[:, :k], U[:, k:]
    A = Ud.conj().T @ (Vp.conj().T @ Vbar)
    F = 1.0 / (lam[None, :k] - lam[k:, None])
    B = Ud @ (F * A) @ Ur.conj().T
    return Vbar @ Ur.conj().T + Vp @ (B + B.conj().T)


@pytest.mark.parametrize("N,m,k,seed", [(8, 6, 3, 1), (16, 8, 2, 2), (12, 5, 4, 3)])
def test_truncation_adjoint_matches_finite_differences(N, m, k, seed):
    rng = np.random.default_rng(seed)
    Vp = _rand(rng, N, m)
    H = _herm(rng, N)
    V, lam, _ = _truncate(Vp, k)
    assert lam[k - 1] - lam[k] > 1e-3 * lam[0]  # a clear cut: the truncation is differentiable
    Vbar_p = _truncation_adjoint(Vp, H @ V, k)
    h = 1e-6
    for _ in range(4):
        E = _rand(rng, N, m)
        fd = (_loss(_truncate(Vp + h * E, k)[0], H) - _loss(_truncate(Vp - h * E, k)[0], H)) / (2 * h)
        an = 2 * np.real(np.sum(Vbar_p.conj() * E))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_truncation_adjoint_needs_the_spectral_term():
    """Dropping B (the kept x discarded eigenvector response) breaks the gradient:
    V'^dag V' changes with V', so U_r does too."""
    rng = np.random.default_rng(5)
    Vp = _rand(rng, 8, 6)
    H = _herm(rng, 8)
    k = 3
    V, _, U = _truncate(Vp, k)
    without = (H @ V) @ U[:, :k].conj().T
    E = _rand(rng, 8, 6)
    h = 1e-6
    fd = (_loss(_truncate(Vp + h * E, k)[0], H) - _loss(_truncate(Vp - h * E, k)[0], H)) / (2 * h)
    assert abs(fd - 2 * np.real(np.sum(without.conj() * E))) > 1e-3 * abs(fd)


@pytest.mark.parametrize("axis,chan", [("y", "dep"), ("z", "ad"), ("x", "dep")])
def test_gate_and_channel_adjoint_matches_finite_differences(axis, chan):
    """One rotation on qubit q, its channel, a truncation: dL/dtheta from the chain
    (truncation adjoint, then the expansion adjoint) against central differences."""
    n, q, c, k = 3, 1, 2, 3
    rng = np.random.default_rng(11)
    V = _rand(rng, 2 ** n, c)
    H = _herm(rng, 2 ** n)
    ks = O.depolarizing(0.1) if chan == "dep" else O.amplitude_damping(0.25)

    def forward(theta):
        G = O.rotation(axis, theta)
        Vp = np.hstack([O.apply_rows(n, V, [q], K @ G) for K in ks])
        return Vp, _truncate(Vp, k)[0]

    theta = 0.7
    Vp, Vk = forward(theta)
    Vbar_p = _truncation_adjoint(Vp, H @ Vk, k)
    dG = O.rotation_derivative(axis, theta)
    grad = 0.0
    for a, K in enumerate(ks):
        grad += 2 * np.real(np.sum(Vbar_p[:, a * c:(a + 1) * c].conj() * O.apply_rows(n, V, [q], K @ dG)))
    h = 1e-6
    fd = (_loss(forward(theta + h)[1], H) - _loss(forward(theta - h)[1], H)) / (2 * h)
    assert abs(fd - grad) < 1e-6 * max(1.0, abs(grad))
