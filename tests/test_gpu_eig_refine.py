"""The eigensolve of the FP32-state truncation (Sec. II.B) against the oracle's FP64
eigendecomposition of the same Gram matrix.

The FP32-state path solves the Gram matrix in FP32 and refines the kept
eigenvectors in FP64 (lr_set_eig_precision). Every truncation of a 14-qubit run of
the benchmark's circuit family (r = 64, 256-column Gram matrices) is read back
through lr_last_eig and compared with the oracle's eigh of the same FP64 matrix:

* the eigenvalues of the kept subspace (of X^dag G X) and the discarded mass (the
  trace the truncation removes, trace(G) minus the kept eigenvalues) to 1e-13 of the trace, each reported kept eigenvalue to 1e-13 of lambda_1 up to the spread of
  an eigenvalue cluster the FP32 solve cannot separate and the second-order effect of
  its mixing of nearby kept pairs (kept vectors are not rotated among themselves);
* the truncated state: rho_trunc = V' P V'^dag depends on the kept vectors only
  through the projector P, and ||V' (P - P0) V'^dag||_F = ||G^(1/2) (P - P0) G^(1/2)||_F,
  held to 1e-11 of the trace;
* where eigenvalues lie within the FP32 resolution (16 x 2^-24 lambda_1) of the cut,
  the kept set is chosen by the FP32 eigenvalues and may differ there (a tie at the
  state's precision): the bounds grow by the mass of those eigenvalues (twice for rho);
* orthonormality of the kept vectors to 1e-13.
The FP32 solve alone is checked to be at its own level on the same matrices, so the
refinement is what reaches the FP64 bounds.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lret as O  # noqa: E402
from workloads import random_layered  # noqa: E402


@pytest.fixture(scope="module")
def lr():
    import paper_2009_06657_gb300 as m
    return m


def _sqrt_psd(G):
    w, Q = np.linalg.eigh(0.5 * (G + G.conj().T))
    return (Q * np.sqrt(np.clip(w, 0.0, None))) @ Q.conj().T


def _rho_err(G, X, U0, k):
    Gh = _sqrt_psd(G)
    D = X[:, :k] @ X[:, :k].conj().T - U0[:, :k] @ U0[:, :k].conj().T
    return float(np.linalg.norm(Gh @ D @ Gh))


def _cuts(lr, n, r, nchan, mode, iters=1, seed=3000, solver="auto", depth=1, skip=0):
    """Run the benchmark family op by op (the library's default truncation path,
    deferred projections included) and return, for every truncation that drops
    columns, (G, evals, evecs, k, discarded mass of that truncation)."""
    ops = random_layered(n, depth, seed=seed, noise=("dep", 5e-4))
    sim = lr.LRSim(n, r, dtype="c64")
    sim.set_eig_precision(mode, iters)
    sim.set_eigensolver(solver)
    out, seen = [], 0
    for o in ops:
        if not O.is_channel(o):
            lr.run_ops(sim, [o], r=r)
            continue
        lr.run_ops(sim, [o], compress=False)
        d = sim.compress(r, want_discarded=True)  # synchronises; V stays as it is
        G, ev, U, k = sim.last_eig()
        fresh = not out or G.shape != out[-1][0].shape or not np.array_equal(G, out[-1][0])
        seen += 1
        if len(ev) > k and fresh and seen > skip:  # a truncation ran here (m <= r is skipped)
            out.append((G, ev, U, k, d))
        if seen >= skip + nchan:
            break
    sim.close()
    return out


# Resolution of the FP32 solve, relative to lambda_1: its eigenvalues carry errors of
# order 2^-24 lambda_1 times a small growth factor, and the Gram matrix of the FP32
# state carries errors of that order too. The kept set is chosen from the FP32
# eigenvalues, so eigenvalues within this window of the cut may be kept or dropped
# (they are tied at the state's precision); the refinement reaches FP64 accuracy for
# the pairs it separates.
FP32_RES = 16 * 2.0 ** -24
# Mixing angle of a kept pair in the FP32 solve, times the gap: the unit roundoff with a
# small growth factor.
FP32_MIX = 4 * 2.0 ** -24


def _cluster_spread(lam, i, width):
    """Largest distance from lam[i] to an eigenvalue within `width` of it."""
    d = np.abs(lam - lam[i])
    d = d[d <= width]
    return float(d.max()) if d.size else 0.0


def _kept_mixing(lam, i, k, res):
    """Second-order error of the Rayleigh quotient of kept vector i: the refinement does
    not rotate kept vectors among themselves (rho does not depend on it), so the FP32
    solve's mixing of kept pairs, of angle about res / |lam_i - lam_j|, stays and moves
    the quotient by about res^2 / |lam_i - lam_j| (pairs inside the resolution window
    FP32_RES are covered by the cluster spread)."""
    d = np.abs(lam[:k] - lam[i])
    d = d[d > FP32_RES * abs(lam[0])]
    return float(np.sum(res * res / d)) if d.size else 0.0


CASES = {
    # 14 qubits from |0...0>: the first truncations (rank-deficient Gram matrices)
    "n14-start": dict(n=14, nchan=16),
    # 10 qubits after 100 channels: full-rank Gram matrices with a dense spectrum below the cut
    "n10-steady": dict(n=10, nchan=12, depth=5, skip=100),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("solver", ["auto", "tridiag"])
def test_refined_eigensolve_matches_fp64(lr, solver, case):
    kw = dict(CASES[case])
    cuts = _cuts(lr, kw.pop("n"), 64, kw.pop("nchan"), "refined", solver=solver, **kw)
    assert len(cuts) >= 6
    rows = []
    for G, ev, U, k, dropped in cuts:
        lam0, U0 = O.gram_eigh(G)
        tr = float(np.real(np.trace(G)))
        l1 = lam0[0]
        gap = (lam0[k - 1] - lam0[k]) / l1
        X = U[:, :k]
        # eigenvalues of the kept subspace (invariant to rotations inside it)
        H = X.conj().T @ G @ X
        kc = np.linalg.eigvalsh(0.5 * (H + H.conj().T))[::-1]
        e_sub = float(np.max(np.abs(kc - lam0[:k]))) / l1
        # each kept eigenvalue, up to the spread of a cluster the FP32 solve cannot resolve
        e_lam = max(abs(ev[i] - lam0[i]) - _cluster_spread(lam0, i, FP32_RES * l1)
                    - _kept_mixing(lam0, i, k, FP32_MIX * l1) for i in range(k)) / l1
        e_rho = _rho_err(G, U, U0, k) / tr
        e_orth = float(np.max(np.abs(X.conj().T @ X - np.eye(k))))
        e_drop = abs(dropped - float(lam0[k:].sum())) / tr  # the trace the truncation removes
        # mass of the eigenvalues tied with the cut at the FP32 resolution
        win = np.abs(lam0 - 0.5 * (lam0[k - 1] + lam0[k])) <= FP32_RES * l1
        tied = float(np.clip(lam0[win], 0.0, None).sum()) / tr if gap <= FP32_RES else 0.0
        rows.append((gap, e_sub, e_lam, e_rho, e_orth, e_drop, tied))
    for r in rows:
        print("gap %.1e  kept-subspace eigenvalues %.1e  eigenvalues %.1e  rho %.1e  orthonormality %.1e  "
              "discarded %.1e  (tied mass %.1e)" % r)
    for gap, e_sub, e_lam, e_rho, e_orth, e_drop, tied in rows:
        assert e_orth < 1e-13
        assert e_lam < 1e-13
        assert e_sub * l1 / tr < 1e-13 + tied
        assert e_drop < 1e-13 + tied
        assert e_rho < 1e-11 + 2 * tied


def test_fp32_eigensolve_alone_is_at_fp32_level(lr):
    """The same matrices solved in FP32 only: errors at the FP32 level, far above the
    refined ones (the refinement is doing the work)."""
    cuts = _cuts(lr, 14, 64, 16, "fp32")
    errs = []
    for G, ev, U, k, _ in cuts:
        lam0, U0 = O.gram_eigh(G)
        tr = float(np.real(np.trace(G)))
        errs.append(_rho_err(G, U, U0, k) / tr)
        assert errs[-1] < 1e-4
    assert max(errs) > 1e-11, errs


def test_refined_eps_rule_on_fp32_state(lr):
    """Threshold rule (Sec. II.B) on the FP32 state: the kept count is chosen on the
    device from the FP32 eigenvalues and the refinement runs on every column the
    rule may keep; the kept count and the state match the oracle."""
    from workloads import random_pauli_sum
    n, eps = 8, 1e-3
    ops = random_layered(n, 2, seed=1201, noise=("dep", 0.01), qubit_jitter=(0.5, 1.5))
    ref = O.run_lret(n, ops, eps=eps)
    sim = lr.LRSim(n, 64, dtype="c64")
    sim.set_eps(eps)
    lr.run_ops(sim, ops, r=0)
    assert sim.info()["columns"] == ref.L.shape[1]
    p = sim.probs().double().cpu().numpy()
    assert np.sum(np.abs(p - ref.probs())) < 1e-5
    terms = random_pauli_sum(n, 8, seed=5)
    assert abs(sim.expect(terms) - ref.expect(terms)) < 1e-5 * sum(abs(c) for c, _ in terms)
    assert abs(sim.info()["discarded"] - ref.discarded) < 1e-5
