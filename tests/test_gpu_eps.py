"""The threshold rule and the rank history (Sec. II.B-C) on the GPU.

* The per-truncation log (lr_set_trunc_log) against the oracle's record of the same
  truncations: columns before and after, lambda_1, lambda_k, lambda_{k+1}, discarded
  mass and gap, with the intermediate rank of Eq. 8 derived from it.
* The eps rule at the paper's eps / p = 0.1 setting (p = 1e-3, eps = 1e-4): the kept
  counts equal the oracle's at every truncation, and the distortion of Eq. 10 of the
  GPU's Prob(x) (against exact density-matrix evolution, Eq. 1, and the noiseless
  statevector) equals the oracle's LRET distortion.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lret as O  # noqa: E402
from workloads import random_layered, random_pauli_sum  # noqa: E402

TOL = {"c128": 1e-11, "c64": 1e-5}


@pytest.fixture(scope="module")
def lr():
    import paper_2009_06657_gb300 as m
    return m


def _oracle_cuts(st):
    # the library skips truncations that drop nothing (m <= r); the oracle logs them too
    return [e for e in st.log if e["k"] < e["m"]]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_truncation_log_matches_oracle(lr, dtype):
    n, r = 8, 12
    ops = random_layered(n, 2, seed=1500, noise=("mixed", 1e-2, 2e-2), qubit_jitter=(0.5, 1.5))
    ref = O.run_lret(n, ops, r=r)
    sim = lr.LRSim(n, r, dtype=dtype)
    sim.set_trunc_log(4096)
    lr.run_ops(sim, ops, r=r)
    log = sim.trunc_log()
    cuts = _oracle_cuts(ref)
    assert len(log) == len(cuts) > 10
    tol = TOL[dtype]
    for g, e in zip(log, cuts):
        lam = e["lam"]
        assert (g["m"], g["k"]) == (e["m"], e["k"])
        assert abs(g["lambda_1"] - lam[0]) < tol
        assert abs(g["discarded"] - e["dropped"]) < tol
        assert abs(g["trace"] - float(np.sum(lam))) < tol
        if dtype == "c128":
            assert abs(g["lambda_k"] - lam[e["k"] - 1]) < tol and abs(g["lambda_k1"] - lam[e["k"]]) < tol
            assert abs(g["gap"] - e["gap"]) < 1e-9
        # Eq. 8: V_I^3 = N (4^M V)^3 / M with M = 1 and 4^M V = m
        assert abs(g["V_I"] ** 3 - n * g["m"] ** 3) < 1e-9 * g["V_I"] ** 3
    assert abs(sum(g["discarded"] for g in log) - sim.info()["discarded"]) < tol
    sim.reset()
    assert sim.trunc_log() == []
    sim.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_eps_rule_kept_counts_and_distortion_match_oracle(lr, dtype):
    n, p, eps = 10, 1e-3, 1e-4
    ops = random_layered(n, 4, seed=1600, noise=("dep", p), qubit_jitter=(0.5, 1.5))
    ref = O.run_lret(n, ops, eps=eps)
    sim = lr.LRSim(n, 64, dtype=dtype)
    sim.set_eps(eps)
    sim.set_trunc_log(8192)
    lr.run_ops(sim, ops, r=0)
    ks = [g["k"] for g in sim.trunc_log()]
    assert ks == [e["k"] for e in _oracle_cuts(ref)]
    p_gpu = sim.probs().double().cpu().numpy()
    tol = TOL[dtype]
    assert np.sum(np.abs(p_gpu - ref.probs())) < tol
    exact = O.run_fdm(n, ops).probs()
    noiseless = O.run_sv(n, ops).probs()
    d_gpu = O.distortion(p_gpu, exact, noiseless)
    d_ref = O.distortion(ref.probs(), exact, noiseless)
    print(dtype, "Eq. 10 distortion at eps/p = 0.1:", d_gpu, "(oracle", d_ref, "), final rank", ks[-1])
    # |D_gpu - D_ref| <= T(p_gpu, p_ref) / T(exact, noiseless)
    assert abs(d_gpu - d_ref) <= tol / O.variational_distance(exact, noiseless)
    sim.close()
