"""Adjoint gradients at the sizes of the differentiation workload.

* 14 qubits, r = 32, the hardware-efficient ansatz (6 layers of Ry, Rz on every qubit
  and a CZ ladder: 168 parameters), depolarizing after every gate, 50-term Pauli sum,
  checkpoint every 8 stages: d<H>/dtheta at 16 seeded parameters against central finite
  differences (h = 1e-4) of the oracle's Algorithm 1 in FP64, stored in
  tests/golden/hea14_fd.json by tests/golden/make_hea14_fd.py (oracle only).
* 6 qubits at full rank (r = 64 = 2^6, nothing discarded but zero eigenvalues): every
  parameter against the parameter-shift rule on exact density-matrix evolution (Eq. 1),
  computed here by the oracle.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lret as O  # noqa: E402
from workloads import hea, random_pauli_sum  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hea14_fd.json")


@pytest.fixture(scope="module")
def lr():
    import paper_2009_06657_gb300 as m
    return m


def _grad(lr, n, r, ops, th, terms, dtype, ckpt):
    import torch
    sim = lr.LRSim(n, r, dtype=dtype)
    t = torch.tensor(th, requires_grad=True)
    v = lr.LRExpectation.apply(t, sim, ops, terms, r, ckpt)
    v.backward()
    out = float(v.detach()), t.grad.numpy().copy()
    sim.close()
    return out


# Tolerances on d<H>/dtheta (|H| coefficients sum to about 40 here).
#  complex128: central differences with h = 1e-4 carry h^2 |f'''| / 6 (about 1e-8 |f'''|)
#    plus rounding of the two FP64 runs over 2h; the adjoint itself is FP64.
#  complex64: the forward state and the adjoint run in FP32 (FP64 sums and eigenproblem);
#    the gradient of a sum of 50 terms inherits the FP32 state error times sum |c_t|.
GRAD_TOL = {"c128": 1e-6, "c64": 2e-4}


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_hea14_gradient_matches_oracle_finite_differences(lr, dtype):
    ref = json.load(open(GOLDEN))
    n, r = ref["n"], ref["r"]
    ops, th = hea(n, ref["layers"], seed=ref["seed"], noise=("dep", ref["p"]),
                  qubit_jitter=tuple(ref["qubit_jitter"]))
    terms = random_pauli_sum(n, 50, seed=ref["terms_seed"])
    csum = sum(abs(c) for c, _ in terms)
    v, g = _grad(lr, n, r, ops, th, terms, dtype, 8)
    assert abs(v - ref["expect"]) < (1e-11 if dtype == "c128" else 1e-5) * csum
    err = np.abs(g[ref["pids"]] - np.array(ref["grad_fd"]))
    print(dtype, "max |adjoint - FD| over 16 parameters:", float(err.max()),
          "largest |dH/dtheta|:", float(np.abs(ref["grad_fd"]).max()))
    assert float(err.max()) < GRAD_TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_full_rank_gradient_matches_parameter_shift_on_exact_evolution(lr, dtype):
    """Every parameter of a 6-qubit, 6-layer ansatz at full rank (r = 64: every
    truncation drops only null directions of V'), against the parameter-shift rule on
    exact density-matrix evolution (Eq. 1). A depolarizing channel with p = 0.5 on every
    qubit first makes the state strongly mixed, so the smallest kept eigenvalue of every
    truncation stays above 1.5e-2 lambda_1 (the oracle's own run) and the FP64
    eigenvectors, hence the adjoint, are accurate to about u64 sum_cuts lambda_1 /
    lambda_k sum |c_t| = 5e-12. From a pure start the smallest kept eigenvalues at full
    rank reach 1e-13 lambda_1 and the adjoint inherits the eigenvectors' u64 lambda_1 /
    lambda_k error (measured 1e-6 in complex128)."""
    n = 6
    ops, th = hea(n, 6, seed=4100, noise=("dep", 1e-2))
    ops = [{"op": "dep", "q": q, "p": 0.5} for q in range(n)] + ops
    terms = random_pauli_sum(n, 20, seed=4101)
    _, g = _grad(lr, n, 2 ** n, ops, th, terms, dtype, 8)
    g_ps = O.gradient_param_shift_fdm(n, ops, th, terms)
    err = float(np.max(np.abs(g - g_ps)))
    print(dtype, "max |adjoint - parameter shift| over", len(th), "parameters:", err)
    # complex64: the FP32 state's error (the 1e-5 bound per expectation) times sum |c_t|
    assert err < (1e-10 if dtype == "c128" else 1e-4)
