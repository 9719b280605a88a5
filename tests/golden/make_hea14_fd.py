"""Writes hea14_fd.json beside this script: the reference for the gradient test of the
14-qubit hardware-efficient ansatz (6 layers of Ry, Rz on every qubit and a CZ ladder,
168 parameters, depolarizing channels after every gate, r = 32, 50-term Pauli sum).

Every number comes from the oracle alone (oracle/lret.py, NumPy FP64): <H> through
Algorithm 1 and its central finite differences with h = 1e-4 at 16 parameter indices
drawn from a seeded generator. The per-qubit noise strengths are scaled by U(0.5, 1.5)
(identical channels on a near-product state make exactly tied cuts, where the
truncated state, and so its derivative, is not unique), and the first instance whose
cuts stay separated under the finite-difference steps is used: wherever the last kept
eigenvalue lambda_k is not negligible (above 1e-12 lambda_1), lambda_k - lambda_{k+1}
exceeds 1e-3 lambda_k, ten times what a step of h moves an eigenvalue by relative to
itself, so no cut changes order inside a stencil. Run from the repository root:
python tests/golden/make_hea14_fd.py [output path] (about half an hour of CPU time).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lret as O  # noqa: E402
from workloads import hea, random_pauli_sum  # noqa: E402

N, R, LAYERS, P, H = 14, 32, 6, 1e-3, 1e-4
GAP_MIN, ZERO_REL = 1e-3, 1e-12


def min_gap(st):
    """Smallest (lambda_k - lambda_{k+1}) / lambda_k over cuts with a non-negligible lambda_k."""
    g = [(e["lam"][e["k"] - 1] - e["lam"][e["k"]]) / e["lam"][e["k"] - 1] for e in st.log
         if e["k"] < e["m"] and e["lam"][e["k"] - 1] > ZERO_REL * e["lam"][0]]
    return min(g) if g else np.inf


def main():
    terms = random_pauli_sum(N, 50, seed=4001)
    for seed in range(4000, 4040):
        ops, th = hea(N, LAYERS, seed=seed, noise=("dep", P), qubit_jitter=(0.5, 1.5))
        st = O.run_lret(N, ops, r=R)
        gap = min_gap(st)
        print(f"seed {seed}: smallest cut gap relative to the cut eigenvalue {gap:.2e}", flush=True)
        if gap > GAP_MIN:
            break
    else:
        raise SystemExit("no instance with separated cuts")
    pids = sorted(int(i) for i in np.random.default_rng(seed + 2).choice(len(th), 16, replace=False))
    g = O.gradient_fd_lret(N, ops, th, terms, r=R, h=H, pids=pids)
    out = {"n": N, "r": R, "layers": LAYERS, "p": P, "seed": seed, "terms_seed": 4001, "h": H,
           "qubit_jitter": [0.5, 1.5], "min_gap": gap, "expect": st.expect(terms),
           "discarded": st.discarded, "pids": pids, "grad_fd": [float(g[i]) for i in pids]}
    path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(
        os.path.dirname(os.path.abspath(__file__)), "hea14_fd.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
