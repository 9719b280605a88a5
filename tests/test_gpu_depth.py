"""The 12-qubit workload at its full depth: 100 layers of the random Ry/Rz + CNOT
family, after every gate either a depolarizing channel (p = 1e-3) or amplitude
damping (gamma = 2e-3) chosen per gate by the seed, r = 32, complex64 and complex128
states against the FP64 oracle stepped layer by layer beside them.

Every 10 layers: the L1 error of Prob(x) (Eq. 9), the error of <H> for a 16-term
Pauli sum and of <Z_q>, the error of the discarded mass and the trace distance of
rho (Eq. 10's T on the full state), for both precisions. Bars: complex64 1e-5,
complex128 1e-11, on every one of them. The circuit's per-gate channels are
identical on every qubit (no noise jitter) and the seed is the workload's own.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lret as O  # noqa: E402
from workloads import random_layered, random_pauli_sum  # noqa: E402

N, R, DEPTH, SEED = 12, 32, 100, 2000
TOL = {"c64": 1e-5, "c128": 1e-11}


@pytest.fixture(scope="module")
def lr():
    import paper_2009_06657_gb300 as m
    return m


def test_full_depth_error_curve(lr):
    ops = random_layered(N, DEPTH, seed=SEED, noise=("mixed", 1e-3, 2e-3))
    per = len(ops) // DEPTH
    terms = random_pauli_sum(N, 16, seed=SEED + 7)
    csum = sum(abs(c) for c, _ in terms)
    st = O.LRETState(N)
    sims = {d: lr.LRSim(N, R, dtype=d) for d in ("c64", "c128")}
    rows = []
    for L in range(DEPTH):
        layer = ops[L * per:(L + 1) * per]
        for o in layer:
            if O.is_gate(o):
                qs, U = O.gate_matrix(o)
                st.gate(qs, U)
            else:
                st.channel(o["q"], O.channel_kraus(o))
                st.compress(r=R)
        for sim in sims.values():
            lr.run_ops(sim, layer, r=R)
        if (L + 1) % 10:
            continue
        pref, href, zref = st.probs(), st.expect(terms), st.z_expect()
        row = {"layer": L + 1, "discarded": st.discarded}
        for d, sim in sims.items():
            p = sim.probs().double().cpu().numpy()
            z, _ = sim.z_expect()
            row[f"l1_{d}"] = float(np.abs(p - pref).sum())
            row[f"h_{d}"] = abs(sim.expect(terms) - href) / csum
            row[f"z_{d}"] = float(np.max(np.abs(z - zref)))
            row[f"td_{d}"] = O.trace_distance_lowrank(sim.state().astype(np.complex128), st.L)
            row[f"disc_{d}"] = abs(sim.info()["discarded"] - st.discarded)
        rows.append(row)
        print(json.dumps(row), flush=True)
    out = os.environ.get("LRET_CURVE_OUT")
    if out:
        with open(out, "w") as f:
            json.dump(rows, f, indent=1)
    for sim in sims.values():
        sim.close()
    assert len(rows) == DEPTH // 10 and len(st.log) > 1000
    for row in rows:
        for d in ("c64", "c128"):
            for key in ("l1", "h", "z", "disc", "td"):
                assert row[f"{key}_{d}"] < TOL[d], (row["layer"], key, d, row)
