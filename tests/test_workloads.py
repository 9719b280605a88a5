"""The synthetic input recipes (CPU): the generators produce the shapes, counts and
distributions the benchmark and the parity tests are stated on, deterministically
from their seeds."""
import numpy as np
import pytest

from workloads import count_ops, hea, random_layered, random_pauli_sum


def test_benchmark_layer_counts_and_order():
    """20 qubits, one layer: Ry, channel, Rz, channel on every qubit, then 10 CNOTs on a
    perfect matching, each followed by a channel on both of its qubits: 50 gates,
    60 channels (one truncation each)."""
    n = 20
    ops = random_layered(n, 1, seed=3000, noise=("dep", 5e-4))
    gates = [o for o in ops if o["op"] in ("ry", "rz", "cnot")]
    chans = [o for o in ops if o["op"] == "dep"]
    assert len(gates) == 50 and len(chans) == 60 and len(ops) == 110
    assert count_ops(ops) == (50, 60)
    assert all(o["p"] == 5e-4 for o in chans)
    # one-qubit part: per qubit Ry, dep, Rz, dep on that qubit
    for q in range(n):
        blk = ops[4 * q:4 * q + 4]
        assert [o["op"] for o in blk] == ["ry", "dep", "rz", "dep"]
        assert all(o["q"] == q for o in blk)
        assert all(0.0 <= o["theta"] < 2 * np.pi for o in (blk[0], blk[2]))
    # two-qubit part: a perfect matching, each CNOT followed by channels on its qubits
    tail = ops[4 * n:]
    touched = []
    for i in range(0, len(tail), 3):
        g, c1, c2 = tail[i:i + 3]
        assert g["op"] == "cnot" and g["q"][0] != g["q"][1]
        assert (c1["q"], c2["q"]) == (g["q"][0], g["q"][1])
        touched += g["q"]
    assert sorted(touched) == list(range(n))


def test_mixed_noise_draws_both_kinds_per_gate():
    ops = random_layered(12, 4, seed=2000, noise=("mixed", 1e-3, 2e-3))
    kinds = [o["op"] for o in ops if o["op"] in ("dep", "ad")]
    assert 0.3 < kinds.count("dep") / len(kinds) < 0.7
    assert all(o["p"] == 1e-3 for o in ops if o["op"] == "dep")
    assert all(o["gamma"] == 2e-3 for o in ops if o["op"] == "ad")
    # the two channels after a CNOT share one coin
    for i, o in enumerate(ops):
        if o["op"] == "cnot":
            assert ops[i + 1]["op"] == ops[i + 2]["op"]


def test_qubit_jitter_scales_each_qubit_within_bounds():
    ops = random_layered(6, 2, seed=5, noise=("dep", 1e-2), qubit_jitter=(0.5, 1.5))
    per_q = {}
    for o in ops:
        if o["op"] == "dep":
            per_q.setdefault(o["q"], set()).add(round(o["p"], 15))
    assert all(len(v) == 1 for v in per_q.values())  # one strength per qubit
    vals = [next(iter(v)) for v in per_q.values()]
    assert all(0.5e-2 <= v <= 1.5e-2 for v in vals) and len(set(vals)) == 6


def test_pauli_sum_law():
    n, T = 20, 4000
    terms = random_pauli_sum(n, T, seed=3001)
    w = np.array([len(s) for _, s in terms])
    assert w.min() == 1 and w.max() == 4
    assert all(abs(np.mean(w == k) - 0.25) < 0.03 for k in (1, 2, 3, 4))
    for _, s in terms:
        qs = [q for q, _ in s]
        assert len(set(qs)) == len(qs) and all(0 <= q < n for q in qs)
        assert all(l in "XYZ" for _, l in s)
    letters = [l for _, s in terms for _, l in s]
    assert all(abs(letters.count(l) / len(letters) - 1 / 3) < 0.03 for l in "XYZ")
    c = np.array([c for c, _ in terms])
    assert abs(c.mean()) < 0.06 and 0.95 < c.std() < 1.05


def test_hea_gradient_workload_shape():
    """14 qubits, 6 layers: 168 differentiable rotations (ids 0..167 in op order,
    N(0, 0.5^2) angles), a 13-CZ ladder per layer, a channel on every touched qubit."""
    ops, theta = hea(14, 6, seed=4000, noise=("dep", 1e-3))
    rot = [o for o in ops if o["op"] in ("ry", "rz")]
    assert len(rot) == 168 and [o["pid"] for o in rot] == list(range(168))
    assert np.array_equal(theta, [o["theta"] for o in rot])
    assert 0.3 < theta.std() < 0.7
    assert sum(1 for o in ops if o["op"] == "cz") == 6 * 13
    assert sum(1 for o in ops if o["op"] == "dep") == 168 + 2 * 6 * 13


@pytest.mark.parametrize("gen", ["layered", "pauli", "hea"])
def test_generators_are_deterministic_in_their_seed(gen):
    if gen == "layered":
        a, b, c = (random_layered(8, 3, seed=s, noise=("mixed", 1e-3, 2e-3)) for s in (7, 7, 8))
    elif gen == "pauli":
        a, b, c = (random_pauli_sum(8, 30, seed=s) for s in (7, 7, 8))
    else:
        a, b, c = (hea(8, 2, seed=s)[0] for s in (7, 7, 8))
    assert a == b and a != c


def test_batch_recipe_ranges_and_miniature():
    """256 circuits: n in 8..18, r in {8, 16, 32, 64}, depth in 40..200; a scaled
    batch draws the same n, r and depths (scaled), so it is a miniature of the full one."""
    from workloads import batch_circuits
    full = batch_circuits(count=256, depth_scale=1.0)
    assert len(full) == 256
    ns = [c["n"] for c in full]
    assert min(ns) == 8 and max(ns) == 18
    assert {c["r"] for c in full} == {8, 16, 32, 64}
    assert all(40 <= c["depth"] <= 200 for c in full)
    mini = batch_circuits(count=256, depth_scale=0.05)
    for a, b in zip(full, mini):
        assert (a["n"], a["r"]) == (b["n"], b["r"])
        assert b["depth"] == max(1, int(round(a["depth"] * 0.05)))
