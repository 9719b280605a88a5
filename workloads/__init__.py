"""Seeded synthetic workloads shared by the oracle and the CUDA path.

This module holds no arithmetic of the low-rank method. It only draws random
numbers (NumPy PCG64 via ``default_rng``) and writes them into plain op lists:
gate names, qubit indices, angles, channel names and strengths, and Pauli
strings with coefficients. Each consumer turns these descriptions into
matrices with its own code.

Op list format (a list of dicts, applied in order):

* ``{"op": "ry"|"rz"|"rx", "q": int, "theta": float, "pid": int}`` -- a
  one-qubit rotation; ``pid`` is the parameter index (``-1`` = fixed).
* ``{"op": "cnot", "q": [control, target]}`` and ``{"op": "cz", "q": [a, b]}``.
* ``{"op": "dep", "q": int, "p": float}`` -- one-qubit depolarizing channel.
* ``{"op": "ad", "q": int, "gamma": float}`` -- one-qubit amplitude damping.
* ``{"op": "bf", "q": int, "p": float}`` -- one-qubit bit flip.
* ``{"op": "h", "q": int}`` and the other fixed one-qubit gates x, y, z, s, t.
* ``{"op": "unitary", "q": [q_0, ..., q_{k-1}], "U": (2^k, 2^k) complex array}``
  -- a dense k-qubit gate, row/column index sum_i b(q_i) 2^(k-1-i).
* ``{"op": "diag", "q": [q_0, ..., q_{k-1}], "d": (2^k,) complex array}`` -- a
  diagonal k-qubit gate, entries in the same index order.

Qubit ``q`` is bit ``q`` of the computational-basis index (little-endian).
Channels follow the gate they decorate; the low-rank runners truncate after
every channel (one-qubit Kraus groups, Sec. II.C with M = 1).

Workload families (Sec. III.A uses random layered circuits; the sizes below
are those of the five benchmark configurations):

* ``random_layered``: per layer, Ry then Rz on every qubit (angles U[0, 2pi)),
  then CNOTs on a seeded random perfect matching (first of each pair is the
  control; with odd n one qubit idles). A channel follows every gate on every
  qubit that gate touches.
* ``hea``: hardware-efficient ansatz, per layer Ry and Rz on every qubit
  (angles N(0, 0.5^2), all differentiable) then a CZ ladder CZ(0,1)...CZ(n-2,n-1).
* ``random_pauli_sum``: T terms, weight U{1..min(4, n)}, distinct qubits,
  uniform X/Y/Z, coefficients N(0, 1).
* ``grover``: amplitude amplification of the basis states of Hamming weight
  <= 2 (Sec. III.D), each Grover iterate one dense n-qubit unitary or a
  diagonal oracle plus a diffuser; depolarizing noise on every qubit after the
  initial Hadamards and after every iterate. The iterate's entries are the
  circuit's definition (a sign per basis state, and the reflection about the
  uniform superposition), written out here as plain arrays.
* ``random_dense``: layers of seeded Haar-random dense k-qubit gates on random
  qubit subsets, each followed by channels on the qubits it touches.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "random_layered",
    "hea",
    "random_rb",
    "random_pauli_sum",
    "grover",
    "grover_good",
    "random_dense",
    "count_ops",
    "CONFIGS",
]


def _channel(rng, q, noise, scale=None):
    """Return the channel op for qubit q under a noise spec.

    noise: ("dep", p) | ("ad", gamma) | ("bf", p) | ("mixed", p_dep, gamma_ad)
    For "mixed", one seeded coin per gate picks the kind (drawn by the caller).
    scale: optional per-qubit multipliers of the strength.
    """
    kind = noise[0]
    f = 1.0 if scale is None else float(scale[q])
    if kind == "dep":
        return {"op": "dep", "q": int(q), "p": float(noise[1]) * f}
    if kind == "ad":
        return {"op": "ad", "q": int(q), "gamma": float(noise[1]) * f}
    if kind == "bf":
        return {"op": "bf", "q": int(q), "p": float(noise[1]) * f}
    raise ValueError(f"unknown noise kind {kind!r}")


def _noise_for_gate(rng, noise):
    if noise is None:
        return None
    if noise[0] == "mixed":
        return ("dep", noise[1]) if rng.random() < 0.5 else ("ad", noise[2])
    return noise


def random_layered(n, depth, seed, noise=("dep", 1e-3), two_qubit="cnot",
                   param_ids=False, qubit_jitter=None):
    """Seeded random layered circuit (Ry, Rz on every qubit, then a matching).

    qubit_jitter=(lo, hi) multiplies each qubit's channel strength by a seeded
    U(lo, hi) factor. With identical channels on every qubit a near-product
    state has exactly degenerate eigenvalues, so a rank cut can fall inside a
    tie (several equally correct truncations); distinct strengths remove that.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    scale = None
    if qubit_jitter is not None:
        scale = np.random.default_rng(seed + 7919).uniform(qubit_jitter[0], qubit_jitter[1], size=n)
    ops = []
    pid = 0
    for _ in range(depth):
        for q in range(n):
            for name in ("ry", "rz"):
                theta = float(rng.uniform(0.0, 2.0 * np.pi))
                ops.append({"op": name, "q": q, "theta": theta,
                            "pid": pid if param_ids else -1})
                if param_ids:
                    pid += 1
                nz = _noise_for_gate(rng, noise)
                if nz is not None:
                    ops.append(_channel(rng, q, nz, scale))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            a, b = int(perm[i]), int(perm[i + 1])
            ops.append({"op": two_qubit, "q": [a, b]})
            nz = _noise_for_gate(rng, noise)
            if nz is not None:
                ops.append(_channel(rng, a, nz, scale))
                ops.append(_channel(rng, b, nz, scale))
    return ops


RB_ONE_QUBIT = ("x", "y", "z", "s", "t", "rx", "ry", "rz")
RB_TWO_QUBIT = ("swap", "cz", "cnot")


def random_rb(n, depth, seed, noise=("dep", 1e-3), qubit_jitter=None):
    """Seeded dense random circuit over the randomized-benchmarking gate set
    (X, Y, Z, S, T, RX, RY, RZ, SWAP, CZ, CNOT): in every layer, walking up the
    qubits, a two-qubit gate on the adjacent pair (q, q+1) or a one-qubit gate
    on q, each with probability 1/2 (rotation angles U[0, 2 pi)); a channel
    follows every gate on each qubit it touches. noise as for random_layered,
    plus ("mixed3", p_dep, gamma_ad, p_bf) drawing one of the three kinds per gate.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    scale = None
    if qubit_jitter is not None:
        scale = np.random.default_rng(seed + 7919).uniform(qubit_jitter[0], qubit_jitter[1], size=n)

    def nz_for_gate():
        if noise is None:
            return None
        if noise[0] == "mixed3":
            k = int(rng.integers(3))
            return (("dep", noise[1]), ("ad", noise[2]), ("bf", noise[3]))[k]
        return _noise_for_gate(rng, noise)

    ops = []
    for _ in range(depth):
        q = 0
        while q < n:
            if q + 1 < n and rng.random() < 0.5:
                name = RB_TWO_QUBIT[int(rng.integers(len(RB_TWO_QUBIT)))]
                ops.append({"op": name, "q": [q, q + 1]})
                nz = nz_for_gate()
                if nz is not None:
                    ops.append(_channel(rng, q, nz, scale))
                    ops.append(_channel(rng, q + 1, nz, scale))
                q += 2
            else:
                name = RB_ONE_QUBIT[int(rng.integers(len(RB_ONE_QUBIT)))]
                op = {"op": name, "q": q}
                if name.startswith("r"):
                    op["theta"] = float(rng.uniform(0.0, 2.0 * np.pi))
                    op["pid"] = -1
                ops.append(op)
                nz = nz_for_gate()
                if nz is not None:
                    ops.append(_channel(rng, q, nz, scale))
                q += 1
    return ops


def hea(n, layers, seed, noise=("dep", 1e-3), theta_std=0.5, qubit_jitter=None):
    """Hardware-efficient ansatz: (Ry, Rz on every qubit, CZ ladder) x layers.

    Every rotation is differentiable; parameter ids run 0..2*n*layers-1 in op
    order. Returns (ops, theta) where theta is the initial parameter vector.
    """
    rng = np.random.default_rng(seed)
    scale = None
    if qubit_jitter is not None:
        scale = np.random.default_rng(seed + 7919).uniform(qubit_jitter[0], qubit_jitter[1], size=n)
    ops = []
    thetas = []
    for _ in range(layers):
        for name in ("ry", "rz"):
            for q in range(n):
                th = float(rng.normal(0.0, theta_std))
                ops.append({"op": name, "q": q, "theta": th, "pid": len(thetas)})
                thetas.append(th)
                nz = _noise_for_gate(rng, noise)
                if nz is not None:
                    ops.append(_channel(rng, q, nz, scale))
        for q in range(n - 1):
            ops.append({"op": "cz", "q": [q, q + 1]})
            nz = _noise_for_gate(rng, noise)
            if nz is not None:
                ops.append(_channel(rng, q, nz, scale))
                ops.append(_channel(rng, q + 1, nz, scale))
    return ops, np.asarray(thetas, dtype=np.float64)


def grover_good(n, max_weight=2):
    """Boolean mask over the 2^n basis states: Hamming weight <= max_weight."""
    x = np.arange(2 ** n, dtype=np.int64)
    hw = np.zeros(2 ** n, dtype=np.int64)
    for q in range(n):
        hw += (x >> q) & 1
    return hw <= max_weight


def grover(n, iterates=None, p=1e-3, dense=True, max_weight=2, qubit_jitter=None, seed=0):
    """Amplitude amplification of {x : HW(x) <= max_weight} on n qubits.

    Ops: H on every qubit, then `iterates` Grover iterates (default
    floor(pi/4 sqrt(1/p_good))). dense=True writes each iterate as one
    n-qubit "unitary" op on qubits [n-1, ..., 0] (so its index is the basis
    index x); dense=False writes it as a "diag" sign oracle, H on every qubit, a
    "diag" reflection about |0...0> (+1 at x = 0, -1 elsewhere) and H on every
    qubit again. p > 0 puts a depolarizing channel of strength p on every
    qubit after the Hadamards and after each iterate; qubit_jitter = (lo, hi)
    scales qubit q's strength by a seeded U[lo, hi) factor.
    Returns (ops, iterates).
    """
    good = grover_good(n, max_weight)
    N = 2 ** n
    if iterates is None:
        iterates = int(np.floor(np.pi / 4.0 * np.sqrt(N / good.sum())))
    sign = np.where(good, -1.0, 1.0).astype(np.complex128)
    allq = list(range(n - 1, -1, -1))
    ops = []

    scale = np.ones(n)
    if qubit_jitter is not None:
        scale = np.random.default_rng(seed + 7919).uniform(qubit_jitter[0], qubit_jitter[1], size=n)

    def noise():
        if p > 0:
            for q in range(n):
                ops.append({"op": "dep", "q": q, "p": float(p * scale[q])})

    for q in range(n):
        ops.append({"op": "h", "q": q})
    noise()
    if dense:
        # (2|s><s| - I) O with |s> the uniform superposition, O = diag(sign)
        U = (np.full((N, N), 2.0 / N, dtype=np.complex128) - np.eye(N, dtype=np.complex128)) * sign[None, :]
    refl0 = -np.ones(N, dtype=np.complex128)
    refl0[0] = 1.0
    for _ in range(iterates):
        if dense:
            ops.append({"op": "unitary", "q": allq, "U": U})
        else:
            ops.append({"op": "diag", "q": allq, "d": sign})
            for q in range(n):
                ops.append({"op": "h", "q": q})
            ops.append({"op": "diag", "q": allq, "d": refl0})
            for q in range(n):
                ops.append({"op": "h", "q": q})
        noise()
    return ops, iterates


def _haar_unitary(rng, d):
    """Haar-random d x d unitary: QR of a complex Gaussian, phases fixed."""
    Z = (rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    ph = np.diag(R) / np.abs(np.diag(R))
    return Q * ph[None, :]


def random_dense(n, layers, seed, k_range=(3, 5), noise=("dep", 1e-3)):
    """Per layer one dense k-qubit gate (k uniform in k_range, distinct random
    qubits in random order, Haar-random matrix), then a channel on each of its
    qubits."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(layers):
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        k = min(k, n)
        qs = [int(q) for q in rng.choice(n, size=k, replace=False)]
        ops.append({"op": "unitary", "q": qs, "U": _haar_unitary(rng, 2 ** k)})
        if noise is not None:
            for q in qs:
                ops.append(_channel(rng, q, _noise_for_gate(rng, noise)))
    return ops


def random_pauli_sum(n, T, seed, max_weight=4):
    """T random Pauli strings: list of (coeff, [(qubit, 'X'|'Y'|'Z'), ...])."""
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(T):
        w = int(rng.integers(1, min(max_weight, n) + 1))
        qs = rng.choice(n, size=w, replace=False)
        letters = rng.integers(0, 3, size=w)
        c = float(rng.normal())
        terms.append((c, [(int(q), "XYZ"[int(l)]) for q, l in zip(qs, letters)]))
    return terms


def count_ops(ops):
    """(gates, channels) in an op list."""
    g = sum(1 for o in ops if o["op"] not in ("dep", "ad", "bf"))
    c = sum(1 for o in ops if o["op"] in ("dep", "ad", "bf"))
    return g, c


# The five benchmark workloads (sizes and laws of the paper-style random
# circuits; seeds are 1000 * config_id + instance).
CONFIGS = {
    "c1_6q_r13": dict(n=6, r=13, depth=40, noise=("dep", 0.0033), seed=1000),
    "c2_12q_r32": dict(n=12, r=32, depth=100, noise=("mixed", 1e-3, 2e-3), seed=2000),
    "c3_20q_r64": dict(n=20, r=64, depth=200, noise=("dep", 5e-4), seed=3000),
    "c4_14q_hea": dict(n=14, r=32, layers=6, noise=("dep", 1e-3), seed=4000,
                       terms=50, ckpt_every=8),
    "c5_batch256": dict(count=256, n_range=(8, 18), ranks=(8, 16, 32, 64),
                        depth_range=(40, 200), noise=("mixed", 1e-3, 2e-3), seed=5000),
}


def batch_circuits(count=256, n_range=(8, 18), ranks=(8, 16, 32, 64),
                   depth_range=(40, 200), noise=("mixed", 1e-3, 2e-3), seed=5000,
                   depth_scale=1.0):
    """Seeded heterogeneous batch: list of dicts {n, r, depth, ops}.

    depth_scale < 1 shrinks every depth (for quick tests); the draws are the
    same for every scale so a scaled batch is a prefix-faithful miniature.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        r = int(rng.choice(ranks))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        d = max(1, int(round(depth * depth_scale)))
        ops = random_layered(n, d, seed + 1 + i, noise=noise)
        out.append({"n": n, "r": r, "depth": d, "ops": ops})
    return out
