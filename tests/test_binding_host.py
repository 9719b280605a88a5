"""Host-side logic of the Python binding that needs no device: how `run_ops`
turns an op list into library calls (gate kinds, Kraus groups of M channels
per truncation), checked with a recording stand-in for the simulation handle."""
import numpy as np
import pytest

from workloads import grover, random_dense, random_layered


class Recorder:
    """Stands in for LRSim: records the calls run_ops makes."""

    def __init__(self):
        self.calls = []

    def apply_rotation(self, axis, q, theta, pid):
        self.calls.append(("rot", axis, q))

    def apply_gate(self, qubits, U, dU=None, param_id=-1):
        self.calls.append(("gate", tuple(qubits), np.asarray(U).shape))

    def apply_diagonal(self, qubits, d):
        self.calls.append(("diag", tuple(qubits), np.asarray(d).shape))

    def apply_channel(self, kind, q, p):
        self.calls.append(("chan", kind, q))

    def compress(self, r=0):
        self.calls.append(("compress", r))


@pytest.fixture(scope="module")
def run_ops():
    """sim.py's run_ops without the compiled library: the module's source runs with a
    stand-in for its library handles (run_ops only calls methods of the handle)."""
    import os
    import types
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "paper_2009_06657_gb300", "sim.py")).read()
    mod = types.ModuleType("_sim_for_test")
    fake_ffi = types.SimpleNamespace(LR_DEPOLARIZING=0, LR_AMPLITUDE_DAMPING=1, LR_BIT_FLIP=2)
    mod.__dict__.update({"_ffi": fake_ffi, "check": None, "lib": None})
    code = src.replace("from . import _ffi\nfrom ._ffi import check, lib\n", "")
    exec(compile(code, "sim.py", "exec"), mod.__dict__)
    return mod.run_ops


@pytest.mark.parametrize("M", [1, 2, 3])
def test_kraus_groups_truncate_after_every_mth_channel_and_at_the_end(run_ops, M):
    ops = random_layered(4, 2, seed=11, noise=("dep", 1e-3))
    rec = Recorder()
    run_ops(rec, ops, r=8, group=M)
    kinds = [c[0] for c in rec.calls]
    nch = kinds.count("chan")
    assert kinds.count("compress") == -(-nch // M)
    # every compress follows exactly M channels (the last one the remainder)
    since = 0
    for k in kinds:
        if k == "chan":
            since += 1
        elif k == "compress":
            assert since == M or (since == nch % M and since > 0)
            since = 0
    assert kinds[-1] == "compress"


def test_dense_and_diagonal_ops_map_to_their_calls(run_ops):
    ops, t = grover(5, iterates=1, p=1e-3, dense=True)
    rec = Recorder()
    run_ops(rec, ops, r=8)
    assert ("gate", (4, 3, 2, 1, 0), (32, 32)) in rec.calls
    ops2, _ = grover(5, iterates=1, p=1e-3, dense=False)
    rec2 = Recorder()
    run_ops(rec2, ops2, r=8)
    assert sum(1 for c in rec2.calls if c[0] == "diag") == 2
    assert all(c[2] == (32,) for c in rec2.calls if c[0] == "diag")
    ops3 = random_dense(6, 3, seed=5, k_range=(3, 4))
    rec3 = Recorder()
    run_ops(rec3, ops3, r=8)
    assert sum(1 for c in rec3.calls if c[0] == "gate") == 3


def test_unknown_op_is_rejected(run_ops):
    with pytest.raises(ValueError):
        run_ops(Recorder(), [{"op": "nope", "q": 0}])
