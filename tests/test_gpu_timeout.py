"""The bounded device-side wait and its failure path (LR_ETIMEOUT), without faulting
the GPU: a kernel waits on an mbarrier that nothing arrives on, with a short poll
limit, gives up, returns, and the host reads the timeout through the status word; a
simulation then runs normally on the same context."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lret as O  # noqa: E402
from workloads import random_layered  # noqa: E402


@pytest.fixture(scope="module")
def lr():
    import paper_2009_06657_gb300 as m
    return m


def test_bounded_wait_runs_out_and_reports_timeout(lr):
    import torch

    from paper_2009_06657_gb300._ffi import LR_ETIMEOUT, LR_OK, lib
    s = torch.cuda.Stream()
    sp = C.c_void_p(s.cuda_stream)
    assert lib.lr_selftest_wait(1 << 12, 0, sp) == LR_ETIMEOUT  # nothing arrives
    assert lib.lr_selftest_wait(1 << 24, 1, sp) == LR_OK        # another thread arrives
    assert lib.lr_selftest_wait(1 << 10, 0, None) == LR_ETIMEOUT  # legacy default stream
    # the context is intact: a truncated circuit still matches the oracle
    n, r = 5, 6
    ops = random_layered(n, 2, seed=77, noise=("mixed", 0.01, 0.02))
    sim = lr.LRSim(n, r, dtype="c128")
    lr.run_ops(sim, ops, r=r)
    p = sim.probs().cpu().numpy()
    assert np.sum(np.abs(p - O.run_lret(n, ops, r=r).probs())) < 1e-10
    assert sim.info()["converged"]
    sim.close()
