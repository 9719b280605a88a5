"""The allocation-free expectation entry point, lr_expect_static.

It serves callers that cannot allocate device memory when they read out: a
server that reserved all device memory for its own pool, or a thread that must
not take the device-wide synchronisation of cudaMalloc/cudaFree. Its scratch is a fixed
device array inside the library. This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-11, "c64": 1e-5}


def _static_expect(lib, V, n, dtype_code, xm, zm, cf, stream):
    out = C.c_double(0.0)
    st = lib.lr_expect_static(C.c_void_p(V.data_ptr()), n, V.shape[1], V.shape[1], dtype_code, len(cf),
                              xm.ctypes.data_as(C.POINTER(C.c_uint64)), zm.ctypes.data_as(C.POINTER(C.c_uint64)),
                              cf.ctypes.data_as(C.POINTER(C.c_double)), C.byref(out), C.c_void_p(stream))
    return st, out.value


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_static_expectation_matches_handle_on_two_calls(dtype):
    import torch

    import paper_2009_06657_gb300 as lr
    from paper_2009_06657_gb300._ffi import LR_C64, LR_C128, LR_OK, lib
    from workloads import random_layered, random_pauli_sum

    n, r = 9, 12
    sim = lr.LRSim(n, r, dtype=dtype)
    lr.run_ops(sim, random_layered(n, 2, seed=6100, noise=("mixed", 1e-2, 2e-2)), r=r)
    V = torch.from_numpy(sim.state()).cuda()  # caller-owned device state, leading dimension = columns
    code = LR_C64 if dtype == "c64" else LR_C128
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different term sets: the shared scratch keeps the
    # first call's contents, which the second must not depend on
    for seed, T in ((6101, 40), (6102, 17)):
        terms = random_pauli_sum(n, T, seed=seed)
        want = sim.expect(terms)
        xm, zm, cf = lr.pauli_masks(terms, n)
        st, got = _static_expect(lib, V, n, code, xm, zm, cf, stream)
        assert st == LR_OK
        assert abs(got - want) < TOL[dtype]
    sim.close()


def test_static_expectation_rejects_too_many_terms():
    import torch

    import paper_2009_06657_gb300 as lr
    from paper_2009_06657_gb300._ffi import LR_C64, LR_ECAPACITY, LR_STATIC_MAX_TERMS, lib
    from workloads import random_pauli_sum

    n = 4
    V = torch.zeros((1 << n, 2), dtype=torch.complex64, device="cuda")
    terms = random_pauli_sum(n, LR_STATIC_MAX_TERMS + 1, seed=6103)
    xm, zm, cf = lr.pauli_masks(terms, n)
    st, _ = _static_expect(lib, V, n, LR_C64, xm, zm, cf, torch.cuda.current_stream().cuda_stream)
    assert st == LR_ECAPACITY
