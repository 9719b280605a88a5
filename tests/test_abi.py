"""Host-side checks of the C ABI: the library loads, every declared symbol is
exported, and host-only helpers (Kraus presets, argument validation that needs
no device) behave."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lret.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\*?\s+\*?(lr_[a-z_0-9]+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    so = os.path.join(ROOT, "paper_2009_06657_gb300", "_lib", "liblret.so")
    if not os.path.exists(so):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2009_06657_gb300._ffi as f
    return f


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(lib.lib, name), name
    assert set(decl) == set(lib.exported_symbols())


def test_kraus_presets_match_oracle(lib):
    from oracle import lret as O
    from paper_2009_06657_gb300.sim import kraus_preset
    for kind, ref in (("dep", O.depolarizing), ("ad", O.amplitude_damping), ("bf", O.bit_flip)):
        for p in (0.0, 1e-3, 0.37, 1.0):
            buf, K = kraus_preset(kind, p)
            mats = buf[: 8 * K].view(np.complex128).reshape(K, 2, 2)
            want = np.stack(ref(p))
            assert mats.shape == want.shape
            assert np.max(np.abs(mats - want)) < 1e-15


def test_preset_rejects_bad_probability(lib):
    import ctypes as C
    out = np.zeros(32)
    K = C.c_int(0)
    st = lib.lib.lr_kraus_preset(0, 1.5, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(K))
    assert st == lib.LR_EINVAL
    st = lib.lib.lr_kraus_preset(7, 0.1, out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(K))
    assert st == lib.LR_EINVAL


def test_init_rejects_bad_sizes_without_device(lib):
    import ctypes as C
    h = C.c_void_p()
    assert lib.lib.lr_init(0, 4, 0, None, C.byref(h)) == lib.LR_EINVAL
    assert lib.lib.lr_init(31, 4, 0, None, C.byref(h)) == lib.LR_EINVAL
    assert lib.lib.lr_init(4, 0, 0, None, C.byref(h)) == lib.LR_EINVAL
    assert lib.lib.lr_init(4, 4, 5, None, C.byref(h)) == lib.LR_EINVAL


def test_pauli_masks_encoding():
    from paper_2009_06657_gb300.sim import pauli_masks
    xm, zm, cf = pauli_masks([(0.5, [(0, "X"), (2, "Y"), (3, "Z")])], 4)
    assert int(xm[0]) == 0b0101 and int(zm[0]) == 0b1100 and cf[0] == 0.5


def test_launch_counter_reads_without_device(lib):
    n = lib.lib.lr_launch_count()
    assert isinstance(n, int) and n >= 0
