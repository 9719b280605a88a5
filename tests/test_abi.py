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


def test_status_codes_match_header_and_have_messages(lib):
    """The binding's status constants are the header's, and every code (including
    the bounded-wait give-up, LR_ETIMEOUT) has its own message."""
    src = open(os.path.join(ROOT, "include", "lret.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (LR_E[A-Z]+)\s+(-?\d+)", src)}
    assert {"LR_EINVAL", "LR_EKRAUS", "LR_ECAPACITY", "LR_ETIMEOUT", "LR_ECUDA"} <= set(codes)
    msgs = set()
    for name, val in codes.items():
        assert getattr(lib, name) == val, name
        msg = lib.lib.lr_status_string(val).decode()
        assert msg and msg not in msgs, name
        msgs.add(msg)
    assert "timed out" in lib.lib.lr_status_string(codes["LR_ETIMEOUT"]).decode()


def test_pauli_mask_action_matches_kronecker_product():
    """The header's action of a Pauli string given by its masks,
    P|x> = i^{#Y} (-1)^{popcount(x & zmask)} |x ^ xmask>, against the dense
    Kronecker product of the single-qubit matrices (qubit q = bit q of x)."""
    import numpy as np

    from oracle import lret as O
    from paper_2009_06657_gb300.sim import pauli_masks
    from workloads import random_pauli_sum
    n = 4
    terms = random_pauli_sum(n, 12, seed=9) + [(1.0, [(1, "Y"), (3, "Y")]), (1.0, [(0, "Y"), (2, "Z")])]
    xm, zm, _ = pauli_masks(terms, n)
    for t, (_, string) in enumerate(terms):
        mats = [O.I2] * n
        for q, s in string:
            mats[q] = O.PAULI[s]
        dense = np.array([[1.0 + 0j]])
        for q in range(n - 1, -1, -1):
            dense = np.kron(dense, mats[q])
        ny = sum(1 for _, s in string if s == "Y")
        P = np.zeros((2 ** n, 2 ** n), dtype=complex)
        for x in range(2 ** n):
            sign = -1.0 if bin(x & int(zm[t])).count("1") % 2 else 1.0
            P[x ^ int(xm[t]), x] = (1j ** ny) * sign
        assert np.max(np.abs(P - dense)) < 1e-15


def test_package_import_fails_loudly_without_the_library(tmp_path):
    """A copy of the package without _lib/liblret.so must refuse to import:
    there is no CPU or pure-Python fallback."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_2009_06657_gb300")
    dst = tmp_path / "paper_2009_06657_gb300"
    dst.mkdir()
    for f in os.listdir(src):
        if f.endswith(".py"):
            shutil.copy(os.path.join(src, f), dst / f)
    p = subprocess.run([sys.executable, "-c", "import paper_2009_06657_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300,
                       env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert p.returncode != 0
    assert "ImportError" in p.stderr and "liblret.so" in p.stderr


def test_launch_counter_reads_without_device(lib):
    n = lib.lib.lr_launch_count()
    assert isinstance(n, int) and n >= 0


def test_batch_options_struct_matches_the_header(lib):
    """lr_batch_opts_default (host only) fills the caller's struct: every field the
    Python mirror declares holds the header's default, and nothing past the mirror's
    size is written (a field added to one side only would show here)."""
    import ctypes as C
    f = lib
    size = C.sizeof(f.lr_batch_opts)
    buf = (C.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    f.lib.lr_batch_opts_default(C.cast(buf, C.POINTER(f.lr_batch_opts)))
    o = f.lr_batch_opts.from_buffer(buf)
    assert o.dtype == f.LR_C64 and o.eig_precision == f.LR_EIGP_REFINED and o.eig_iters == 1
    assert o.rows_per_split == 0 and not o.splits and o.use_graph == 1 and not o.stream
    assert o.tensor_cores == 1 and o.cluster_min_m == 256
    assert all(b == 0xAB for b in buf[size:])
