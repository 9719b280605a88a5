"""Host-side accounting of bench.py (no GPU): the algorithmic work per launch that
the roofline divides by a kernel's time, the per-kernel rates, the peaks it is
compared against and the host-to-device bytes of the end-to-end figure. Expected
values are written out by hand from the workload's sizes (20 qubits, r = 64,
K = 4, complex64 state)."""
import json
import os

import pytest

import bench

N = 1 << 20
R = 64
ESZ = 8  # complex64


def test_algorithmic_work_per_launch():
    a = bench.algorithmic()
    # Gram of the row pairs: 2^19 rows x (128 x 128) complex MACs, half by symmetry
    assert a["gram"]["flop"] == pytest.approx(8 * 2**19 * 128 * 128 / 2)
    assert a["gram"]["bytes"] == N * R * ESZ == 536_870_912
    # projection on the row pairs: reads V, writes V_new
    assert a["project"]["flop"] == pytest.approx(8 * 2**19 * 128 * 128)
    assert a["project"]["bytes"] == 2 * 536_870_912
    # Householder reduction of the 256 x 256 matrix; reads the FP64 complex Gram
    assert a["eigh"]["flop"] == pytest.approx(16 / 3 * 256**3)
    assert a["eigh"]["bytes"] == 256 * 256 * 16
    # 64 Pauli terms, 4 per pass: 16 passes, each reading a row and its 4 partner rows
    assert a["pauli"]["bytes"] == 16 * 5 * 536_870_912


def test_kernel_rooflines_rates():
    peaks = {"hbm_gbs": 6000.0, "tf32_tflops": 900.0}
    kt = {"gram": (10.0, 40), "eigh": (60.0, 60), "pauli": (7.5, 1), "unknown": (1.0, 1), "readout": (0.0, 0)}
    out = bench.kernel_rooflines(kt, peaks)
    assert set(out) == {"gram", "eigh", "pauli"}  # no launches or no model: no row
    g = out["gram"]
    assert g["ms_per_launch"] == pytest.approx(0.25) and g["launches"] == 40
    assert g["hbm_gbs"] == pytest.approx(536_870_912 / 0.25e-3 / 1e9)
    assert g["hbm_frac"] == pytest.approx(g["hbm_gbs"] / 6000.0)
    assert g["tflops"] == pytest.approx(8 * 2**19 * 128 * 128 / 2 / 0.25e-3 / 1e12)
    # issued 3xTF32 work: three passes over the real view's upper triangle by 128-row blocks
    issued = 3 * 2 * 2**19 * (128 * 256 + 128 * 128)
    assert g["tensor_issued_tflops"] == pytest.approx(issued / 0.25e-3 / 1e12)
    assert g["tensor_issued_frac"] == pytest.approx(g["tensor_issued_tflops"] / 900.0)
    e = out["eigh"]
    assert e["tflops"] == pytest.approx(16 / 3 * 256**3 / 1e-3 / 1e12)  # 1 ms per solve: 0.0895 TFLOP/s
    assert "tflops" not in out["pauli"]


def test_peaks_come_from_the_measured_file():
    peaks = bench.load_peaks()
    assert peaks["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        assert peaks["hbm_gbs"] == d["hbm_gbs"]
        assert peaks["tf32_tflops"] == pytest.approx(d["bf16_tflops"] * 1.1 / 2.25)
        assert "measured" in peaks["source"]
    else:
        assert peaks["source"] == "fallback"


def test_host_to_device_bytes_per_step():
    ops = [{"op": "ry", "q": 0, "theta": 0.1, "pid": -1},
           {"op": "dep", "q": 0, "p": 5e-4},
           {"op": "cnot", "q": [0, 1]}]
    # angle and parameter id; four 2x2 complex128 Kraus matrices; a 4x4 complex128 gate and its qubits
    assert bench.h2d_bytes(ops) == 16 + 4 * 64 + (16 * 16 + 8)
