"""Register budget of the benchmark's hot kernels (CPU: nvcc cross-compiles for
sm_103a without a GPU). A spill in one of these kernels puts local-memory traffic
on the critical path of every truncation, so the build is checked for it: ptxas
must report zero spill stores for each kernel below (the batched cluster
eigensolver, which indexes its task list by blockIdx.y, at most 8 bytes: one or two
registers), and the cluster eigensolver must fit the 128 registers its 512-thread
launch allows."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2009_06657_gb300", "csrc")

# translation unit -> substrings of the mangled names of its hot instantiations
HOT = {
    "eigh_cluster.cu": ["k_eigh_clusterIfE", "k_eigh_cluster_batchIfE"],
    "gram_tc.cu": ["k_gram_pair_tc"],
    "proj_tc.cu": ["k_proj_pair_tc"],
    "readout.cu": ["k_pauli_expect_gIfLi2E"],
    "expand.cu": ["k_expandIfLi4E"],
    "gemm.cu": ["k_gram_reduce_herm_f32x4"],
    "eigh_refine.cu": ["k_rfILi", "k_rf_batchILi"],
}


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def _ptxas_report(tu, tmpdir):
    cmd = [_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-Xptxas", "-v", "-c", os.path.join(CSRC, tu), "-o", os.path.join(tmpdir, tu + ".o")]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    out, name = {}, None
    for line in p.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m:
            out.setdefault(name, {})["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            out.setdefault(name, {})["regs"] = int(m.group(1))
    return out


@pytest.mark.skipif(_nvcc() is None, reason="nvcc not available")
def test_hot_kernels_do_not_spill(tmp_path):
    with cf.ThreadPoolExecutor(max_workers=len(HOT)) as ex:
        reports = dict(zip(HOT, ex.map(lambda tu: _ptxas_report(tu, str(tmp_path)), HOT)))
    for tu, keys in HOT.items():
        for key in keys:
            hits = {n: r for n, r in reports[tu].items() if key in n}
            assert hits, f"{key} not found in {tu}"
            for n, r in hits.items():
                allowed = 8 if "k_eigh_cluster_batch" in n else 0
                assert r.get("spill", 0) <= allowed, f"{n} spills {r['spill']} bytes"
    eig = [r for n, r in reports["eigh_cluster.cu"].items() if "k_eigh_cluster" in n and "IfE" in n]
    assert len(eig) == 2 and all(r["regs"] <= 128 for r in eig)
