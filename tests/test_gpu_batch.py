"""Batched execution (many circuits of uneven n, r and depth in one CUDA graph)
against one-at-a-time runs of the same circuits and against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import lret as O  # noqa: E402
from workloads import batch_circuits, random_layered  # noqa: E402


@pytest.fixture(scope="module")
def lr():
    import paper_2009_06657_gb300 as m
    return m


def _small_batch():
    out = []
    specs = [(3, 2, 2), (5, 4, 2), (7, 8, 1), (4, 2, 3), (6, 16, 1), (8, 4, 1)]
    for i, (n, r, d) in enumerate(specs):
        out.append({"n": n, "r": r, "ops": random_layered(n, d, seed=5100 + i, noise=("mixed", 2e-2, 4e-2),
                                                           qubit_jitter=(0.5, 1.5))})
    return out


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_batch_matches_single_runs(lr, dtype):
    circs = _small_batch()
    b = lr.LRBatch(circs, dtype=dtype)
    b.run()
    tol = 1e-11 if dtype == "c128" else 1e-5
    for i, cd in enumerate(circs):
        sim = lr.LRSim(cd["n"], cd["r"], dtype=dtype)
        sim.set_eigensolver("tridiag")
        lr.run_ops(sim, cd["ops"], r=cd["r"])
        p1 = sim.probs().double().cpu().numpy()
        pb = b.probs(i).double().cpu().numpy()
        assert np.sum(np.abs(p1 - pb)) < tol, i
        assert abs(b.info(i)["discarded"] - sim.info()["discarded"]) < tol
        sim.close()
    b.close()


def test_batch_matches_oracle_fp64(lr):
    circs = _small_batch()
    b = lr.LRBatch(circs, dtype="c128")
    b.run()
    for i, cd in enumerate(circs):
        ref = O.run_lret(cd["n"], cd["ops"], r=cd["r"])
        pb = b.probs(i).cpu().numpy()
        assert np.sum(np.abs(pb - ref.probs())) < 1e-10, i
        assert abs(b.info(i)["discarded"] - ref.discarded) < 1e-10
    b.close()


def test_graph_and_direct_launches_agree_and_rerun_is_reproducible(lr):
    circs = _small_batch()
    outs = []
    for use_graph in (True, False):
        b = lr.LRBatch(circs, dtype="c64", use_graph=use_graph)
        b.run()
        first = [b.probs(i).cpu().numpy() for i in range(len(circs))]
        b.reset()
        b.run()
        second = [b.probs(i).cpu().numpy() for i in range(len(circs))]
        for x, y in zip(first, second):
            assert np.array_equal(x, y)
        outs.append(first)
        b.close()
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


def test_heterogeneous_batch_workload_miniature(lr):
    """The 256-circuit family (n in 8..18, r in {8,16,32,64}, identical channels
    on every qubit) at 2% depth. Its cuts include exact eigenvalue ties, so two
    correct runs need not agree; what holds for every correct run: Tr rho =
    1 - discarded mass, and each run lies within its discarded mass (in L1 of
    Prob(x)) of the exact evolution, so two runs differ by at most the sum of
    their discarded masses."""
    circs = batch_circuits(count=24, depth_scale=0.02)
    b = lr.LRBatch(circs, dtype="c64")
    b.run()
    st = b.stats()
    assert st["gates"] > 0 and st["truncations"] > 0
    for i in (0, 5, 11, 23):
        cd = circs[i]
        pb = b.probs(i).double()
        inf = b.info(i)
        assert abs(float(pb.sum()) - (1.0 - inf["discarded"])) < 1e-5
        sim = lr.LRSim(cd["n"], cd["r"], dtype="c64")
        lr.run_ops(sim, cd["ops"], r=cd["r"])
        d1 = sim.info()["discarded"]
        assert float((sim.probs().double() - pb).abs().sum()) < inf["discarded"] + d1 + 1e-5
        sim.close()
    b.close()


@pytest.mark.parametrize("prec", ["refined", "fp32", "fp64"])
def test_batch_eigensolve_precisions_match_oracle(lr, prec):
    """A complex64 batch with each eigensolve precision against the oracle: the
    FP32 solve of every eigenvector with the FP64 refinement of the kept ones
    (default), the FP32 solve alone, and the solver in FP64 arithmetic."""
    circs = _small_batch()
    b = lr.LRBatch(circs, dtype="c64", eig_precision=prec)
    b.run()
    for i, cd in enumerate(circs):
        ref = O.run_lret(cd["n"], cd["ops"], r=cd["r"])
        pb = b.probs(i).double().cpu().numpy()
        inf = b.info(i)
        assert inf["converged"]
        assert np.sum(np.abs(pb - ref.probs())) < 1e-5, (prec, i)
        assert abs(inf["discarded"] - ref.discarded) < 1e-5, (prec, i)
    b.close()


def test_refined_batch_matches_refined_single_runs(lr):
    """The batched refinement (one launch per phase for all circuits of a step) and the
    single-circuit refinement after the same tridiagonal FP32 solve."""
    circs = _small_batch()
    b = lr.LRBatch(circs, dtype="c64", eig_precision="refined")
    b.run()
    for i, cd in enumerate(circs):
        sim = lr.LRSim(cd["n"], cd["r"], dtype="c64")
        sim.set_eigensolver("tridiag")
        sim.set_eig_precision("refined")
        lr.run_ops(sim, cd["ops"], r=cd["r"])
        p1 = sim.probs().double().cpu().numpy()
        pb = b.probs(i).double().cpu().numpy()
        # the two Gram matrices come from FP32 states through different kernels, so they
        # (and the FP64 sums the refinement makes exact for each) differ at FP32 level
        assert np.sum(np.abs(p1 - pb)) < 1e-5, i
        assert abs(b.info(i)["discarded"] - sim.info()["discarded"]) < 1e-5, i
        sim.close()
    b.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_per_circuit_split_counts_do_not_change_results(lr, dtype):
    """Per-circuit Gram split counts (as an autotuned table gives them) change only
    the order of the Gram sums."""
    circs = _small_batch()
    tol = 1e-11 if dtype == "c128" else 1e-5
    outs = []
    for splits in (None, [64, 1, 3, 2, 16, 8]):
        b = lr.LRBatch(circs, dtype=dtype, splits=splits)
        b.run()
        outs.append([(b.probs(i).double().cpu().numpy(), b.info(i)["discarded"]) for i in range(len(circs))])
        b.close()
    for (p0, d0), (p1, d1) in zip(*outs):
        assert np.sum(np.abs(p0 - p1)) < tol and abs(d0 - d1) < tol


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_cluster_and_one_cta_eigensolvers_of_a_batch_agree(lr, dtype):
    """Truncations whose Gram matrix has at least cluster_min_m rows run on the 8-CTA
    cluster solver, in a graph branch beside the one-CTA solver of the others: every
    truncation on one solver (0; 2), or split between the two (64: the 9-qubit circuit's
    128- and 64-row matrices on the cluster, the rest on one CTA; with the graph and
    with direct launches on two streams), gives the same states."""
    circs = _small_batch() + [{"n": 9, "r": 32, "ops": random_layered(9, 2, seed=5400, noise=("mixed", 2e-2, 4e-2),
                                                                     qubit_jitter=(0.5, 1.5))}]
    tol = 1e-11 if dtype == "c128" else 1e-5
    outs = []
    for cmin, graph in ((0, True), (2, True), (64, True), (64, False)):
        b = lr.LRBatch(circs, dtype=dtype, cluster_min_m=cmin, use_graph=graph)
        b.run()
        outs.append([(b.probs(i).double().cpu().numpy(), b.info(i)) for i in range(len(circs))])
        b.close()
    for other in outs[1:]:
        for i, ((p0, i0), (p1, i1)) in enumerate(zip(outs[0], other)):
            assert i1["converged"], i
            assert np.sum(np.abs(p0 - p1)) < tol, i
            assert abs(i0["discarded"] - i1["discarded"]) < tol, i
    # and the 9-qubit circuit against the oracle
    ref = O.run_lret(9, circs[-1]["ops"], r=32)
    assert np.sum(np.abs(outs[2][-1][0] - ref.probs())) < tol
    assert abs(outs[2][-1][1]["discarded"] - ref.discarded) < tol


def test_tensor_core_tasks_of_a_batch_match_single_runs_and_oracle(lr):
    """Circuits with 2^12 row pairs and more take the batched tcgen05 Gram and
    projection (one launch each per step for all of them, blocks mapped to tasks through
    prefix tables) beside SIMT tasks of small circuits in the same steps: each against
    its one-at-a-time run (tensor cores on) and the smallest ranks against the oracle."""
    specs = [(13, 8, 2), (13, 16, 2), (13, 32, 1), (14, 64, 1), (6, 8, 2), (13, 64, 1)]
    circs = []
    for i, (n, r, d) in enumerate(specs):
        ops = random_layered(n, d, seed=5300 + i, noise=("mixed", 1e-3, 2e-3), qubit_jitter=(0.5, 1.5))
        circs.append({"n": n, "r": r, "ops": ops})
    b = lr.LRBatch(circs, dtype="c64")
    b.run()
    for i, cd in enumerate(circs):
        sim = lr.LRSim(cd["n"], cd["r"], dtype="c64")
        sim.set_eigensolver("tridiag")
        lr.run_ops(sim, cd["ops"], r=cd["r"])
        p1 = sim.probs().double().cpu().numpy()
        pb = b.probs(i).double().cpu().numpy()
        inf = b.info(i)
        assert inf["converged"] and inf["compressions"] > 0, i
        assert abs(float(pb.sum()) - (1.0 - inf["discarded"])) < 1e-5, i
        assert np.sum(np.abs(p1 - pb)) < 1e-5, i
        assert abs(inf["discarded"] - sim.info()["discarded"]) < 1e-5, i
        sim.close()
    for i in (0, 1):  # 13 qubits, r = 8 and 16: the oracle finishes in seconds
        ref = O.run_lret(circs[i]["n"], circs[i]["ops"], r=circs[i]["r"])
        pb = b.probs(i).double().cpu().numpy()
        assert np.sum(np.abs(pb - ref.probs())) < 1e-5, i
        assert abs(b.info(i)["discarded"] - ref.discarded) < 1e-5, i
    b.close()
