"""Benchmark: noisy gate-steps/sec of low-rank noisy-circuit evolution on GB300.

Workload (synthetic, seeded): 20 qubits, rank r = 64, random layered circuit
(Ry, Rz on every qubit, then CNOTs on a random perfect matching), one-qubit
depolarizing channel p = 5e-4 after every gate on every qubit it touches
(K = 4 Kraus matrices, r*K = 256 columns before each truncation). V is
2^20 x 64 complex64 (0.54 GB), the expansion 2^20 x 256 (2.1 GB): both far
larger than L2, so no flush is needed between steps.

One step = one circuit layer through the whole forward path: 50 gates, each
fused with its channel expansion, 60 truncations (Gram, eigensolve,
projection), then the readouts Prob(x) and <H> for a 64-term random Pauli sum.
A noisy gate-step is one gate with its channel(s) and truncation(s).

Prints one JSON line (see the keys below). --impl reference times the CPU
oracle on this host on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS, RANK, P_DEP, DEPTH, N_TERMS, SEED = 20, 64, 5e-4, 200, 64, 3000
METRIC = "noisy gate-steps/sec at 20q r=64 (mixed vs FP64), adjoint grad time/forward"


def workload_config():
    return {"workload": "random layered Ry/Rz+CNOT, 20 qubits, r=64, depolarizing p=5e-4 after every gate "
                        "(K=4, rK=256), <H> of 64 random Pauli terms",
            "n_qubits": N_QUBITS, "rank": RANK, "kraus": 4, "depth_total": DEPTH, "step": "one circuit layer",
            "gates_per_step": None, "truncations_per_step": None,
            "l2_policy": "inputs larger than L2 (V 0.54 GB, expansion 2.1 GB)"}


_LAYERS = None


def get_layers():
    global _LAYERS
    if _LAYERS is None:
        from workloads import random_layered
        ops = random_layered(N_QUBITS, DEPTH, seed=SEED, noise=("dep", P_DEP))
        layers, cur = [], []
        per_layer = 2 * N_QUBITS * 2 + (N_QUBITS // 2) * 3  # gates + their channels
        for o in ops:
            cur.append(o)
            if len(cur) == per_layer:
                layers.append(cur)
                cur = []
        assert not cur and len(layers) == DEPTH
        _LAYERS = layers
    return _LAYERS


def count(ops):
    from workloads import count_ops
    return count_ops(ops)


def max_over_ranks(ms, world, device=None):
    """Slowest rank's time (replicas run independent circuits; the job ends when
    the last one does). Barrier on both sides so no rank starts the next phase
    early."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def aggregate_value(units_per_rank, world, ms_max):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2009_06657_gb300 as lr
    from workloads import random_pauli_sum

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    layers = get_layers()
    terms = random_pauli_sum(N_QUBITS, N_TERMS, seed=SEED + 1)
    xm, zm, cf = lr.pauli_masks(terms, N_QUBITS)
    sim = lr.LRSim(N_QUBITS, RANK, dtype="c64", stream=stream)
    probs = torch.empty(1 << N_QUBITS, dtype=torch.float32, device=dev)
    g_per, c_per = count(layers[0])

    def step(i):
        lr.run_ops(sim, layers[i % DEPTH], r=RANK)
        sim.probs(probs)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
        sim.expect_masks(xm, zm, cf)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(dev.index)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        n_launch0 = lr.launch_count()
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        sim.expect_masks(xm, zm, cf)  # readout of <H> at the end of the timed region
        e1.record(stream)
        n_launch = lr.launch_count() - n_launch0
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)

        # per-kernel device time over one more step (CUDA events on the handle's stream)
        sim.set_timing(True)
        step(args.warmup + args.steps)
        sim.expect_masks(xm, zm, cf)
        ktimes = sim.kernel_times()
        sim.set_timing(False)

        # end to end through the public API with host buffers: host parameters in,
        # Prob(x) and <H> copied back to pinned host memory, every step
        host_p = torch.empty(1 << N_QUBITS, dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_e2e = max(1, min(args.steps, 3))
        for i in range(n_e2e):
            lr.run_ops(sim, layers[(args.warmup + args.steps + 1 + i) % DEPTH], r=RANK)
            sim.probs(probs)
            host_p.copy_(probs, non_blocking=True)
            sim.expect_masks(xm, zm, cf)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / n_e2e

        # readouts beyond the step (Sec. II.D sampling, App. A entropy) on the same state:
        # 1000 shots from Prob(x) and the entropy of the 64-column state, CUDA events
        rd = {}
        u = np.random.default_rng(SEED + 2).random(1000)
        sim.sample(u)  # warm-up (allocates the CDF buffer)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(5):
            sim.sample(u)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_s = ev0.elapsed_time(ev1) / 5
        sbytes = (1 << N_QUBITS) * RANK * 8 + (1 << N_QUBITS) * 8 * 3  # V once; CDF write, offset pass
        rd["sample_1000_shots_ms"] = t_s
        rd["sample_hbm_gbs"] = sbytes / (t_s * 1e-3) / 1e9
        S = sim.entropy()
        ev0.record(stream)
        for _ in range(3):
            S = sim.entropy()
        ev1.record(stream)
        torch.cuda.synchronize()
        rd["entropy_ms"] = ev0.elapsed_time(ev1) / 3
        rd["entropy_bits"], rd["effective_rank"] = S

    info = sim.info()
    sim.close()
    eigv = bench_eig_variants(dev, stream, layers) if (rank == 0 and not args.no_eig_variants) else None
    # FP64 comparators at the same size (few truncations; rate per noisy gate-step)
    fp64 = bench_fp64(args, layers, dev, stream) if (rank == 0 and not args.no_fp64) else None
    adj = bench_adjoint(dev, stream) if (rank == 0 and not args.no_adjoint) else None
    bat = (bench_batch(dev, stream, scale=args.batch_scale, cluster_min_m=args.batch_cluster_min_m)
           if (rank == 0 and not args.no_batch) else None)
    epsl = bench_eps(dev, stream) if (rank == 0 and not args.no_eps) else None
    grv = bench_grover(dev, stream) if (rank == 0 and not args.no_grover) else None
    return dict(ms=ms, g_per=g_per, c_per=c_per, ktimes=ktimes, clk=clk, e2e_s=e2e_s, fp64=fp64, info=info,
                adjoint=adj, batch=bat, eps=epsl, launches=n_launch, readouts=rd, grover=grv, eig_variants=eigv)


def bench_fp64(args, layers, dev, stream):
    """Plain FP64 low-rank GPU path on the same GB300: complex128 torch/cuBLAS
    GEMMs and torch.linalg.eigh, plus this library's own complex128 path.
    Times truncation steps at the steady state (c = 64 -> 256 columns)."""
    import torch

    import paper_2009_06657_gb300 as lr
    out = {}
    # (a) this library, complex128 (FP64 Jacobi eigensolve, FP64 Gram)
    sim = lr.LRSim(N_QUBITS, RANK, dtype="c128", stream=stream)
    ops = layers[0]
    # advance until the first truncation at full width has happened
    idx = 0
    with torch.cuda.stream(stream):
        while sim.info()["compressions"] < 1:
            o = ops[idx]; idx += 1
            lr.run_ops(sim, [o], r=RANK)
        torch.cuda.synchronize()
        n_tr = 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        while n_tr < 4 and idx < len(ops):
            o = ops[idx]; idx += 1
            lr.run_ops(sim, [o], r=RANK)
            if o["op"] in ("dep",):
                n_tr += 1
        sim.info()  # flush a deferred projection inside the timed region
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) * 1e-3 / max(n_tr, 1)
    sim.close()
    out["ours_c128_s_per_truncation"] = dt
    # (b) plain torch complex128 (cuBLAS ZGEMM + cuSOLVER eigh)
    N = 1 << N_QUBITS
    g = torch.Generator(device=dev).manual_seed(1)
    V = torch.randn(N, RANK, dtype=torch.complex128, device=dev, generator=g)
    V /= torch.linalg.norm(V)
    K = [torch.eye(2, dtype=torch.complex128, device=dev) * (1 - P_DEP) ** 0.5]
    sx = torch.tensor([[0, 1], [1, 0]], dtype=torch.complex128, device=dev)
    sy = torch.tensor([[0, -1j], [1j, 0]], dtype=torch.complex128, device=dev)
    sz = torch.tensor([[1, 0], [0, -1]], dtype=torch.complex128, device=dev)
    K += [s * (P_DEP / 3) ** 0.5 for s in (sx, sy, sz)]

    def plain_step(V, q):
        Vt = V.reshape(N >> (q + 1), 2, 1 << q, V.shape[1])
        Vp = torch.cat([torch.einsum("ab,ibjc->iajc", k, Vt).reshape(N, -1) for k in K], dim=1)
        G = Vp.conj().T @ Vp
        lam, U = torch.linalg.eigh(G)
        return Vp @ U[:, -RANK:].flip(1)

    with torch.cuda.stream(stream):
        V = plain_step(V, 0)
        torch.cuda.synchronize()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(reps):
            V = plain_step(V, 1 + i)
        e1.record(stream)
        torch.cuda.synchronize()
        out["torch_c128_s_per_truncation"] = e0.elapsed_time(e1) * 1e-3 / reps
    del V
    torch.cuda.empty_cache()
    return out


def bench_eig_variants(dev, stream, layers):
    """The same 20-qubit layers with the three eigensolve precisions of the FP32
    state (lr_set_eig_precision): FP32 solve + FP64 refinement (the headline
    path), FP32 solve alone, FP64 solve. One warm-up layer, one layer timed with
    CUDA events, one more with per-kernel-class events."""
    import torch

    import paper_2009_06657_gb300 as lr
    g_per, _ = count(layers[0])
    out = {}
    for mode in ("refined", "fp32", "fp64"):
        sim = lr.LRSim(N_QUBITS, RANK, dtype="c64", stream=stream)
        sim.set_eig_precision(mode)
        with torch.cuda.stream(stream):
            lr.run_ops(sim, layers[0], r=RANK)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            lr.run_ops(sim, layers[1], r=RANK)
            sim.info()  # flush the deferred projection inside the timed region
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            sim.set_timing(True)
            lr.run_ops(sim, layers[2], r=RANK)
            kt = sim.kernel_times()
        sim.close()
        ent = {"layer_ms": ms, "gate_steps_per_s": g_per / (ms * 1e-3)}
        for cls in ("eigh", "refine"):
            t, c = kt[cls]
            ent[cls + "_ms_per_launch"] = t / c if c else None
        out[mode] = ent
    out["refined_over_fp32_time"] = out["refined"]["layer_ms"] / out["fp32"]["layer_ms"]
    return out


def bench_adjoint(dev, stream, reps=2):
    """Adjoint gradient time / forward time on the 14-qubit hardware-efficient
    ansatz: 6 layers of Ry, Rz on every qubit plus a CZ ladder (168 parameters,
    angles N(0, 0.5^2)), depolarizing p = 1e-3 after every gate, r = 32,
    complex64 state, checkpoint every 8 stages, 50-term random Pauli sum.
    The forward pass records the tape (truncation eigenvectors and
    eigenvalues, state checkpoints); the backward pass recomputes states
    between checkpoints and runs the adjoint kernels."""
    import torch

    import paper_2009_06657_gb300 as lr
    from workloads import hea, random_pauli_sum
    n, r = 14, 32
    ops, th = hea(n, 6, seed=4000, noise=("dep", 1e-3))
    terms = random_pauli_sum(n, 50, seed=4001)
    sim = lr.LRSim(n, r, dtype="c64", stream=stream)
    fwd, bwd = [], []
    with torch.cuda.stream(stream):
        for i in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.reset()
            sim.set_checkpoint(8)
            sim.set_record(True)
            lr.run_ops(sim, ops, r=r, thetas=th)
            val = sim.expect(terms)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g = sim.backward(terms, len(th))
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            sim.set_record(False)
            if i > 0:
                fwd.append(t1 - t0)
                bwd.append(t2 - t1)
    sim.close()
    f, b = statistics.median(fwd), statistics.median(bwd)
    return {"workload": "14-qubit HEA, 6 layers, 168 parameters, r=32, dep p=1e-3, 50 Pauli terms, "
                        "checkpoint every 8 stages", "forward_s": f, "backward_s": b,
            "adjoint_over_forward": b / f, "grad_norm": float(sum(x * x for x in g) ** 0.5)}


def bench_grover(dev, stream, reps=3):
    """Amplitude amplification of the basis states of Hamming weight <= 2 at 13
    qubits (Sec. III.D's largest size): Hadamards, 7 Grover iterates, a
    depolarizing channel (p = 1e-3) on every qubit after the Hadamards and after
    each iterate, each followed by a truncation to rank 41 (0.5 % of full rank),
    complex64. Dense form: each iterate is one 8192 x 8192 unitary held on the
    device (lr_apply_gate_device); factorised form: sign oracle and reflection as
    diagonal gates between two Hadamard layers. CUDA events on the handle's stream."""
    import numpy as np
    import torch

    import paper_2009_06657_gb300 as lr
    from workloads import grover, grover_good
    n, r = 13, 41
    ops, t = grover(n, p=1e-3, dense=True)
    U = torch.tensor(next(o["U"] for o in ops if o["op"] == "unitary"), dtype=torch.complex64, device=dev)
    ops_dev = [dict(o, U=U) if o["op"] == "unitary" else o for o in ops]
    ops_fact, _ = grover(n, p=1e-3, dense=False)
    good = torch.tensor(grover_good(n), device=dev)
    sim = lr.LRSim(n, r, dtype="c64", stream=stream)
    probs = torch.empty(1 << n, dtype=torch.float32, device=dev)
    out = {"workload": "13-qubit Grover / amplitude amplification, HW(x) <= 2, 7 iterates, dep p=1e-3 "
                       "on every qubit after each layer, r=41 (0.5% of full rank), complex64"}
    with torch.cuda.stream(stream):
        for name, seq in (("dense", ops_dev), ("factorised", ops_fact)):
            ts = []
            for i in range(reps + 1):
                sim.reset()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lr.run_ops(sim, seq, r=r)
                sim.probs(probs)
                e1.record(stream)
                torch.cuda.synchronize()
                if i > 0:
                    ts.append(e0.elapsed_time(e1))
            out[name + "_circuit_ms"] = statistics.median(ts)
            out[name + "_good_probability"] = float(probs[good].double().sum())
        # one dense iterate on the final 41-column state: 8 D^2 c real flops
        c = sim.info()["columns"]
        D = 1 << n
        allq = list(range(n - 1, -1, -1))
        sim.apply_gate(allq, U)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            sim.apply_gate(allq, U)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out["dense_iterate_columns"] = c
        out["dense_iterate_ms"] = ms
        out["dense_iterate_tflops"] = 8.0 * D * D * c / (ms * 1e-3) / 1e12
        out["dense_iterate_gate_read_gbs"] = D * D * 8 * ((c + 31) // 32) / (ms * 1e-3) / 1e9
    out["iterates"] = t
    sim.close()
    return out


def bench_batch(dev, stream, scale=1.0, sample_single=4, eig_precision="refined", cluster_min_m=None):
    """256 seeded circuits (n ~ U{8..18}, r in {8,16,32,64}, depth ~ U{40..200}
    layers scaled by `scale`, mixed depolarizing 1e-3 / amplitude damping 2e-3),
    complex64, the eigensolve `eig_precision` (FP32 solve + FP64 refinement of the
    kept eigenvectors by default), Gram split counts from the autotuned table,
    advanced together by one CUDA-graph launch (timed once with CUDA events, after
    a warm-up run of the same circuits at 2% depth); against the first
    `sample_single` circuits run one at a time through the single-circuit path
    (rate per gate-step). cluster_min_m: Gram matrices with at least this many rows
    go to the 8-CTA cluster eigensolver (None: the library's default)."""
    import torch

    import paper_2009_06657_gb300 as lr
    from paper_2009_06657_gb300.autotune import DEFAULT_TABLE, BatchTable
    from workloads import batch_circuits
    table = BatchTable.load_or_empty()
    circs = batch_circuits(count=256, depth_scale=scale)
    splits = table.splits_for(circs)
    with torch.cuda.stream(stream):
        warm = batch_circuits(count=256, depth_scale=0.02)
        wb = lr.LRBatch(warm, dtype="c64", stream=stream, eig_precision=eig_precision,
                        splits=table.splits_for(warm), cluster_min_m=cluster_min_m)
        wb.run()
        torch.cuda.synchronize()
        wb.close()
        t0 = time.perf_counter()
        b = lr.LRBatch(circs, dtype="c64", stream=stream, eig_precision=eig_precision, splits=splits,
                       cluster_min_m=cluster_min_m)
        t_build = time.perf_counter() - t0
        st = b.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = lr.launch_count()
        e0.record(stream)
        b.run()
        e1.record(stream)
        n_launch = lr.launch_count() - n0
        torch.cuda.synchronize()
        t_batch = e0.elapsed_time(e1) / 1e3
        trunc = sum(b.info(i)["compressions"] for i in range(len(circs)))
        b.close()
        # one at a time (sample)
        gates = 0
        t1 = time.perf_counter()
        for cd in circs[:sample_single]:
            sim = lr.LRSim(cd["n"], cd["r"], dtype="c64", stream=stream)
            sim.set_eig_precision(eig_precision)
            lr.run_ops(sim, cd["ops"], r=cd["r"])
            sim.info()
            gates += sum(1 for o in cd["ops"] if o["op"] in ("rx", "ry", "rz", "cnot", "cz"))
            sim.close()
        torch.cuda.synchronize()
        t_single = time.perf_counter() - t1
    return {"workload": f"256 random circuits, n U{{8..18}}, r in {{8,16,32,64}}, depth U{{40..200}} x {scale}, "
                        "mixed depolarizing 1e-3 / amplitude damping 2e-3, complex64",
            "eig_precision": eig_precision,
            "cluster_min_m": cluster_min_m if cluster_min_m is not None else "library default (256)",
            "splits_table": os.path.basename(DEFAULT_TABLE) if table.entries else None,
            "splits_table_device": table.device or None,
            "gates": st["gates"], "truncations": st["truncations"], "truncations_done": trunc,
            "schedule_steps": st["steps"], "graph_kernels_per_run": n_launch, "build_s": t_build,
            "batch_s": t_batch, "batch_gate_steps_per_s": st["gates"] / t_batch,
            "single_gate_steps_per_s": gates / t_single, "single_sample_circuits": sample_single,
            "speedup": (st["gates"] / t_batch) / (gates / t_single)}


def bench_eps(dev, stream, n=13, depth=3, p=1e-3, eps=1e-4):
    """The eps rule at the paper's eps / p = 0.1 setting (Sec. III.A: p = 0.1 %,
    eps = 1e-4, 13 qubits): the random layered family with depolarizing channels,
    complex64 (refined eigensolve), the kept rank chosen on the device at every
    truncation; CUDA-event time of the whole circuit after one untimed run, the rank
    history from the truncation log and V_I of Eq. 8. Depth 3: in the fourth layer the
    rule keeps more than 64 columns, so the next channel's Gram matrix would exceed the
    eigensolvers' 256 columns."""
    import numpy as np
    import torch

    import paper_2009_06657_gb300 as lr
    from workloads import random_layered
    ops = random_layered(n, depth, seed=SEED + 10, noise=("dep", p))
    gates = sum(1 for o in ops if o["op"] in ("rx", "ry", "rz", "cnot", "cz"))
    sim = lr.LRSim(n, 64, dtype="c64", capacity=256, stream=stream)
    sim.set_eps(eps)
    sim.set_trunc_log(1 << 16)
    try:
        with torch.cuda.stream(stream):
            lr.run_ops(sim, ops, r=0)
            sim.info()
            sim.reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lr.run_ops(sim, ops, r=0)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            log = sim.trunc_log()
            info = sim.info()
    except RuntimeError as ex:
        sim.close()
        return {"error": str(ex)}
    sim.close()
    ks = np.array([e["k"] for e in log]) if log else np.zeros(1)
    return {"workload": f"{n} qubits, depth {depth} random layered family, depolarizing p = {p}, eps = {eps} "
                        "(eps / p = 0.1), complex64",
            "gate_steps_per_s": gates / t, "s": t, "gates": gates, "truncations": len(log),
            "final_rank": int(info["columns"]), "max_rank": int(ks.max()), "mean_rank": float(ks.mean()),
            "mean_V_I": float(np.mean([e["V_I"] for e in log])) if log else None,
            "discarded": info["discarded"]}


# Algorithmic work of one steady-state launch of each kernel class on the
# benchmark workload (n = 20, c = k = r = 64 columns, K = 4 Kraus matrices,
# m = K r = 256), structured truncation path (the Gram and projection act on the
# row pairs of the channel's qubit; V' is never formed).
def algorithmic():
    N, r, K, esz = 1 << N_QUBITS, RANK, 4, 8
    N2, m = N // 2, 4 * RANK
    return {
        # Gram of the row pairs: (2r x 2r) Hermitian, N/2 rows, complex MAC = 8 flop, half by symmetry.
        # Issued tensor work: the real view (N/2 x 4r) Gram's upper triangle by 128-row blocks
        # (128 x 256 + 128 x 128 at 4r = 256), three TF32 passes (hi hi, hi lo, lo hi)
        "gram": {"flop": 8.0 * N2 * (2 * r) ** 2 / 2, "bytes": N * r * esz,
                 "mma_flop": 3 * 2.0 * N2 * (128 * 4 * r + 128 * (4 * r - 128))},
        # projection on the row pairs: (N/2 x 2r) x (2r x 2r), read V and write V_new; issued:
        # the real (N/2 x 4r) x (4r x 4r) product, three TF32 passes
        "project": {"flop": 8.0 * N2 * (2 * r) * (2 * r), "bytes": 2 * N * r * esz,
                    "mma_flop": 3 * 2.0 * N2 * (4 * r) * (4 * r)},
        # Householder reduction of the m x m Hermitian matrix dominates: (16/3) m^3 flop
        "eigh": {"flop": 16.0 / 3.0 * m ** 3, "bytes": m * m * 16},
        # FP64 refinement of the kept eigenvectors: G X (m x m x r) and X^dag X (r x m x r) complex
        # FP64 products, then X^dag X and the Lowdin product for each of the three
        # orthonormalisation steps (FP32 products not counted)
        "refine": {"flop": 8.0 * (m * m * r + 4 * r * m * r + 3 * m * r * r), "bytes": None},
        # expansion for two-qubit gates (gate only, K = 1): read and write V
        "expand": {"flop": None, "bytes": 2 * N * r * esz},
        "readout": {"flop": None, "bytes": N * r * esz + N * 4},
        # <H>: one pass over V per group of 4 terms, reading each row and its 4 partner rows
        "pauli": {"flop": None, "bytes": -(-N_TERMS // 4) * 5 * N * r * esz},
    }


# DRAM bytes (read + write) per launch from one ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum, m = 256, median of the three launches
# of the 18-qubit profiling case); the eigensolver's traffic does not depend on the
# qubit count (it reads the m x m Gram matrix).
NCU_TRAFFIC = {"eigh": 1230080}


def kernel_rooflines(kt, peaks):
    alg = algorithmic()
    out = {}
    for k, (ms, cnt) in kt.items():
        if cnt == 0 or k not in alg:
            continue
        t = ms / cnt * 1e-3
        a = alg[k]
        e = {"ms_per_launch": ms / cnt, "launches": cnt}
        if a["bytes"]:
            e["hbm_gbs"] = a["bytes"] / t / 1e9
            e["hbm_frac"] = e["hbm_gbs"] / peaks["hbm_gbs"]
        if a["flop"]:
            e["tflops"] = a["flop"] / t / 1e12
        if a.get("mma_flop"):
            # tensor work the kernel issues (3xTF32 on the real view) against the TF32 dense peak
            e["tensor_issued_tflops"] = a["mma_flop"] / t / 1e12
            e["tensor_issued_frac"] = e["tensor_issued_tflops"] / peaks["tf32_tflops"]
        out[k] = e
    return out


def profile_case(n, solver="auto", eig_precision="refined"):
    """A short run for profilers: the first 12 ops of the benchmark's circuit
    family on n qubits (r = 64), which reach 64 columns and then truncate the
    256-column Gram matrix through the tensor-core Gram, the eigensolver
    (`solver`: auto = the cluster solver at this size, or tridiag; `eig_precision`:
    refined, fp32 or fp64) and the tensor-core projection."""
    import torch

    import paper_2009_06657_gb300 as lr
    from workloads import random_layered
    ops = random_layered(n, 1, seed=SEED, noise=("dep", P_DEP))
    sim = lr.LRSim(n, RANK, dtype="c64")
    sim.set_eigensolver(solver)
    sim.set_eig_precision(eig_precision)
    lr.run_ops(sim, ops[:12], r=RANK)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": n, "solver": solver, "eig_precision": eig_precision, "info": {k: v for k, v in sim.info().items() if isinstance(v, (int, float))}}))
    sim.close()


def profile_batch(scale):
    """One run of the batched workload (256 circuits of the benchmark's batch family,
    depths scaled by `scale`) for profilers: no timing, no single-circuit comparison."""
    import torch

    import paper_2009_06657_gb300 as lr
    from paper_2009_06657_gb300.autotune import BatchTable
    from workloads import batch_circuits
    circs = batch_circuits(count=256, depth_scale=scale)
    b = lr.LRBatch(circs, dtype="c64", splits=BatchTable.load_or_empty().splits_for(circs))
    b.run()
    torch.cuda.synchronize()
    print(json.dumps({"profile_batch": scale, "stats": b.stats()}))
    b.close()


def profile_readouts(n):
    """A short run for profilers of the kernels beyond the truncation: one dense
    13-qubit Grover iterate (8192 x 8192 unitary on 41 columns), then on an n-qubit
    state of the benchmark family (r = 64): the grouped <H> readout of 64 Pauli
    terms, 1000 measurement shots and the entropy."""
    import numpy as np
    import torch

    import paper_2009_06657_gb300 as lr
    from workloads import grover, random_layered, random_pauli_sum
    ops, _ = grover(13, p=1e-3, dense=True)
    U = torch.tensor(next(o["U"] for o in ops if o["op"] == "unitary"), dtype=torch.complex64, device="cuda")
    g = lr.LRSim(13, 41, dtype="c64")
    lr.run_ops(g, [dict(o, U=U) if o["op"] == "unitary" else o for o in ops[:40]], r=41)
    g.apply_gate(list(range(12, -1, -1)), U)
    torch.cuda.synchronize()
    sim = lr.LRSim(n, RANK, dtype="c64")
    lr.run_ops(sim, random_layered(n, 1, seed=SEED, noise=("dep", P_DEP))[:12], r=RANK)
    terms = random_pauli_sum(n, N_TERMS, seed=SEED + 1)
    val = sim.expect(terms)
    shots = sim.sample(np.random.default_rng(SEED + 2).random(1000))
    S = sim.entropy()
    torch.cuda.synchronize()
    print(json.dumps({"profile_readouts": n, "expect": val, "shots": int(len(shots)), "entropy": S[0]}))
    g.close()
    sim.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-readouts", type=int, default=0,
                    help="run only the dense-gate and readout kernels on an n-qubit state for profilers and exit")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="run only a short n-qubit case for profilers (no timing) and exit")
    ap.add_argument("--profile-batch", type=float, default=0.0,
                    help="run only the batched workload once at this depth scale for profilers and exit")
    ap.add_argument("--profile-solver", default="auto", choices=["auto", "tridiag", "cluster", "jacobi"],
                    help="eigensolver of --profile-case")
    ap.add_argument("--profile-eig-precision", default="refined", choices=["refined", "fp32", "fp64"],
                    help="eigensolve precision of --profile-case")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-grover", action="store_true")
    ap.add_argument("--no-eig-variants", action="store_true")
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-cluster-min-m", type=int, default=None)
    ap.add_argument("--no-eps", action="store_true")
    args = ap.parse_args()
    if args.profile_readouts:
        profile_readouts(args.profile_readouts)
        return
    if args.profile_batch:
        profile_batch(args.profile_batch)
        return
    if args.profile_case:
        profile_case(args.profile_case, args.profile_solver, args.profile_eig_precision)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        return
    import json as _j
    peaks = load_peaks()
    value = aggregate_value(res["g_per"] * args.steps, world, res["ms"])
    kt = res["ktimes"]
    dom = max(kt, key=lambda k: kt[k][0])
    kr = kernel_rooflines(kt, peaks)
    d = kr.get(dom, {})
    if dom in ("gram", "project"):
        # tensor-core GEMMs: useful flops against the TF32 dense peak
        bound, ach, peak, unit = "tensor", d.get("tflops"), peaks["tf32_tflops"], "TFLOP/s"
    elif dom == "eigh":
        # FP32 SIMT arithmetic: chip-wide FP32 peak (the kernel occupies one cluster of
        # 8 SMs; the share of those 8 SMs is reported separately below)
        bound, ach, peak, unit = "alu", d.get("tflops"), peaks["fp32_tflops"], "TFLOP/s"
    else:
        bound, ach, peak, unit = "hbm", d.get("hbm_gbs"), peaks["hbm_gbs"], "GB/s"
    cfg = workload_config()
    cfg["gates_per_step"] = res["g_per"]
    cfg["truncations_per_step"] = res["c_per"]
    out = {
        "metric": METRIC, "value": value, "unit": "noisy gate-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 state: FP32 gates, 3xTF32 tensor-core Gram/projection; eigensolve FP32 then FP64 "
                 "refinement of the kept eigenvectors (FP64 eigenvalues and discarded mass); FP64 sums",
        "data": "synthetic (seeded random circuits)", "config": cfg,
        "gpu_launches": None,
        "kernel_ms_per_step": {k: v[0] for k, v in kt.items()},
        "kernel_launches_per_step": {k: v[1] for k, v in kt.items()},
        "roofline": {"kernel": dom, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                     "frac": (ach / peak) if ach else None, "traffic": NCU_TRAFFIC.get(dom),
                     "peak_source": peaks["source"]},
        "kernels": kr,
        "clocks": res["clk"],
        "e2e": {"value": res["g_per"] / res["e2e_s"], "unit": "noisy gate-steps/s",
                "h2d_bytes_per_step": h2d_bytes(get_layers()[0]), "d2h_bytes_per_step": (1 << N_QUBITS) * 4 + 8},
        "fp64": None, "cpu_baseline": None, "adjoint": res.get("adjoint"), "batch": res.get("batch"),
        "readouts": res.get("readouts"), "grover": res.get("grover"), "eig_variants": res.get("eig_variants"),
        "eps_rule": res.get("eps"),
    }
    out["gpu_launches"] = res["launches"]  # the library's own launch counter over the timed region
    if res["fp64"]:
        f = res["fp64"]
        tps = res["c_per"] / res["g_per"]  # truncations per gate-step
        out["fp64"] = {k.replace("_s_per_truncation", "_gate_steps_per_s"): 1.0 / (v * tps) for k, v in f.items()}
        out["fp64"]["mixed_over_ours_c128"] = value / out["fp64"]["ours_c128_gate_steps_per_s"]
        out["fp64"]["mixed_over_torch_c128"] = value / out["fp64"]["torch_c128_gate_steps_per_s"]
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(res)
    print(_j.dumps(out))


def h2d_bytes(ops):
    b = 0
    for o in ops:
        if o["op"] in ("ry", "rz", "rx"):
            b += 8 + 8  # angle + parameter id
        elif o["op"] in ("cnot", "cz"):
            b += 16 * 16 + 8
        else:
            b += 4 * 64  # Kraus set (4 x 2x2 complex128)
    return b


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        # FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (nominal unit counts and clock)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "tf32_tflops": d["bf16_tflops"] * 1.1 / 2.25,
                "fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12,
                "source": "hbm, bf16 measured (MEASURED_PEAKS.json); tf32 = measured bf16 x nominal 1.1/2.25; "
                          "fp32 = chip-wide SIMT peak from unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "tf32_tflops": 1900.0 * 1.1 / 2.25,
            "fp32_tflops": 152 * 128 * 2 * 2.07e9 / 1e12, "source": "fallback"}


def cpu_truncations(count):
    """Bounded CPU sample: the oracle runs the first layer's ops; the prefix that
    brings the state to 64 columns is untimed, then the next `count` full-width
    truncations (channel, c = 64 -> 256 -> 64, Gram, eigh, projection) are timed
    one by one. Returns their durations in seconds."""
    from oracle import lret as O
    ops = get_layers()[0]
    st = O.LRETState(N_QUBITS)
    times = []
    for o in ops:
        if O.is_gate(o):
            qs, U = O.gate_matrix(o)
            st.gate(qs, U)
        else:
            full = st.L.shape[1] == RANK
            t0 = time.perf_counter()
            st.channel(o["q"], O.channel_kraus(o))
            st.compress(r=RANK)
            if full and st.log[-1]["m"] == 4 * RANK:
                times.append(time.perf_counter() - t0)
                if len(times) >= count:
                    break
    return times


def cpu_baseline(res):
    times = cpu_truncations(3)
    s_per_tr, n_tr = statistics.median(times), len(times)
    tps = res["c_per"] / res["g_per"]
    return {"value": 1.0 / (s_per_tr * tps), "unit": "noisy gate-steps/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"oracle (NumPy complex128) on the host: {n_tr} full-width truncations (2^20 x 256 "
                      f"Gram, eigh, projection) of the 20-qubit workload, extrapolated per noisy gate-step"}


def run_reference(args):
    """The oracle as it stands on the host cores: W untimed and K timed full-width
    truncations of the benchmark workload (one per step), reported per noisy
    gate-step like the GPU arm."""
    times = cpu_truncations(args.warmup + args.steps)
    per = times[args.warmup:] or times
    s_per_tr = statistics.median(per)
    g_per, c_per = count(get_layers()[0])
    v = 1.0 / (s_per_tr * c_per / g_per)
    cfg = workload_config()
    cfg["gates_per_step"] = g_per
    cfg["truncations_per_step"] = c_per
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "noisy gate-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded random circuits)",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": "noisy gate-steps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"oracle (NumPy complex128) on the host: {len(per)} timed full-width "
                                       f"truncations of the 20-qubit workload after {args.warmup} untimed, "
                                       f"extrapolated per noisy gate-step"},
            "e2e": {"value": v, "unit": "noisy gate-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


if __name__ == "__main__":
    main()
