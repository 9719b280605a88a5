"""Autotuner of the batched path's Gram split count, with a persisted table.

A truncation of the batch forms the Gram matrix of the row pairs in `splits`
slices of the 2^(n-1) row pairs (one partial (2c x 2c) Gram matrix per slice and
column tile, reduced in a fixed order afterwards). More slices give more thread
blocks per circuit; fewer slices give less partial data to reduce. The best count
depends on n, on r (the tile count) and on the GPU, so it is measured: for every
(n, r) class a probe batch of `copies` identical circuits of that class (one layer
of the random Ry/Rz + CNOT family with depolarizing channels) runs once per
candidate split count, timed with CUDA events on the batch's stream, and the
fastest count is kept.

The table is a JSON file: {"device": ..., "candidates": [...], "entries":
[{"n", "r", "splits", "ms": {candidate: time}}]}. Lookup is exact on (n, r); a
class that was not tuned takes the entry of the same r with the nearest n (the
smaller n on a tie), and a rank with no entry at all takes 0 (the library's rule
from rows_per_split).

    python -m paper_2009_06657_gb300.autotune --out table.json   (needs the GPU)

The table read by default is `tuning/batch_splits.json` beside this module; the
environment variable LRET_TUNING_TABLE names another file (for a GPU or a workload
the committed table was not measured on).
"""
from __future__ import annotations

import argparse
import json
import os

DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "batch_splits.json")
TABLE_ENV = "LRET_TUNING_TABLE"
CANDIDATES = (1, 2, 4, 8, 16, 32, 64)


def table_path():
    """The table file in use: $LRET_TUNING_TABLE if set and non-empty, else the committed one."""
    return os.environ.get(TABLE_ENV) or DEFAULT_TABLE


class BatchTable:
    """(n, r) -> Gram split count, with the lookup rule of the module docstring."""

    def __init__(self, entries=None, device="", candidates=CANDIDATES):
        self.entries = {}
        self.times = {}
        self.device = device
        self.candidates = tuple(candidates)
        for e in entries or []:
            self.add(e["n"], e["r"], e["splits"], e.get("ms"))

    def add(self, n, r, splits, ms=None):
        if int(splits) < 1:
            raise ValueError("split count must be >= 1")
        self.entries[(int(n), int(r))] = int(splits)
        if ms is not None:
            self.times[(int(n), int(r))] = {str(k): float(v) for k, v in ms.items()}

    def lookup(self, n, r):
        key = (int(n), int(r))
        if key in self.entries:
            return self.entries[key]
        same_r = [nn for (nn, rr) in self.entries if rr == key[1]]
        if not same_r:
            return 0
        best = min(same_r, key=lambda nn: (abs(nn - key[0]), nn))
        return self.entries[(best, key[1])]

    def splits_for(self, circuits):
        return [self.lookup(c["n"], c["r"]) for c in circuits]

    def to_json(self):
        ents = []
        for (n, r), sp in sorted(self.entries.items()):
            e = {"n": n, "r": r, "splits": sp}
            if (n, r) in self.times:
                e["ms"] = self.times[(n, r)]
            ents.append(e)
        return {"device": self.device, "candidates": list(self.candidates), "entries": ents}

    def save(self, path):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(self.to_json(), f, indent=1)

    @classmethod
    def load(cls, path=None):
        with open(path or table_path()) as f:
            d = json.load(f)
        return cls(d.get("entries", []), d.get("device", ""), d.get("candidates", CANDIDATES))

    @classmethod
    def load_or_empty(cls, path=None):
        path = path or table_path()
        return cls.load(path) if os.path.exists(path) else cls()


def probe_circuits(n, r, copies, seed=7000):
    from workloads import random_layered
    return [{"n": n, "r": r, "ops": random_layered(n, 1, seed + i, noise=("dep", 1e-3))} for i in range(copies)]


def time_batch(circuits, splits, eig_precision="refined", reps=3):
    """Best of `reps` timed runs (ms) of one batch whose circuits all use `splits`."""
    import torch

    from .sim import LRBatch
    stream = torch.cuda.Stream()
    b = LRBatch(circuits, dtype="c64", stream=stream, eig_precision=eig_precision,
                splits=[splits] * len(circuits))
    best = float("inf")
    try:
        b.run()  # warm-up
        for _ in range(reps):
            b.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run()
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
    finally:
        b.close()
    return best


def tune(ns=range(8, 19), ranks=(8, 16, 32, 64), candidates=CANDIDATES, copies=8, reps=3,
         eig_precision="refined", log=None):
    import torch
    table = BatchTable(device=torch.cuda.get_device_name(0), candidates=candidates)
    for r in ranks:
        for n in ns:
            circs = probe_circuits(n, r, copies)
            pairs = 1 << (n - 1)
            ms = {}
            for sp in candidates:
                if sp > pairs:
                    continue
                ms[sp] = time_batch(circs, sp, eig_precision, reps)
            best = min(ms, key=lambda k: (ms[k], k))
            table.add(n, r, best, ms)
            if log:
                log(f"n={n} r={r}: splits {best} ({ms[best]:.3f} ms; " +
                    ", ".join(f"{k}: {v:.3f}" for k, v in ms.items()) + ")")
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="table file to write (default: $LRET_TUNING_TABLE or the committed table)")
    ap.add_argument("--copies", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    table = tune(copies=args.copies, reps=args.reps, log=print)
    out = args.out or table_path()
    table.save(out)
    print("wrote", out)


if __name__ == "__main__":
    main()
