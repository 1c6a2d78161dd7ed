"""Autotuner for the batched solver's tile shapes.

The batched kernel has two compiled variants per system: panel width 32
(variant 0) or 16 (variant 1). For each system kind (0: pivoted FP64 LU,
1: BF16 block LU + FP64 refinement) and size bucket, `tune()` builds a batch
of systems drawn from that bucket, times every variant with CUDA events on the
GPU and keeps the fastest. The table is stored as JSON beside this file (one
entry per GPU name); `variants()` maps a batch's sizes and kinds to the tuned
choice (variant 0 where nothing was tuned).
"""
from __future__ import annotations

import json
import os

import numpy as np

BUCKETS = (32, 64, 128, 256, 513)          # bucket b holds BUCKETS[b] <= n < BUCKETS[b+1]
VARIANTS = (0, 1)
TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_batched.json")


def bucket_of(n) -> np.ndarray:
    return np.clip(np.searchsorted(BUCKETS, np.asarray(n), side="right") - 1, 0, len(BUCKETS) - 2)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "none"


def load_table(path: str = TABLE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def variants(n, kind, table: dict | None = None, gpu: str | None = None) -> np.ndarray:
    """Per-system variant from the tuned table (0 where untuned)."""
    n = np.asarray(n)
    kind = np.asarray(kind)
    if table is None:
        table = load_table()
    entry = table.get(gpu or _gpu_name()) or (next(iter(table.values())) if table else None)
    out = np.zeros(len(n), dtype=np.uint8)
    if not entry:
        return out
    b = bucket_of(n)
    for k in (0, 1):
        choice = entry.get("choice", {}).get(str(k))
        if choice:
            sel = kind == k
            out[sel] = np.asarray(choice, dtype=np.uint8)[b[sel]]
    return out


def tune(seed: int = 7, per_bucket: int = 304, reps: int = 3, path: str | None = TABLE, device="cuda") -> dict:
    """Time every variant per kind and size bucket; write and return the table."""
    import torch

    import paper_2604_09517_gb300 as hpl

    rng = np.random.default_rng(seed)
    choice, times = {}, {}
    for k in (0, 1):
        choice[str(k)], times[str(k)] = [], []
        for b in range(len(BUCKETS) - 1):
            n = rng.integers(BUCKETS[b], BUCKETS[b + 1], per_bucket)
            bt = hpl.Batch(n, np.full(per_bucket, k, dtype=np.uint8), device=device)
            ms = []
            for v in VARIANTS:
                bt.plan(variant=v)
                best = float("inf")
                for _ in range(reps + 1):                       # first run warms up
                    bt.generate(seed)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    bt.run()
                    e1.record()
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                ms.append(best)
            choice[str(k)].append(int(VARIANTS[int(np.argmin(ms))]))
            times[str(k)].append(ms)
            del bt
    entry = {"buckets": list(BUCKETS), "variants": {"0": "panel 32", "1": "panel 16"}, "choice": choice,
             "best_of_ms": times, "systems_per_bucket": per_bucket}
    table = load_table(path) if path else {}
    table[_gpu_name()] = entry
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    print(json.dumps(tune(), indent=1))
