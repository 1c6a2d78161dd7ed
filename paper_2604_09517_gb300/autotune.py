"""Autotuner for the batched solver's tile shapes.

The batched kernel has two panel widths per system, 32 (variant 0) or 16
(variant 1), and two residencies: a plan whose systems all use the 16-wide
panel runs two CTAs per SM (its shared memory fits twice), any other plan one.
For each system kind (0: pivoted FP64 LU, 1: BF16 block LU + FP64 refinement)
and size bucket, `tune()` builds a batch of systems drawn from that bucket and
times, with CUDA events on the GPU, the 32-wide panel at one CTA per SM and the
16-wide panel at one and at two CTAs per SM; each bucket keeps the faster
width. Because the residency belongs to the whole launch, a bucket that
prefers the 32-wide panel would pull every other system down to one CTA per
SM, so `tune()` then times a whole mixed batch (the benchmark's size
distribution) both ways, per-bucket widths against 16 everywhere, and records
the faster as the table's policy. The table is stored as JSON beside this file
(one entry per GPU name); `variants()` maps a batch's sizes and kinds to the
tuned choice (variant 0 where nothing was tuned).
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
    if entry.get("policy") == "narrow":
        out[:] = 1
        return out
    b = bucket_of(n)
    for k in (0, 1):
        choice = entry.get("choice", {}).get(str(k))
        if choice:
            sel = kind == k
            out[sel] = np.asarray(choice, dtype=np.uint8)[b[sel]]
    return out


def _time_batch(hpl, bt, seed: int, variant, reps: int, one_per_sm: bool) -> float:
    """Best of `reps` timed runs (after one untimed) of a planned batch."""
    import torch
    hpl.batched_config(0, 1 if one_per_sm else 0)
    try:
        bt.plan(variant=variant)
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
    finally:
        hpl.batched_config(0, 0)
    return best


def tune(seed: int = 7, per_bucket: int = 304, reps: int = 3, path: str | None = TABLE, device="cuda",
         batch_seed: int = 1, batch_count: int = 4096) -> dict:
    """Time every shape per kind and size bucket, then the whole-batch policy;
    write and return the table."""
    import paper_2604_09517_gb300 as hpl

    rng = np.random.default_rng(seed)
    choice, times = {}, {}
    for k in (0, 1):
        choice[str(k)], times[str(k)] = [], []
        for b in range(len(BUCKETS) - 1):
            n = rng.integers(BUCKETS[b], BUCKETS[b + 1], per_bucket)
            bt = hpl.Batch(n, np.full(per_bucket, k, dtype=np.uint8), device=device)
            t32 = _time_batch(hpl, bt, seed, 0, reps, True)
            t16_1 = _time_batch(hpl, bt, seed, 1, reps, True)
            t16_2 = _time_batch(hpl, bt, seed, 1, reps, False)
            choice[str(k)].append(0 if t32 < t16_2 else 1)
            times[str(k)].append({"panel32_1_per_sm": t32, "panel16_1_per_sm": t16_1, "panel16_2_per_sm": t16_2})
            del bt
    # whole-batch policy on the benchmark's size distribution
    nb = hpl.batch_sizes(batch_seed, batch_count)
    kind = np.array([0 if s < batch_count // 2 else 1 for s in range(batch_count)], dtype=np.uint8)
    bt = hpl.Batch(nb, kind, device=device)
    bkt = bucket_of(nb)
    per_bucket_v = np.array([choice[str(int(k))][int(b_)] for k, b_ in zip(kind, bkt)], dtype=np.uint8)
    t_per_bucket = _time_batch(hpl, bt, batch_seed, per_bucket_v, reps, False)
    t_narrow = _time_batch(hpl, bt, batch_seed, 1, reps, False)
    del bt
    policy = "narrow" if t_narrow <= t_per_bucket else "per_bucket"
    entry = {"buckets": list(BUCKETS), "variants": {"0": "panel 32", "1": "panel 16"}, "choice": choice,
             "best_of_ms": times, "systems_per_bucket": per_bucket, "policy": policy,
             "policy_ms": {"per_bucket": t_per_bucket, "narrow": t_narrow,
                           "batch": f"{batch_count} systems, sizes of seed {batch_seed}, half general"}}
    table = load_table(path) if path else {}
    table[_gpu_name()] = entry
    if path:
        with open(path, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return table


if __name__ == "__main__":
    print(json.dumps(tune(), indent=1))
