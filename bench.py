#!/usr/bin/env python
"""Benchmark: HPL FP64 LU solve (n=32768, NB=256, depth-1 look-ahead) on GB300,
with the HPL-MxP mixed-precision solve (n=98304, NB=4096) reported beside it.

One step = one full solve of a fresh seeded system: lu_factor (PFACT, SWAP,
DTRSM, DGEMM update, look-ahead) + lu_solve, all in the library's CUDA
kernels through the C ABI. The matrix (8.6 GB) is regenerated on the device
before each step, outside the timed interval; it is far larger than L2, so no
L2 flush is needed. value = credited flops (2n^3/3 + 2n^2) / time, summed over
ranks, divided by the slowest rank's time.

The mixed-precision solve (BF16 block-LU on the tcgen05 tensor cores + FP64
GMRES refinement) is timed the same way and reported under "mxp", with its
speedup over the FP64 LU's rate.

Prints one JSON line (rank 0). --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Solve TFLOP/s (2n³/3+2n²): FP64 LU vs MxP+IR at HPL residual<16, % peak"
FP64_FLOP_PER_CLK_PER_SM = 4.0      # 2 DFMA/clk/SM: nominal 1.25 TF/s / (152 SMs * 2.07 GHz)
NUM_SMS = 152
MAX_SM_MHZ = 2070.0
# DRAM bytes (read + write) per flop of the DFMA update kernel, from one ncu
# capture of an m=7936, n=7680, k=256 launch of k_dgemm_sub<64> (956.9 MB for
# 31.21 GFLOP); the traffic of an update launch scales with its C tile, i.e.
# with flops at fixed k.
DGEMM_DRAM_BYTES_PER_FLOP = 956.9e6 / 31.21e9
# Same for the tcgen05 trailing update of the mixed-precision solve, from one
# ncu capture each of the step-0 update at n = 24576, NB = 4096 (m = 20480,
# k = 4096, 3.436 TFLOP): key (prec, storage). BF16, FP8, FP16 and TF32 with
# FP32 storage on the pair kernel with the bulk-tensor epilogue and two-atom
# stages (4.711, 3.807, 4.743 and 11.132 GB,
# profiles/k_gemm_tc_pair_update_two_atom_stages_n24576.txt); BF16 operands
# with BF16 storage on the single-CTA kernel's per-thread epilogue (3.512 GB,
# k_gemm_tc_update_bf16_vs_fp32_storage_n24576.txt). At fixed k a launch's
# traffic scales with its C tile, i.e. with its flops; captured at the
# bench's panel width only, so another width reports null.
MXP_DRAM_BYTES_PER_FLOP = {(0, 0): 4.711e9 / 3.436e12, (1, 0): 3.807e9 / 3.436e12, (2, 0): 4.743e9 / 3.436e12,
                           (3, 0): 11.132e9 / 3.436e12, (0, 1): 3.512e9 / 3.436e12}
MXP_TRAFFIC_NB = 4096


def flops(n: int) -> float:
    return 2.0 * n ** 3 / 3.0 + 2.0 * n ** 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--nb", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample-n", type=int, default=8192)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mxp", action="store_true", help="skip the mixed-precision solve")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched solve")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the differentiable solve")
    ap.add_argument("--no-emulation", action="store_true", help="skip the tensor-core FP64 emulation line")
    ap.add_argument("--batched-count", type=int, default=4096)
    ap.add_argument("--mxp-n", type=int, default=98304)
    ap.add_argument("--mxp-nb", type=int, default=4096)
    ap.add_argument("--mxp-fp8-nb", type=int, default=4096)
    ap.add_argument("--mxp-ns-iters", type=int, default=1,
                    help="Newton-Schulz steps per diagonal block in the n = 98304 solves (library default 2)")
    ap.add_argument("--mxp-inner", default="fp32", choices=["fp32", "fp64"],
                    help="GMRES inner matrix-vector products of the mixed-precision solves: on an FP32 copy of A "
                         "(default) or on the FP64 A; residuals and the acceptance test are FP64 either way")
    ap.add_argument("--mxp-large-n", type=int, default=0,
                    help="also time one regenerated-A, BF16-storage solve of this size (0: skip)")
    return ap.parse_args()


def workload_config(a):
    return {"workload": f"hpl_fp64_lu_n{a.n}_nb{a.nb}_lookahead1", "n": a.n, "nb": a.nb, "nrhs": 1,
            "lookahead": 1, "seed": a.seed, "matrix": "i.i.d. uniform[-0.5,0.5) FP64, SplitMix64 counter generator",
            "l2": f"inputs larger than L2 ({8.0 * a.n * a.n / 1e9:.1f} GB matrix), no flush",
            "parallelism": "replicas (one independent solve per GPU)"}


# --- distributed plumbing ----------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# --- clocks --------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for k, v in zip(names[1:], parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(k)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --- oracle timing (CPU baseline and the reference arm) ------------------------------

def time_oracle(n: int, seed: int):
    import oracle
    A = oracle.generate(seed, oracle.STREAM_A, n, n)
    b = oracle.generate(seed, oracle.STREAM_B, n, 1)[:, 0]
    t0 = time.perf_counter()
    LU, ipiv, info, _ = oracle.getrf(A)
    x = oracle.getrs(LU, ipiv, b)
    dt = time.perf_counter() - t0
    return dt, oracle.num_threads(), oracle.scaled_residual(A, x, b)


def time_oracle_one_core(n: int, seed: int):
    """The oracle's getrf + getrs of one n-system on a single host core (a
    child process with OMP_NUM_THREADS=1, so the parent's thread pool is
    untouched)."""
    code = ("import sys, time; sys.path.insert(0, %r); import oracle; "
            "A = oracle.generate(%d, oracle.STREAM_A, %d, %d); b = oracle.generate(%d, oracle.STREAM_B, %d, 1)[:, 0]; "
            "t0 = time.perf_counter(); LU, ip, info, _ = oracle.getrf(A); x = oracle.getrs(LU, ip, b); "
            "print(time.perf_counter() - t0)") % (ROOT, seed, n, n, seed, n)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    return float(out.stdout.strip().splitlines()[-1])


def time_oracle_batched(seed: int, count: int, sample: int):
    """The oracle on a sample of the batched workload's systems (the first
    sample/2 general ones and the first sample/2 dominant ones), and the
    whole batch extrapolated by credited flops of each kind."""
    import numpy as np

    import oracle
    n = oracle.batch_sizes(seed, count)
    half = count // 2
    t = {0: 0.0, 1: 0.0}
    fl = {0: 0.0, 1: 0.0}
    for s in list(range(sample // 2)) + list(range(half, half + sample // 2)):
        kind = 0 if s < half else 1
        m = int(n[s])
        A = oracle.generate(seed, oracle.batch_stream_a(s), m, m, dominant=bool(kind))
        b = oracle.generate(seed, oracle.batch_stream_b(s), m, 1)[:, 0]
        t0 = time.perf_counter()
        if kind == 0:
            oracle.solve(A, b)
        else:
            oracle.mxp_solve(A, b, 16, prec=oracle.PREC_BF16, refine=0, ns_iters=3)
        t[kind] += time.perf_counter() - t0
        fl[kind] += flops(m)
    total_fl = {k: sum(flops(int(m)) for s, m in enumerate(n) if (s >= half) == bool(k)) for k in (0, 1)}
    est = sum(t[k] * total_fl[k] / fl[k] for k in (0, 1) if fl[k] > 0)
    return sum(t.values()), est, oracle.num_threads()


def run_reference(a, d: Dist):
    if d.rank != 0:
        return
    # the same bounded sample as cpu_baseline: one n = 8192 system per step
    # (about 12 s on 16 Grace cores), so both report the oracle at one rate
    n = a.cpu_sample_n
    for _ in range(a.warmup):
        time_oracle(n, a.seed)
    times = []
    sr = None
    cores = 1
    for _ in range(a.steps):
        dt, cores, sr = time_oracle(n, a.seed)
        times.append(dt)
    total = sum(times)
    value = flops(n) * len(times) / total / 1e12
    sample = (f"oracle getrf+getrs (unblocked FP64, OpenMP over columns) of one n={n} system per step, "
              f"standing in for the n={a.n} workload of config (rate in TFLOP/s at the sample size)")
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(a), "reference_sample_n": n}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "scaled_residual": sr}
    print(json.dumps(line), flush=True)


# --- our arm -------------------------------------------------------------------------

def measured_peaks():
    """Pool-measured peaks (copy bandwidth, cuBLAS BF16) or the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def run_batched(a, d: Dist, dev):
    """4096 systems, n ~ U{32..512}: half general (pivoted FP64 LU), half
    diagonally dominant (BF16 block LU + FP64 refinement), one persistent
    launch captured in a CUDA graph and replayed; inputs regenerated before
    each replay (untimed)."""
    import numpy as np
    import torch

    import paper_2604_09517_gb300 as hpl

    count = a.batched_count
    n_all = hpl.batch_sizes(a.seed, count)
    kind_all = np.array([0 if s < count // 2 else 1 for s in range(count)], dtype=np.uint8)
    # several GPUs: each rank solves its share of the systems, no exchange
    ids = np.nonzero(hpl.batch_shard(n_all, kind_all, d.world) == d.rank)[0] if d.world > 1 else np.arange(count)
    n, kind = n_all[ids], kind_all[ids]
    bt = hpl.Batch(n, kind, device=dev, ids=ids)
    bt.generate(a.seed)
    bt.plan()
    bt.run()
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            bt.run()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(a.warmup):
        bt.generate(a.seed)
        g.replay()
    torch.cuda.synchronize(dev)
    step_ms = []
    for _ in range(a.steps):
        bt.generate(a.seed)
        d.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        d.barrier()
        step_ms.append(e0.elapsed_time(e1))
    recs = bt.info()
    ok = int(d.sum(float(sum(1 for r in recs if r["status"] == 0))))
    work = float(sum(flops(int(m)) for m in n_all))
    total_ms = d.max(sum(step_ms))
    value = work * len(step_ms) / (total_ms * 1e-3) / 1e12
    fp64_work = float(sum(flops(int(m)) for m, k in zip(n_all, kind_all) if k == 0))
    dom = [r["iters"] for r, k in zip(recs, kind) if k == 1]
    extra = {}
    if d.rank == 0 and not a.no_cpu:
        sample = min(64, count)
        t_s, t_est, cores = time_oracle_batched(a.seed, count, sample)
        extra = {"cpu_oracle_sample": f"{sample} systems ({sample // 2} general, {sample // 2} dominant), "
                                      f"{t_s:.2f} s on {cores} cores; whole batch extrapolated by flops of each kind",
                 "cpu_oracle_extrapolated_ms": t_est * 1e3}
    return {**extra, "workload": f"batched_{count}_n32to512_half_fp64_half_bf16ir", "systems": count, "value": value,
            "unit": "TFLOP/s", "ms_per_step": total_ms / len(step_ms), "solved_ok": ok,
            "flops_per_step": work, "fp64_share_of_flops": fp64_work / work, "cuda_graph": True,
            "gpu_launches_per_step": 1, "scaling": "strong" if d.world > 1 else None,
            "systems_per_rank": int(len(ids)),
            "max_refine_iters": int(d.max(float(max(dom) if dom else 0)))}


def run_adjoint(a, d: Dist, dev):
    """Differentiable solve: n = 4096 dominant A, 64 right-hand sides; forward
    BF16 block LU + FP64 GMRES refinement, backward grad_B = A^-T G and
    grad_A = -grad_B X^T on the saved factor."""
    import numpy as np
    import torch

    import paper_2604_09517_gb300 as hpl

    n, nrhs, nb = 4096, 64, 2048
    A = hpl.generate(a.seed, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT, device=dev)
    B = hpl.generate(a.seed, hpl.STREAM_B, n, nrhs, device=dev)
    G = torch.from_numpy(np.random.default_rng(a.seed).standard_normal((n, nrhs))).to(dev)
    stream = torch.cuda.current_stream(dev)
    fwd, bwd = [], []
    for it in range(a.warmup + a.steps):
        torch.cuda.synchronize(dev)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        X, info, ws = hpl.mxp_solve(A, B, nb=nb, refine=hpl.REFINE_IR)
        e1.record(stream)
        gB, gA, binfo = hpl.lu_solve_backward(A, X, G, ws, nb=nb, refine=hpl.REFINE_IR)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        if it >= a.warmup:
            fwd.append(e0.elapsed_time(e1))
            bwd.append(e1.elapsed_time(e2))
    fi, bi = info.read(), binfo.read()
    extra = {}
    if d.rank == 0 and not a.no_cpu:
        import oracle
        A0, B0, G0 = A.cpu().numpy(), B.cpu().numpy(), G.cpu().numpy()
        t0 = time.perf_counter()
        X0, _ = oracle.solve(A0, B0)
        t1 = time.perf_counter()
        oracle.adjoint(A0, X0, G0)
        t2 = time.perf_counter()
        extra = {"cpu_oracle_forward_ms": (t1 - t0) * 1e3, "cpu_oracle_backward_ms": (t2 - t1) * 1e3,
                 "cpu_oracle_cores": oracle.num_threads(),
                 "cpu_oracle_kind": "FP64 getrf+getrs; adjoint = its own FP64 LU, transposed solves, outer product"}
    return {**extra, "workload": "diff_solve_n4096_nrhs64", "refinement": "classic, all 64 columns as one block",
            "forward_ms": statistics.median(fwd), "backward_ms": statistics.median(bwd),
            "forward_ms_mean": sum(fwd) / len(fwd), "backward_ms_mean": sum(bwd) / len(bwd),
            "forward_status": fi["status_name"],
            "backward_status": binfo.read()["status_name"], "forward_scaled_residual": fi["scaled_residual"],
            "backward_scaled_residual": bi["scaled_residual"], "forward_iters": fi["iters"],
            "backward_iters": bi["iters"],
            "grad_a_outer_product_gflop": 2.0 * n * n * nrhs / 1e9}


def step_model(recs, n: int, nb: int, measured_ms: float):
    """Per-step phase times of the last timed FP64 solve and a fit of the
    per-step performance model (paper Sec. III-A.1, without the broadcast on
    one GPU): step k costs SWAP(k) + TRSM(k) + max(update(k), PFACT(k+1)),
    the panel of step k+1 running beside the update. Each phase time is fitted
    as work / rate + fixed cost by least squares."""
    import numpy as np
    ph, st, ms, wk = recs["phase"], recs["step"], recs["ms"], recs["work"]
    # the last solve: from the last record of PFACT step 0 on
    first = np.nonzero((ph == 0) & (st == 0))[0]
    if first.size == 0:
        return None
    sel = np.arange(first[-1], ph.size)
    ph, st, ms, wk = ph[sel], st[sel], ms[sel], wk[sel]
    nsteps = (n + nb - 1) // nb
    t = np.zeros((4, nsteps))
    w = np.zeros((4, nsteps))
    for p_, k_, m_, w_ in zip(ph, st, ms, wk):
        if 0 <= p_ <= 3 and 0 <= k_ < nsteps:
            t[p_, k_] += m_
            w[p_, k_] += w_

    def fit(p_):
        mask = w[p_] > 0
        if mask.sum() < 1:
            return None, None
        x, y = w[p_][mask], t[p_][mask]
        if mask.sum() < 2 or np.ptp(x) <= 1e-6 * x.max():
            return y.sum() / x.sum(), 0.0          # same work every step: a rate only
        X = np.stack([x, np.ones(x.size)], axis=1)
        coef, *_ = np.linalg.lstsq(X, y, rcond=None)
        return coef[0], coef[1]

    fits = {p_: fit(p_) for p_ in range(4)}

    def pred(p_, k_):
        a_, b_ = fits[p_]
        return a_ * w[p_, k_] + b_ if a_ is not None and w[p_, k_] > 0 else 0.0

    total = 0.0
    exposed, swap_over = None, None
    for k_ in range(nsteps):
        tu = pred(3, k_)
        tp = pred(0, k_ + 1) if k_ + 1 < nsteps else 0.0
        total += pred(1, k_) + pred(2, k_) + max(tu, tp)
        if exposed is None and t[0, k_ + 1 if k_ + 1 < nsteps else k_] > t[3, k_] and k_ + 1 < nsteps:
            exposed = k_
        if swap_over is None and t[1, k_] > t[3, k_] and t[3, k_] > 0:
            swap_over = k_
    rate = lambda p_, scale: (1.0 / fits[p_][0] / scale) if fits[p_][0] else None
    every = max(1, nsteps // 8)
    rows = [[k_, n - k_ * nb, round(t[3, k_], 3), round(t[0, k_], 3), round(t[1, k_], 3), round(t[2, k_], 3)]
            for k_ in range(0, nsteps, every)]
    return {"model": "T_k = SWAP_k + TRSM_k + max(UPDATE_k, PFACT_{k+1}); phase = work / rate + fixed (least squares)",
            "fit": {"update_tflops": rate(3, 1e9), "update_fixed_ms": fits[3][1],
                    "pfact_gflops": rate(0, 1e6), "pfact_fixed_ms": fits[0][1],
                    "swap_gbs": rate(1, 1e6), "swap_fixed_ms": fits[1][1],
                    "trsm_gflops": rate(2, 1e6), "trsm_fixed_ms": fits[2][1]},
            "predicted_ms": total, "measured_ms": measured_ms,
            "panel_not_hidden_from_step": exposed, "swap_exceeds_update_from_step": swap_over,
            "steps_columns": ["k", "rows", "update_ms", "pfact_ms", "swap_ms", "trsm_ms"], "steps": rows}


def run_emulated(a, d: Dist, dev, ipiv_native):
    """The same FP64 LU solve with the trailing update on the BF16 tensor cores
    at FP64 accuracy (sliced products, opts.fp64_emulation = 1): rate, scaled
    residual, and whether its pivots equal those of the DFMA solve."""
    import torch

    import paper_2604_09517_gb300 as hpl

    n, nb, seed = a.n, min(a.nb, 256), a.seed
    A = hpl.colmajor(n, n, device=dev)
    b = torch.empty(n, dtype=torch.float64, device=dev)
    b0 = torch.empty(n, dtype=torch.float64, device=dev)
    ipiv = torch.empty(n, dtype=torch.int32, device=dev)
    info = hpl.Info(dev)
    opts = hpl.make_opts(nb=nb, lookahead=1, fp64_emulation=1)
    import ctypes
    lib = hpl.load()
    ws = hpl.workspace(lib.lu_factor_workspace_size(n, ctypes.byref(opts)), dev)
    sws = hpl.workspace(lib.lu_solve_workspace_size(n, 1), dev)
    stream = torch.cuda.current_stream(dev)
    times = []
    for it in range(a.warmup + a.steps):
        hpl.generate(seed, hpl.STREAM_A, n, n, out=A)
        hpl.generate(seed, hpl.STREAM_B, n, 1, out=b.view(n, 1))
        b0.copy_(b)
        hpl.set_phase_timing(it == a.warmup + a.steps - 1)
        d.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hpl.lu_factor(A, nb=nb, lookahead=1, ipiv=ipiv, ws=ws, info=info, fp64_emulation=1)
        hpl.lu_solve(A, ipiv, b, ws=sws)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        d.barrier()
        if it >= a.warmup:
            times.append(e0.elapsed_time(e1))
    total = d.max(sum(times))
    phases = hpl.phase_times()
    hpl.set_phase_timing(False)
    rec = info.read()
    sr = float(hpl.scaled_residual(None, b, b0, seed=seed, kind=hpl.GEN_GENERAL))
    upd_ms, upd_fl, _ = phases["update"]
    out = {"workload": f"hpl_fp64_lu_n{n}_nb{nb}_lookahead1_update_on_bf16_tensor_cores",
           "phases_last_step_ms": {k: v[0] for k, v in phases.items() if v[2]},
           "update_fp64_equivalent_tflops": upd_fl / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None,
           "update_bf16_tensor_tflops": 66.0 * upd_fl / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None,
           "value": d.sum(flops(n) * len(times)) / (total * 1e-3) / 1e12, "unit": "TFLOP/s",
           "ms_per_step": total / len(times), "status": rec["status_name"], "scaled_residual": sr,
           "pivots_equal_dfma_solve": bool(torch.equal(ipiv, ipiv_native)) if nb == a.nb else None,
           "method": "FP64-accurate trailing update from exact BF16 slice products (11 slices of 6 bits, "
                     "66 slice products in 11 exact groups, combined in 64-bit integers); panel, swaps, TRSM "
                     "and solves in FP64"}
    del A, ws
    torch.cuda.empty_cache()
    return out


def run_small(a, d: Dist, dev):
    """The small HPL case: n = 1024, NB = 64, no look-ahead (16 panel steps,
    latency-bound). The 8 MB matrix fits in L2, so L2 is flushed (a 256 MB
    write) before each timed solve; the oracle's time for the same system is
    reported beside it."""
    import torch

    import paper_2604_09517_gb300 as hpl

    n, nb, seed, reps = 1024, 64, a.seed, 20
    A = hpl.colmajor(n, n, device=dev)
    b = torch.empty(n, dtype=torch.float64, device=dev)
    ipiv = torch.empty(n, dtype=torch.int32, device=dev)
    info = hpl.Info(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    times = []
    for it in range(a.warmup + reps):
        hpl.generate(seed, hpl.STREAM_A, n, n, out=A)
        hpl.generate(seed, hpl.STREAM_B, n, 1, out=b.view(n, 1))
        flush.fill_(it & 0xff)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hpl.lu_factor(A, nb=nb, lookahead=0, ipiv=ipiv, info=info)
        hpl.lu_solve(A, ipiv, b)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if it >= a.warmup:
            times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    out = {"workload": "hpl_fp64_lu_n1024_nb64_no_lookahead", "ms_per_solve": ms, "median_ms": statistics.median(times),
           "value": flops(n) / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "solves": reps,
           "status": info.read()["status_name"], "l2": "flushed (256 MB write) before each timed solve"}
    if d.rank == 0 and not a.no_cpu:
        dt, cores, _ = time_oracle(n, seed)
        out["cpu_oracle_ms"] = dt * 1e3
        out["cpu_oracle_cores"] = cores
        out["cpu_oracle_one_core_ms"] = time_oracle_one_core(n, seed) * 1e3
    del A, flush
    torch.cuda.empty_cache()
    return out


def run_mxp(a, d: Dist, dev, fp64_value, prec=0, regen=False, cpu=None, storage=0, n=None, steps=None,
            warmup=None):
    """HPL-MxP solve of the diagonally dominant system (n = 98304, NB = 4096):
    block-LU factor on the tcgen05 tensor cores (BF16 update; FP8 E4M3 with
    prec = 1, NB = 4096; scaled FP16 with prec = 2; TF32 with prec = 3) + FP64 GMRES refinement.
    regen: the library regenerates A from the seed instead of reading a
    stored FP64 copy. storage = 1 keeps the working matrix in BF16. n, steps,
    warmup override the defaults (a one-off larger solve)."""
    import torch

    import paper_2604_09517_gb300 as hpl

    n = n or a.mxp_n
    nb, seed = (a.mxp_fp8_nb if prec == 1 else a.mxp_nb), a.seed
    n_steps = steps or a.steps
    n_warm = a.warmup if warmup is None else warmup
    A = None if regen else hpl.generate(seed, hpl.STREAM_A, n, n, hpl.GEN_DIAG_DOMINANT, device=dev)
    b = hpl.generate(seed, hpl.STREAM_B, n, 1, device=dev)[:, 0].contiguous()
    X = hpl.colmajor(n, 1, device=dev)
    info = hpl.Info(dev)
    ws = None
    # FP32 inner products with FP32 storage only: the BF16-stored factor is
    # coarse enough that an FP32-accurate correction needs a second outer step
    # (measured: 2 corrections and 8 preconditioner applications against 1 and
    # 4). The larger regenerated solve keeps FP64 ones too: an FP32 copy of A
    # at n = 262144 would need 275 GB.
    use_f32 = a.mxp_inner == "fp32" and n == a.mxp_n and storage == 0
    inner = hpl.INNER_FP32 if use_f32 else hpl.INNER_FP64
    for _ in range(n_warm):
        X, info, ws = hpl.mxp_solve(A, b, nb=nb, X=X, ws=ws, info=info, prec=prec, seed=seed, storage=storage,
                                        ns_iters=a.mxp_ns_iters, inner=inner)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    hpl.set_phase_timing(True)
    clocks = ClockSampler(d.local)
    clocks.start()
    step_ms, launches = [], 0
    for _ in range(n_steps):
        d.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = hpl.launch_count()
        e0.record(stream)
        X, info, ws = hpl.mxp_solve(A, b, nb=nb, X=X, ws=ws, info=info, prec=prec, seed=seed, storage=storage,
                                        ns_iters=a.mxp_ns_iters, inner=inner)
        e1.record(stream)
        launches += hpl.launch_count() - l0
        torch.cuda.synchronize(dev)
        d.barrier()
        step_ms.append(e0.elapsed_time(e1))
    phases = hpl.phase_times()
    hpl.set_phase_timing(False)
    clk = clocks.stop()
    rec = info.read()
    total_ms = d.max(sum(step_ms))
    value = d.sum(flops(n) * len(step_ms)) / (total_ms * 1e-3) / 1e12
    peaks = measured_peaks()
    upd_ms, upd_flops, upd_cnt = phases["update"]
    achieved = upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None
    # FP8 and TF32 dense peaks: the measured BF16 peak times the nominal ratio
    # to BF16 (FP8 4.5 / 2.25, TF32 1.1 / 2.25 PFLOP/s)
    ratio = {1: 2.0, 3: 1.1 / 2.25}.get(prec, 1.0)
    peak = peaks["bf16_tflops_sustained"] * ratio
    del A, X, ws
    torch.cuda.empty_cache()
    tag = {0: "bf16", 1: "fp8e4m3", 2: "fp16", 3: "tf32"}[prec]
    stag = "_bf16storage" if storage else ""
    # the factorization alone: the step minus its refinement phase
    refine_ms = phases["refine"][0] / len(step_ms) if phases["refine"][2] else 0.0
    factor_ms = total_ms / len(step_ms) - refine_ms
    factor_tf = (2.0 * n ** 3 / 3.0) / (factor_ms * 1e-3) / 1e12 if factor_ms > 0 else None
    extra = {"factor_ms": factor_ms, "refine_ms": refine_ms, "factor_tflops": factor_tf,
             f"factor_fraction_of_{tag}_peak": factor_tf / peak if factor_tf else None}
    if cpu and cpu.get("seconds_at_sample_n"):
        sn = a.cpu_sample_n
        extra["cpu_oracle_fp64_lu_extrapolated_s"] = cpu["seconds_at_sample_n"] * (n / sn) ** 3
        extra["cpu_oracle_basis"] = f"oracle FP64 getrf+getrs at n={sn} x (n/{sn})^3"
    return {**extra, "workload": f"hpl_mxp_{tag}{stag}_n{n}_nb{nb}_gmres" + ("_regenerated_a" if regen else ""), "n": n, "nb": nb, "value": value, "unit": "TFLOP/s",
            "ms_per_step": total_ms / len(step_ms), "steps": n_steps, "warmup": n_warm,
            "storage": "bf16" if storage else "fp32", "ns_iters": a.mxp_ns_iters,
            "gmres_inner_products": "fp32 (FP32 copy of A)" if use_f32 else "fp64 (FP64 A)",
            "clocks": clk,
            "status": rec["status_name"], "scaled_residual": rec["scaled_residual"], "refine_iters": rec["iters"],
            "preconditioner_applications": rec["inner_iters"],
            "speedup_vs_fp64_lu_rate": value / fp64_value if fp64_value else None,
            "fp64_lu_time_at_this_n_s": flops(n) / (fp64_value * 1e12) if fp64_value else None,
            f"fraction_of_{tag}_peak": value / peak, "gpu_launches": int(launches),
            "matrix": "uniform[-0.5,0.5) FP64, diagonal = row sum of |a_ij| (diagonally dominant)"
                      + ("; regenerated from the seed, never stored" if regen else "; stored FP64"),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak if achieved else None,
                         "traffic": (MXP_DRAM_BYTES_PER_FLOP[(prec, storage)] * upd_flops / upd_cnt
                                     if upd_cnt and nb == MXP_TRAFFIC_NB and (prec, storage) in MXP_DRAM_BYTES_PER_FLOP
                                     else None),
                         "kernel": (f"k_gemm_tc_pair<{prec}> (tcgen05 {tag} trailing update A22 -= L21 A12, FP32 C, "
                                    "bulk-tensor epilogue)" if not storage else
                                    f"k_gemm_tc<{prec}> (tcgen05 {tag} trailing update A22 -= L21 A12, BF16 C)"),
                         "peak_basis": f"bf16_tflops_sustained ({peaks['source']})" + (
                             {1: " x 2 (FP8/BF16 nominal)", 3: " x 1.1/2.25 (TF32/BF16 nominal)"}.get(prec, "")),
                         "algorithmic_flops_per_launch": upd_flops / upd_cnt if upd_cnt else None},
            "phases": {k: {"ms_per_step": v[0] / len(step_ms), "intervals": v[2]} for k, v in phases.items() if v[2]}}


def run_ours(a, d: Dist):
    import torch

    import paper_2604_09517_gb300 as hpl

    torch.cuda.set_device(d.local)
    dev = torch.device("cuda", d.local)
    hpl.load()
    n, nb, seed = a.n, a.nb, a.seed
    A = hpl.colmajor(n, n, device=dev)
    b = torch.empty(n, dtype=torch.float64, device=dev)
    b0 = torch.empty(n, dtype=torch.float64, device=dev)
    ipiv = torch.empty(n, dtype=torch.int32, device=dev)
    info = hpl.Info(dev)
    opts = hpl.make_opts(nb=nb, lookahead=1)
    lib = hpl.load()
    import ctypes
    ws = hpl.workspace(lib.lu_factor_workspace_size(n, ctypes.byref(opts)), dev)
    sws = hpl.workspace(lib.lu_solve_workspace_size(n, 1), dev)
    stream = torch.cuda.current_stream(dev)

    def regenerate():
        hpl.generate(seed, hpl.STREAM_A, n, n, out=A)
        hpl.generate(seed, hpl.STREAM_B, n, 1, out=b.view(n, 1))
        b0.copy_(b)

    def solve():
        hpl.lu_factor(A, nb=nb, lookahead=1, ipiv=ipiv, ws=ws, info=info)
        hpl.lu_solve(A, ipiv, b, ws=sws)

    for _ in range(a.warmup):
        regenerate()
        solve()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(d.local)
    clocks.start()
    hpl.set_phase_timing(True)
    step_ms = []
    launches = 0
    for _ in range(a.steps):
        regenerate()
        d.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = hpl.launch_count()
        e0.record(stream)
        solve()
        e1.record(stream)
        launches += hpl.launch_count() - l0
        torch.cuda.synchronize(dev)
        d.barrier()
        step_ms.append(e0.elapsed_time(e1))
    recs = hpl.phase_records()
    phases = hpl.phase_times()
    hpl.set_phase_timing(False)
    clk = clocks.stop()
    rec = info.read()
    sr = float(hpl.scaled_residual(None, b, b0, seed=seed, kind=hpl.GEN_GENERAL))

    total_ms = d.max(sum(step_ms))
    total_flops = d.sum(flops(n) * len(step_ms))
    value = total_flops / (total_ms * 1e-3) / 1e12
    model = step_model(recs, n, nb, step_ms[-1])

    # roofline of the dominant kernel: the DGEMM trailing update (DFMA, FP64 ALU bound)
    upd_ms, upd_flops, upd_cnt = phases["update"]
    achieved = upd_flops / (upd_ms * 1e-3) / 1e12 if upd_ms > 0 else None
    traffic = DGEMM_DRAM_BYTES_PER_FLOP * upd_flops / upd_cnt if upd_cnt else None
    peak = NUM_SMS * FP64_FLOP_PER_CLK_PER_SM * MAX_SM_MHZ * 1e6 / 1e12
    phase_report = {k: {"ms_per_step": v[0] / max(len(step_ms), 1), "launch_intervals": v[2]}
                    for k, v in phases.items() if v[2]}
    # achieved rates of the phases: SWAP in HBM GB/s (its timer's work is the
    # bytes the interchanges move), PFACT in GFLOP/s and in HBM GB/s with one
    # read and one write of each panel as its algorithmic traffic
    panel_bytes = sum(2.0 * 8.0 * (n - k0) * min(nb, n - k0) for k0 in range(0, n, nb)) * len(step_ms)
    for k, unit in (("swap", "GB/s"), ("pfact", "GFLOP/s"), ("trsm", "GFLOP/s"), ("update", "GFLOP/s")):
        if k in phase_report and phases[k][0] > 0:
            phase_report[k]["rate"] = phases[k][1] / (phases[k][0] * 1e-3) / 1e9
            phase_report[k]["rate_unit"] = unit
    if "pfact" in phase_report and phases["pfact"][0] > 0:
        phase_report["pfact"]["hbm_gbs"] = panel_bytes / (phases["pfact"][0] * 1e-3) / 1e9

    # end to end through the public API with host buffers
    e2e = None
    if not a.no_e2e:
        regenerate()
        A_h = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        A_h.copy_(A)
        b_h = b0.cpu().pin_memory()
        x_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
        # the library's kernel copy from the pinned buffer (hpl_upload): the copy
        # engine's cudaMemcpyAsync of 8.6 GB took 41 ms back to back but 0.3-0.8 s
        # after the GPU had been busy or idle, the kernel copy 41-49 ms every time
        # x comes back the same way (hpl_download: a kernel writing the pinned
        # buffer), not by a copy-engine read-back that can stall the same way
        hpl.upload(A, A_h)
        torch.cuda.synchronize(dev)
        e2e_ms, parts = [], []
        for _ in range(a.steps):
            d.barrier()
            torch.cuda.synchronize(dev)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            hpl.upload(A, A_h)
            hpl.upload(b, b_h)
            ev[1].record(stream)
            solve()
            ev[2].record(stream)
            hpl.download(x_h, b)
            ev[3].record(stream)
            torch.cuda.synchronize(dev)
            d.barrier()
            e2e_ms.append(ev[0].elapsed_time(ev[3]))
            parts.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
        e2e_total = d.max(sum(e2e_ms))
        e2e = {"value": d.sum(flops(n) * len(e2e_ms)) / (e2e_total * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * n * n + 8 * n, "d2h_bytes_per_step": 8 * n,
               "ms_per_step": e2e_total / len(e2e_ms),
               "upload_ms": [round(p[0], 2) for p in parts], "solve_ms": [round(p[1], 2) for p in parts],
               "download_ms": [round(p[2], 3) for p in parts]}
        del A_h

    cpu = None
    if d.rank == 0 and d.world == 1 and not a.no_cpu:
        dt, cores, _ = time_oracle(a.cpu_sample_n, seed)
        scale = (n / a.cpu_sample_n) ** 3
        cpu = {"value": flops(a.cpu_sample_n) / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"oracle getrf+getrs (unblocked FP64, OpenMP) of one n={a.cpu_sample_n} system, "
                         f"{dt:.1f} s; n={n} extrapolated by n^3: {dt * scale:.0f} s",
               "seconds_at_sample_n": dt, "extrapolated_seconds_at_n": dt * scale}

    emu = None if a.no_emulation else run_emulated(a, d, dev, ipiv)
    del A, b, b0, ipiv, ws, sws
    torch.cuda.empty_cache()
    small = run_small(a, d, dev)
    mxp = None if a.no_mxp else run_mxp(a, d, dev, value, cpu=cpu)
    mxp_fp8 = None if a.no_mxp else run_mxp(a, d, dev, value, prec=1, cpu=cpu)
    mxp_fp16 = None if a.no_mxp else run_mxp(a, d, dev, value, prec=2, cpu=cpu)
    mxp_tf32 = None if a.no_mxp else run_mxp(a, d, dev, value, prec=3, cpu=cpu)
    mxp_regen = None if a.no_mxp else run_mxp(a, d, dev, value, regen=True)
    mxp_bf16s = None if a.no_mxp else run_mxp(a, d, dev, value, storage=1)
    # optional: one larger solve that only BF16 storage and a regenerated A fit
    mxp_large = (run_mxp(a, d, dev, value, regen=True, storage=1, n=a.mxp_large_n, steps=1, warmup=1)
                 if a.mxp_large_n and not a.no_mxp else None)
    batched = None if a.no_batched else run_batched(a, d, dev)
    adjoint = None if a.no_adjoint else run_adjoint(a, d, dev)

    if d.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": d.world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": total_ms / len(step_ms), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(a),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak if achieved else None, "traffic": traffic,
                             "algorithmic_flops_per_launch": upd_flops / upd_cnt if upd_cnt else None,
                             "kernel": "k_dgemm_sub (DFMA trailing update)",
                             "peak_basis": "152 SMs x 4 FP64 flop/clk x 2070 MHz"},
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
                "scaled_residual": sr, "status": rec["status_name"], "phases": phase_report, "step_model": model,
                "fraction_of_fp64_peak": value / peak, "fp64_emulated": emu, "small": small, "mxp": mxp, "mxp_fp8": mxp_fp8, "mxp_fp16": mxp_fp16, "mxp_tf32": mxp_tf32, "mxp_regenerated": mxp_regen, "mxp_bf16_storage": mxp_bf16s, "mxp_large": mxp_large, "batched": batched, "adjoint": adjoint}
        print(json.dumps(line), flush=True)


def main():
    a = parse()
    d = Dist()
    if a.impl == "reference":
        run_reference(a, d)          # rank 0 only; other ranks exit without work
    else:
        d.init("nccl")
        run_ours(a, d)
    d.close()


if __name__ == "__main__":
    main()
