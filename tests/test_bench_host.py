"""Host-side logic of bench.py, on CPU: the per-step performance model fit
recovers known phase rates from synthetic per-step records and predicts the
model's own step times; the reference arm (the CPU oracle) prints one JSON
line with the fields the benchmark contract asks for."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _synthetic_records(n, nb, rates, fixed):
    """Per-step records of one factorization whose phases follow
    time = work / rate + fixed exactly (phase ids 0 PFACT, 1 SWAP, 2 TRSM,
    3 update), with the LU's per-step work."""
    nsteps = (n + nb - 1) // nb
    ph, st, ms, wk = [], [], [], []
    for k in range(nsteps):
        c0 = k * nb
        kb = min(nb, n - c0)
        m = n - c0
        m2 = m - kb
        works = {0: m * kb * kb - kb ** 3 / 3.0, 1: 4.0 * kb * (n - kb) * 8, 2: kb * (kb - 1.0) * m2,
                 3: 2.0 * m2 * m2 * kb}
        for p in (0, 1, 2, 3):
            if works[p] <= 0:
                continue
            ph.append(p)
            st.append(k)
            wk.append(works[p])
            ms.append(works[p] / rates[p] + fixed[p])
    return {"phase": np.array(ph), "step": np.array(st), "ms": np.array(ms), "work": np.array(wk)}, nsteps


def test_step_model_recovers_rates_and_predicts_the_model():
    sys.path.insert(0, ROOT)
    import bench
    n, nb = 8192, 256
    # rates in work units per ms: 1.25 TF/s update, 0.2 TF/s panel, 1.3 TF/s TRSM, 800 GB/s swap
    rates = {0: 0.2e9, 1: 0.8e9, 2: 1.3e9, 3: 1.25e9}
    fixed = {0: 5.0, 1: 0.0, 2: 0.4, 3: 0.7}
    recs, nsteps = _synthetic_records(n, nb, rates, fixed)
    out = bench.step_model(recs, n, nb, measured_ms=1.0)
    f = out["fit"]
    assert abs(f["update_tflops"] - 1.25) < 1e-6 and abs(f["update_fixed_ms"] - 0.7) < 1e-6
    assert abs(f["pfact_gflops"] - 200.0) < 1e-6 and abs(f["pfact_fixed_ms"] - 5.0) < 1e-6
    assert abs(f["trsm_gflops"] - 1300.0) < 1e-6 and abs(f["trsm_fixed_ms"] - 0.4) < 1e-6
    # the model's total, computed here from the same per-step times
    t = {p: np.zeros(nsteps) for p in range(4)}
    for p, k, m in zip(recs["phase"], recs["step"], recs["ms"]):
        t[p][k] += m
    want = sum(t[1][k] + t[2][k] + max(t[3][k], t[0][k + 1] if k + 1 < nsteps else 0.0) for k in range(nsteps))
    assert abs(out["predicted_ms"] - want) <= 1e-6 * want
    # first step whose next panel outlasts its update
    exposed = next((k for k in range(nsteps - 1) if t[0][k + 1] > t[3][k]), None)
    assert out["panel_not_hidden_from_step"] == exposed


def test_reference_arm_prints_the_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample-n", "1024"], capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "TFLOP/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["steps"] == 1 and line["warmup"] == 0 and line["config"]["workload"]
    assert line["config"]["reference_sample_n"] == 1024 and "n=1024" in line["cpu_baseline"]["sample"]
