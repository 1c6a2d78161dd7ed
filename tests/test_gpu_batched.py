"""Batched solve of many uneven systems in one persistent launch, against the
CPU oracle system by system (pivots, solutions, residuals, refinement
iteration counts), plus CUDA-graph capture and replay."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


def _np(t):
    return t.detach().cpu().numpy()


def _make(hpl, seed, count, half=None):
    n = hpl.batch_sizes(seed, count)
    half = count // 2 if half is None else half
    kind = np.array([0 if s < half else 1 for s in range(count)], dtype=np.uint8)
    bt = hpl.Batch(n, kind)
    bt.generate(seed)
    return bt


def _check_system(orc, bt, s, A0, b0, emulate=True):
    n = int(bt.n[s])
    rec = bt.info(s)
    x = _np(bt.rhs(s))
    assert rec["status"] == 0, (s, n, rec)
    assert orc.scaled_residual(A0, x, b0) < 16
    x64, _ = orc.solve(A0, b0)
    kappa = np.linalg.cond(A0, np.inf)
    if bt.kind[s] == 0:
        LUo, ipo, _, gap = orc.getrf(A0)
        assert gap > 1e-12, ("near-tie pivot column: pick another seed", s, gap)
        assert np.array_equal(_np(bt.pivots(s)), ipo), s
        assert np.abs(x - x64).max() / np.abs(x64).max() <= 100 * n * EPS * kappa
    else:
        assert np.abs(x - x64).max() / np.abs(x64).max() <= 2 * 16 * n * EPS * kappa
        if emulate:
            nbv = 16 if bt.variant[s] else 32
            emu = orc.mxp_solve(A0, b0, nbv, prec=orc.PREC_BF16, refine=0, ns_iters=3)   # as the batched kernel
            assert abs(rec["iters"] - emu["iters"]) <= 2, (s, rec, emu["iters"])


def test_batched_small_mixed(hpl, orc):
    import torch
    bt = _make(hpl, 2, 40)
    A0 = [_np(bt.matrix(s)).copy(order="F") for s in range(bt.count)]
    b0 = [_np(bt.rhs(s)).copy() for s in range(bt.count)]
    bt.plan()
    bt.run()
    torch.cuda.synchronize()
    for s in range(bt.count):
        _check_system(orc, bt, s, A0[s], b0[s])


@pytest.mark.parametrize("variant", [0, 1])
def test_batched_both_tile_variants(hpl, orc, variant):
    import torch
    bt = _make(hpl, 6, 24)
    A0 = [_np(bt.matrix(s)).copy(order="F") for s in range(bt.count)]
    b0 = [_np(bt.rhs(s)).copy() for s in range(bt.count)]
    bt.plan(variant=variant)
    bt.run()
    torch.cuda.synchronize()
    for s in range(bt.count):
        _check_system(orc, bt, s, A0[s], b0[s])


def test_batched_edge_sizes(hpl, orc):
    import torch
    n = np.array([1, 2, 31, 32, 33, 63, 64, 65, 511, 512, 1, 7, 32, 33, 100, 512], dtype=np.int64)
    kind = np.array([0] * 10 + [1] * 6, dtype=np.uint8)
    bt = hpl.Batch(n, kind)
    bt.generate(9)
    A0 = [_np(bt.matrix(s)).copy(order="F") for s in range(bt.count)]
    b0 = [_np(bt.rhs(s)).copy() for s in range(bt.count)]
    bt.plan()
    bt.run()
    torch.cuda.synchronize()
    for s in range(bt.count):
        _check_system(orc, bt, s, A0[s], b0[s], emulate=n[s] > 1)


def test_batched_cuda_graph_replay(hpl):
    import torch
    bt = _make(hpl, 4, 24)
    bt.plan()
    bt.run()                                   # warm-up outside capture
    torch.cuda.synchronize()
    ref_x = bt.B.clone()
    ref_piv = bt.ipiv.clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        bt.generate(4)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            bt.run()
    for _ in range(2):
        bt.generate(4)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(bt.B, ref_x) and torch.equal(bt.ipiv, ref_piv)
        assert all(r["status"] == 0 for r in bt.info())


def test_batched_singular_system_reported(hpl):
    import torch
    n = np.array([64, 64], dtype=np.int64)
    bt = hpl.Batch(n, np.array([0, 0], dtype=np.uint8))
    bt.generate(3)
    bt.matrix(1)[:, 10] = 0.0
    bt.plan()
    bt.run()
    torch.cuda.synchronize()
    assert bt.info(0)["status"] == 0
    r = bt.info(1)
    assert r["status"] == 2 and r["info"] == 11


@pytest.mark.slow
def test_batched_full_4096(hpl, orc):
    """The batched configuration: 4096 systems, n ~ U{32..512}, half general
    (pivoted FP64), half dominant (BF16 factor + FP64 refinement); every status
    OK and 24 sampled systems checked against the oracle."""
    import torch
    bt = _make(hpl, 1, 4096)
    rng = np.random.default_rng(0)
    sample = np.concatenate([rng.choice(2048, 12, replace=False), 2048 + rng.choice(2048, 12, replace=False)])
    A0 = {int(s): _np(bt.matrix(s)).copy(order="F") for s in sample}
    b0 = {int(s): _np(bt.rhs(s)).copy() for s in sample}
    bt.plan()
    bt.run()
    torch.cuda.synchronize()
    recs = bt.info()
    assert all(r["status"] == 0 for r in recs), [i for i, r in enumerate(recs) if r["status"]][:5]
    for s in sample:
        _check_system(orc, bt, int(s), A0[int(s)], b0[int(s)], emulate=False)


def test_batched_share_matches_whole_batch(hpl):
    """One rank's share of a batch split over two GPUs (Batch with the global
    system ids) generates and solves exactly the systems of the whole batch:
    matrices, solutions and pivots are bit-identical."""
    import torch
    n = hpl.batch_sizes(5, 32)
    kind = np.array([0] * 16 + [1] * 16, dtype=np.uint8)
    whole = hpl.Batch(n, kind)
    whole.generate(5)
    whole.plan()
    whole.run()
    owner = hpl.batch_shard(n, kind, 2)
    for r in (0, 1):
        ids = np.nonzero(owner == r)[0]
        part = hpl.Batch(n[ids], kind[ids], ids=ids)
        part.generate(5)
        part.plan()
        part.run()
        torch.cuda.synchronize()
        for j, g in enumerate(ids):
            assert torch.equal(part.rhs(j), whole.rhs(int(g)))
            if kind[g] == 0:
                assert torch.equal(part.pivots(j), whole.pivots(int(g)))
                assert torch.equal(part.matrix(j), whole.matrix(int(g)))


def test_batched_two_ctas_per_sm_same_results(hpl, orc):
    """A plan whose systems all use 16-wide panels runs two CTAs per SM; the
    one-per-SM kernel gives the same pivots and solutions bit for bit (the same
    per-system code), and both meet the oracle's checks."""
    import torch
    n = np.array([32, 33, 64, 100, 127, 200, 256, 300, 511, 512] * 4, dtype=np.int64)
    kind = np.array([0, 1] * 20, dtype=np.uint8)
    out = []
    try:
        for mode in (0, 1):
            hpl.batched_config(0, mode)
            bt = hpl.Batch(n, kind)
            bt.generate(17)
            if mode == 0:
                A0 = [_np(bt.matrix(s)).copy(order="F") for s in range(bt.count)]
                b0 = [_np(bt.rhs(s)).copy() for s in range(bt.count)]
            bt.plan(variant=1)
            bt.run()
            torch.cuda.synchronize()
            out.append((bt.B.clone(), bt.ipiv.clone(), [r["status"] for r in bt.info()]))
            if mode == 0:
                for s in range(bt.count):
                    _check_system(orc, bt, s, A0[s], b0[s], emulate=False)
    finally:
        hpl.batched_config(0, 0)
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    with pytest.raises(hpl.HplError):
        hpl.batched_config(1, 0)
