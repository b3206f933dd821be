"""The search at the benchmark workloads' full sizes, in the launch configuration
bench.py times.

* exhaustive_small (64 x 65,536, widths 1..256): full element-wise parity.
* ska_mid (4,096 x 1,048,576, IGRID IG(1) / BoxDIT BD-32 / BoxDIT with L^i_max = 12
  on the general kernel's two launches, S_end = 8192): parity on
  sampled rows (the pulse rows, the first and the last), properties that hold at
  any size on every row (Y >= the width-1 SNR, widths in range), and recall of
  the injected pulses through the fused candidate step.
"""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, assert_parity, oracle_grid, run_gpu, torch

pytestmark = pytest.mark.gpu


def test_exhaustive_small_full_parity():
    x, tab = spd_synth.exhaustive_small()
    ndm, nt = x.shape
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS["exh"](256))
    Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), oracle_grid(plan))
    decided = assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="exhaustive_small")
    assert decided > 0.99 * ndm * nt
    # each injected SNR-10 pulse is found at its start with its width (noise permitting)
    hits = 0
    for p in tab:
        r, s, w = int(p["row"]), int(p["start"]), int(p["width"])
        seg = Yg[r, max(0, s - w):s + w]
        hits += int(seg.max() > 7.0)
    assert hits == len(tab)


@pytest.mark.parametrize("name", ["ig1", "bd32", "bd12"])
def test_ska_mid_full_size(name):
    t = torch()
    cfg = spd_synth.SKA_MID
    ndm, nt = cfg["ndm"], cfg["nt"]
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](cfg["s_end"]))
    tab = spd_synth.ska_mid_pulses()
    x = spd_synth.device_noise(ndm, nt, spd_synth.SEED_BASE + 2)
    spd_synth.device_inject(x, tab)
    mu = t.zeros(ndm, device="cuda")
    sg = t.ones(ndm, device="cuda")
    Y = t.empty((ndm, nt), dtype=t.float32, device="cuda")
    W = t.empty((ndm, nt), dtype=t.int16, device="cuda")
    ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
    cap = 1 << 16
    out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.search(plan, x, mu, sg, Y, W, 6.0, 1, out, cnt, ws)
    spd.spd_sync_status(plan, t.cuda.current_stream().cuda_stream)
    n_w = len(plan.widths()[0])
    # properties on every row: width 1 is in every grid, so Y >= z; indices in range
    for r0 in range(0, ndm, 512):
        z = x[r0:r0 + 512]
        assert bool((Y[r0:r0 + 512] >= z - 1e-5 * t.clamp(z.abs(), min=1.0)).all())
        w = W[r0:r0 + 512].to(t.int32) & 0xffff
        assert int(w.max()) < n_w and int(w.min()) >= 0
    # element-wise parity on sampled rows
    rows = sorted({0, ndm - 1} | {int(r) for r in tab["row"][:3]})
    g = oracle_grid(plan)
    xs = x[rows].cpu().numpy()
    Yo, Wo, Y2o = oracle.search(xs.astype(np.float64), g)
    Yg = Y[rows].cpu().numpy()
    Wg = W[rows].cpu().numpy().view(np.uint16)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="ska_mid %s rows %s" % (name, rows))
    # candidates: the strong injected pulses are recalled near their position
    n = int(cnt.item())
    rec = spd.records(out, min(n, cap))
    strong = tab[tab["snr"] >= 9.0]
    found = 0
    for p in strong:
        near = (rec["row"] == p["row"]) & (np.abs(rec["start"] - p["start"]) <= p["width"] + 2 * 8192)
        found += int(near.any())
    assert found >= 0.95 * len(strong), (found, len(strong))
    del x, Y, W
    t.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["f16", "bf16", "u8"])
def test_ska_mid_full_size_stored_types(dtype):
    """The precision workload: the same 4,096 x 1,048,576 series stored as f16,
    bf16 or u8, IG(1): properties on every row, element-wise parity on sampled
    rows against the oracle on the values the stored samples hold."""
    t = torch()
    cfg = spd_synth.SKA_MID
    ndm, nt = cfg["ndm"], cfg["nt"]
    code = {"f16": spd.SPD_F16, "bf16": spd.SPD_BF16, "u8": spd.SPD_U8}[dtype]
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, dtype=code, **ALGOS["ig1"](cfg["s_end"]))
    tab = spd_synth.ska_mid_pulses()
    x = spd_synth.device_noise(ndm, nt, spd_synth.SEED_BASE + 2)
    spd_synth.device_inject(x, tab)
    xs = spd_synth.device_quantize(x, dtype)
    del x
    m0, s0 = (spd_synth.U8_OFFSET, spd_synth.U8_SCALE) if dtype == "u8" else (0.0, 1.0)
    mu = t.full((ndm,), m0, device="cuda")
    sg = t.full((ndm,), s0, device="cuda")
    Y = t.empty((ndm, nt), dtype=t.float32, device="cuda")
    W = t.empty((ndm, nt), dtype=t.int16, device="cuda")
    ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
    spd.execute(plan, xs, mu, sg, Y, W, ws)
    spd.spd_sync_status(plan, t.cuda.current_stream().cuda_stream)
    n_w = len(plan.widths()[0])
    for r0 in range(0, ndm, 512):
        z = (xs[r0:r0 + 512].float() - m0) / s0
        assert bool((Y[r0:r0 + 512] >= z - 1e-5 * t.clamp(z.abs(), min=1.0)).all())
        w = W[r0:r0 + 512].to(t.int32) & 0xffff
        assert int(w.max()) < n_w and int(w.min()) >= 0
    rows = sorted({0, ndm - 1} | {int(r) for r in tab["row"][:2]})
    vals = xs[rows].float().cpu().numpy().astype(np.float64)
    Yo, Wo, Y2o = oracle.search(vals, oracle_grid(plan), m0, s0)
    Yg = Y[rows].cpu().numpy()
    Wg = W[rows].cpu().numpy().view(np.uint16)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="ska_mid %s rows %s" % (dtype, rows))


def test_batched_full_size():
    """The batched workload at full size: 1024/1024/768/512/256 DM trials at
    decimations 1/2/4/8/16 of 2,097,152 samples, BD-16 with S_end = 4,096 in one
    persistent launch (segment 262,144, the bench's tuned choice): properties on
    every row, parity on the first and last row of every range."""
    t = torch()
    shapes = [(1024, 2097152), (1024, 1048576), (768, 524288), (512, 262144), (256, 131072)]
    b = spd.spd_batch_create(spd.SPD_ALGO_BOXDIT, 4096, [n for n, _ in shapes], [m for _, m in shapes],
                             boxdit_lmax=16)
    b.set_segment(262144)
    xs, ys, wis = [], [], []
    for r, (n, m) in enumerate(shapes):
        x = spd_synth.device_noise(n, m, spd_synth.SEED_BASE + 4 + 100 * r)
        tab = spd_synth.pulse_table(100, n, m, spd_synth.SEED_BASE + 5 + 100 * r, width_range=(1, 4096),
                                    snr_range=(6.0, 20.0), min_gap=2 * 4600)
        spd_synth.device_inject(x, tab)
        xs.append(x)
        ys.append(t.empty((n, m), dtype=t.float32, device="cuda"))
        wis.append(t.empty((n, m), dtype=t.int16, device="cuda"))
    mus = [t.zeros(n, device="cuda") for n, _ in shapes]
    sgs = [t.ones(n, device="cuda") for n, _ in shapes]
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    spd.batch_execute(b, xs, ys, wis, mus, sgs, ws)
    spd.spd_batch_status(b, ws.data_ptr(), t.cuda.current_stream().cuda_stream)
    for r, (n, m) in enumerate(shapes):
        plan = spd.spd_plan_create(ndm=n, nt=m, algo=spd.SPD_ALGO_BOXDIT, s_end=4096, boxdit_lmax=16)
        n_w = len(plan.widths()[0])
        for r0 in range(0, n, 256):
            z = xs[r][r0:r0 + 256]
            assert bool((ys[r][r0:r0 + 256] >= z - 1e-5 * t.clamp(z.abs(), min=1.0)).all())
            w = wis[r][r0:r0 + 256].to(t.int32) & 0xffff
            assert int(w.max()) < n_w and int(w.min()) >= 0
        rows = [0, n - 1]
        Yo, Wo, Y2o = oracle.search(xs[r][rows].cpu().numpy().astype(np.float64), oracle_grid(plan))
        assert_parity(ys[r][rows].cpu().numpy(), wis[r][rows].cpu().numpy().view(np.uint16), Yo, Wo, Y2o, m,
                      ctx="batched range %d rows %s" % (r, rows))


def test_proposal_restricted_search_full_size():
    """The proposal workload at full size (4,096 x 1,048,576 f16, white + 1/f
    noise + zero-DM spikes + pulses, BD-16 with table noise): the restricted
    search of 2 % of the blocks gives exactly the plain search's candidates in
    those blocks."""
    from paper_1910_08324_gb300 import proposal as P
    t = torch()
    ndm, nt = 4096, 1 << 20
    grid = dict(algo=spd.SPD_ALGO_BOXDIT, s_end=4096, boxdit_lmax=16, dtype=spd.SPD_F16)
    pulses = spd_synth.pulse_table(500, ndm, nt, 611, width_range=(1, 2048), snr_range=(5.0, 20.0), min_gap=16384)
    x, _ = spd_synth.proposal_series(ndm, nt, 612)
    spd_synth.device_inject_many(x, pulses, amp=spd_synth.proposal_amplitudes(pulses, nt))
    x = x.half()
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **grid)
    nw = len(plan.widths()[0])
    mu = t.empty((ndm, nw), device="cuda")
    sg = t.empty((ndm, nw), device="cuda")
    ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
    spd.noise_stats(plan, x, mu, sg, ws)
    Y = t.empty((ndm, nt), device="cuda")
    W = t.empty((ndm, nt), dtype=t.int16, device="cuda")
    cap = 1 << 23
    out = t.empty(cap * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.search(plan, x, mu, sg, Y, W, 6.0, 1, out, cnt, ws, noise_mode=1)
    k = int(cnt.item())
    assert k <= cap
    ref = spd.records(out, k).copy()
    del Y, W
    bpr = nt // P.BLOCK
    rng = np.random.default_rng(613)
    pulse_blocks = pulses["row"] * bpr + pulses["start"] // P.BLOCK
    sel = np.unique(np.concatenate([rng.choice(ndm * bpr, ndm * bpr // 50, replace=False), pulse_blocks,
                                    [0, bpr - 1, ndm * bpr - 1]]))
    rec = P.search_flagged(x, t.as_tensor(sel, device="cuda"), mu, sg, grid, threshold=6.0, radius=1,
                           noise_mode=1)
    keep = np.isin(ref["row"].astype(np.int64) * bpr + ref["start"] // P.BLOCK, sel)
    assert len(rec) > 1000 and np.array_equal(rec, ref[keep])
