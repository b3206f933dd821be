"""Proposal path on the GPU: block selection and gather against numpy, the
restricted search equal to the plain search on the selected blocks, and what a
network trained on the GPU gains over the plain search on red noise with
zero-DM spikes, judged by the ideal exhaustive search of the FP64 CPU oracle on
each pulse's neighbourhood (the GPU's exhaustive judge is checked against it)."""
import numpy as np
import pytest

import oracle

import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import torch
from oracle import net
from paper_1910_08324_gb300 import proposal as P

pytestmark = pytest.mark.gpu

NEG_INF_BITS = {"f32": 0xff800000, "f16": 0xfc00, "bf16": 0xff80}


def test_select_matches_threshold():
    t = torch()
    rng = np.random.default_rng(1)
    for n in (1, 31, 1000, 70001):
        lg = rng.normal(size=n).astype(np.float32)
        ids = P.select_blocks(t.from_numpy(lg).cuda(), 0.5)
        assert np.array_equal(ids.cpu().numpy(), np.nonzero(lg > 0.5)[0])
    ids = P.select_blocks(t.full((100,), -1.0, device="cuda"), 0.0)
    assert ids.numel() == 0
    # more than 256 tiles of 8192 (larger tiles), and a list shorter than the count
    lg = rng.normal(size=3_000_001).astype(np.float32)
    ref = np.nonzero(lg > 1.0)[0]
    d = t.from_numpy(lg).cuda()
    assert np.array_equal(P.select_blocks(d, 1.0).cpu().numpy(), ref)
    out = t.full((1000,), -7, dtype=t.int64, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.net_select(d, 1.0, out, cnt)
    assert int(cnt.item()) == len(ref) and np.array_equal(out.cpu().numpy(), ref[:1000])


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_gather_matches_numpy(dtype):
    t = torch()
    ndm, nt, ld, block = 3, 4096 * 3 + 1000, 4096 * 3 + 1024, 4096
    tdt, code, bits = {"f32": (t.float32, spd.SPD_F32, np.uint32), "f16": (t.float16, spd.SPD_F16, np.uint16),
                       "bf16": (t.bfloat16, spd.SPD_BF16, np.uint16)}[dtype]
    x = t.randn((ndm, ld), generator=t.Generator().manual_seed(3)).to(tdt).cuda()
    bpr = -(-nt // block)
    ids_h = np.array([0, 5, 3, 11, 999, 7, 4], np.int64)  # 999 lies outside the series
    for left, right in ((0, 0), (256, 4336), (8, 40)):
        width = left + block + right
        ldo = -(-width // 64) * 64
        out = t.empty((len(ids_h), ldo), dtype=tdt, device="cuda")
        spd.net_gather(x, t.as_tensor(ids_h, device="cuda"), len(ids_h), block, left, width, out, dtype=code, nt=nt)
        xb = x.cpu().view(t.int32 if dtype == "f32" else t.int16).numpy().view(bits)
        ref = np.full((len(ids_h), ldo), NEG_INF_BITS[dtype], bits)
        for k, i in enumerate(ids_h):
            if i >= ndm * bpr:
                continue
            r, b = divmod(int(i), bpr)
            for c in range(width):
                q = b * block - left + c
                if 0 <= q < nt:
                    ref[k, c] = xb[r, q]
        got = out.cpu().view(t.int32 if dtype == "f32" else t.int16).numpy().view(bits)
        assert np.array_equal(got, ref), (left, right)


GRIDS = {
    "bd16_f16_table": (dict(algo=spd.SPD_ALGO_BOXDIT, s_end=4096, boxdit_lmax=16, dtype=spd.SPD_F16), 1),
    "ig1_f32_white": (dict(algo=spd.SPD_ALGO_IGRID, s_end=4096, igrid_depth=1, igrid_layers=4,
                           dtype=spd.SPD_F32), 0),
    "exh_f16_white": (dict(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=512, dtype=spd.SPD_F16), 0),
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_search_flagged_equals_plain_search_on_those_blocks(name):
    """The restricted search of a set of blocks gives exactly the candidates the
    plain search of the whole series gives in those blocks."""
    t = torch()
    grid, mode = GRIDS[name]
    ndm, nt = 6, 16 * P.BLOCK
    x = spd_synth.device_noise(ndm, nt, 77)
    tab = spd_synth.pulse_table(40, ndm, nt, 78, width_range=(1, 2048), snr_range=(6, 30))
    spd_synth.device_inject_many(x, tab)
    xs = x if grid["dtype"] == spd.SPD_F32 else x.half()
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **grid)
    ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
    if mode == 1:
        nw = len(plan.widths()[0])
        mu, sg = t.empty((ndm, nw), device="cuda"), t.empty((ndm, nw), device="cuda")
        spd.noise_stats(plan, xs, mu, sg, ws)
    else:
        mu, sg = t.zeros(ndm, device="cuda"), t.ones(ndm, device="cuda")
    Y = t.empty((ndm, nt), device="cuda")
    W = t.empty((ndm, nt), dtype=t.int16, device="cuda")
    cap = 1 << 18
    out = t.empty(cap * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.search(plan, xs, mu, sg, Y, W, 3.0, 2, out, cnt, ws, noise_mode=mode)
    ref = spd.records(out, int(cnt.item())).copy()
    rng = np.random.default_rng(5)
    bpr = nt // P.BLOCK
    sel = np.unique(np.concatenate([rng.choice(ndm * bpr, 30, replace=False), [0, bpr - 1, ndm * bpr - 1]]))
    rec = P.search_flagged(xs, t.as_tensor(sel, device="cuda"), mu, sg, grid, threshold=3.0, radius=2,
                           noise_mode=mode)
    keep = np.isin(ref["row"].astype(np.int64) * bpr + ref["start"] // P.BLOCK, sel)
    assert len(rec) > 50
    assert np.array_equal(rec, ref[keep])


GRIDS_ABI = dict(GRIDS)
GRIDS_ABI["bd12_f32_table"] = (dict(algo=spd.SPD_ALGO_BOXDIT, s_end=3000, boxdit_lmax=12, dtype=spd.SPD_F32), 1)


@pytest.mark.parametrize("name", list(GRIDS_ABI))
def test_propose_search_abi_equals_plain_search_on_flagged_blocks(name):
    """spd_propose_search (network, selection, gather, search and the record map
    all on the device) gives exactly the plain search's candidates in the blocks
    the network flags, in the series' (row, start) order."""
    t = torch()
    grid, mode = GRIDS_ABI[name]
    ndm, nt = 6, 16 * P.BLOCK
    x = spd_synth.device_noise(ndm, nt, 91)
    tab = spd_synth.pulse_table(40, ndm, nt, 92, width_range=(1, 2048), snr_range=(6, 30))
    spd_synth.device_inject_many(x, tab)
    xs = x if grid["dtype"] == spd.SPD_F32 else x.half()
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **grid)
    ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
    nw = len(plan.widths()[0])
    if mode == 1:
        mu, sg = t.empty((ndm, nw), device="cuda"), t.empty((ndm, nw), device="cuda")
        spd.noise_stats(plan, xs, mu, sg, ws)
    else:
        mu, sg = t.zeros(ndm, device="cuda"), t.ones(ndm, device="cuda")
    Y = t.empty((ndm, nt), device="cuda")
    W = t.empty((ndm, nt), dtype=t.int16, device="cuda")
    cap = 1 << 18
    out = t.empty(cap * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.search(plan, xs, mu, sg, Y, W, 3.0, 2, out, cnt, ws, noise_mode=mode)
    ref = spd.records(out, int(cnt.item())).copy()
    params = t.from_numpy(net.init_params(11)).cuda()
    # the blocks the network flags, from the separate calls
    mu1 = (mu[:, 0] if mode == 1 else mu).contiguous()
    sg1 = (sg[:, 0] if mode == 1 else sg).contiguous()
    logits, _ = P.flag_blocks(params, xs, mu1, sg1, dtype=grid["dtype"])
    thr = float(np.quantile(logits.cpu().numpy(), 0.6))
    sel = P.select_blocks(logits, thr).cpu().numpy()
    assert 10 < len(sel) < ndm * (nt // P.BLOCK)
    prop = spd.spd_proposal_create(ndm=ndm, nt=nt, peak_radius=2, max_blocks=64, **grid)
    assert np.array_equal(prop.widths()[0], plan.widths()[0])
    pws = t.empty(prop.workspace_size(), dtype=t.uint8, device="cuda")
    pout = t.empty(cap * 24, dtype=t.uint8, device="cuda")
    pcnt = t.full((1,), -1, dtype=t.int64, device="cuda")
    nb = spd.propose_search(prop, params, xs, mu, sg, pout, pcnt, pws, logit_threshold=thr, threshold=3.0,
                            noise_mode=mode)
    assert nb == len(sel)
    rec = spd.records(pout, int(pcnt.item()))
    keep = np.isin(ref["row"].astype(np.int64) * (nt // P.BLOCK) + ref["start"] // P.BLOCK, sel)
    assert len(rec) > 20
    assert np.array_equal(rec, ref[keep])
    # a short record buffer keeps the first records and the true count
    short = t.empty(7 * 24, dtype=t.uint8, device="cuda")
    spd.propose_search(prop, params, xs, mu, sg, short, pcnt, pws, logit_threshold=thr, threshold=3.0,
                       noise_mode=mode)
    assert int(pcnt.item()) == len(rec) and np.array_equal(spd.records(short, 7), rec[:7])
    # nothing flagged: no records; more flagged blocks than max_blocks: refused
    assert spd.propose_search(prop, params, xs, mu, sg, pout, pcnt, pws, logit_threshold=1e30,
                              noise_mode=mode) == 0
    assert int(pcnt.item()) == 0
    with pytest.raises(spd.SpdError) as e:
        spd.propose_search(prop, params, xs, mu, sg, pout, pcnt, pws, logit_threshold=-1e30, noise_mode=mode)
    assert e.value.status == 5


def oracle_pulse_snr(x, pulses, mu, sigma, plan, width_ratio=4.0):
    """The ideal search's SNR of each injected pulse, from the FP64 oracle: the
    exhaustive grid of ``plan`` searched (table noise mu, sigma of the pulse's row)
    over the pulse's neighbourhood [s0 - w, s0 + w] plus the widest boxcar past
    it; the largest SNR at a start in [s0 - w, s0 + w] whose best width lies
    within a factor ``width_ratio`` of w (0 where none), as ``proposal.pulse_snr``.
    Windows of one length go to the oracle together (its threads split rows)."""
    w_tab, s_tab = plan.widths()
    g = oracle.Grid(w_tab, s_tab)
    lend = int(w_tab[-1])
    nt = x.shape[1]
    mu_h, sg_h = mu.cpu().numpy().astype(np.float64), sigma.cpu().numpy().astype(np.float64)
    rows = pulses["row"].astype(np.int64)
    s0 = pulses["start"].astype(np.int64)
    w = pulses["width"].astype(np.int64)
    a = np.maximum(s0 - w, 0)
    span = int(2 * w.max() + 1 + lend)
    a = np.minimum(a, max(nt - span, 0))  # the window stays inside the row (it still covers the pulse)
    n = min(span, nt)
    xh = x.float().cpu().numpy()
    xs = np.stack([xh[r, i:i + n] for r, i in zip(rows, a)]).astype(np.float64)
    Y, W, _ = oracle.search(xs, g, mu_h[rows], sg_h[rows], noise_mode=1)
    out = np.zeros(len(pulses))
    for k in range(len(pulses)):
        j = np.arange(max(s0[k] - w[k], 0) - a[k], min(s0[k] + w[k] - a[k], n - 1) + 1)
        cw = w_tab[W[k, j]].astype(np.float64)
        ok = (cw <= width_ratio * w[k]) & (cw * width_ratio >= w[k])
        out[k] = max(0.0, float(Y[k, j][ok].max())) if ok.any() else 0.0
    return out


def test_trained_network_gain_on_red_noise_with_spikes():
    """Train the network on the GPU (labels from the plain BoxDIT search), then
    search only the blocks it flags.  Against the plain search of every block,
    judged by the ideal exhaustive search: far fewer false alarms and blocks
    searched, most pulses kept, and the same SNR loss on those found."""
    t = torch()
    nt = 1 << 20
    grid = dict(algo=spd.SPD_ALGO_BOXDIT, s_end=4096, boxdit_lmax=16, dtype=spd.SPD_F16)
    gx = dict(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=2048, dtype=spd.SPD_F16)

    def series(ndm, seed, pulses):
        x, _ = spd_synth.proposal_series(ndm, nt, seed)
        spd_synth.device_inject_many(x, pulses, amp=spd_synth.proposal_amplitudes(pulses, nt))
        return x.half()

    def tables(g, x):
        plan = spd.spd_plan_create(ndm=x.shape[0], nt=nt, **g)
        nw = len(plan.widths()[0])
        mu = t.empty((x.shape[0], nw), device="cuda")
        sg = t.empty((x.shape[0], nw), device="cuda")
        ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
        spd.noise_stats(plan, x, mu, sg, ws)
        return plan, mu, sg, ws

    def plain(plan, x, mu, sg, ws):
        Y = t.empty(x.shape, device="cuda")
        W = t.empty(x.shape, dtype=t.int16, device="cuda")
        cap = 1 << 24
        out = t.empty(cap * 24, dtype=t.uint8, device="cuda")
        cnt = t.zeros(1, dtype=t.int64, device="cuda")
        spd.search(plan, x, mu, sg, Y, W, 6.0, 1, out, cnt, ws, noise_mode=1)
        k = int(cnt.item())
        assert k <= cap
        return spd.records(out, k).copy()

    # training blocks: half hold one pulse, labelled by the plain search
    ntr = 512
    ptr = spd_synth.block_pulses(ntr, nt, P.BLOCK, 21, frac=0.5)
    xtr = series(ntr, 22, ptr)
    plan, mu, sg, ws = tables(grid, xtr)
    y = P.label_blocks(plain(plan, xtr, mu, sg, ws), ptr, ntr, nt)
    X = P.decimated_blocks(xtr, mu[:, 0].contiguous(), sg[:, 0].contiguous(), dtype=spd.SPD_F16)
    del xtr, plan
    params = t.from_numpy(net.init_params(3)).cuda()
    losses, _, _ = P.train(params, X, t.from_numpy(y).cuda(), steps=4000, batch=512, lr=3e-3)
    del X
    assert np.mean(losses[-100:]) < 0.5 * np.mean(losses[:20])

    # held-out series: a pulse in one block of 16
    nev = 128
    pev = spd_synth.block_pulses(nev, nt, P.BLOCK, 31, frac=1 / 16)
    xev = series(nev, 32, pev)
    plan, mu, sg, ws = tables(grid, xev)
    planx, mux, sgx, _ = tables(gx, xev)
    sj_gpu = P.pulse_snr(xev, pev, mux, sgx, gx)
    sj = oracle_pulse_snr(xev, pev, mux, sgx, planx)
    # the GPU's exhaustive judge equals the oracle's (parity bar of the search)
    assert np.all(np.abs(sj_gpu - sj) <= 1e-5 * np.maximum(np.abs(sj), 1.0)), np.abs(sj_gpu - sj).max()
    s_plain = P.score(plain(plan, xev, mu, sg, ws), pev, sj, nev, nt)
    rec, nsearched = P.propose_and_search(params, xev, mu, sg, grid, logit_threshold=0.0)
    s_prop = P.score(rec, pev, sj, nev, nt)
    frac = nsearched / (nev * (nt // P.BLOCK))
    print("\nplain:", s_plain, "\nproposal:", s_prop, "\nblocks searched: %.4f" % frac)
    assert s_plain["judge_found"] >= 0.9 * len(pev)
    assert s_plain["recall"] >= 0.98 and s_plain["snr_loss"] <= 0.07
    assert frac <= 0.2
    assert s_prop["recall"] >= 0.75
    assert s_prop["recall_w16_256"] >= 0.95 and s_prop["recall_w256_4096"] >= 0.95
    assert s_prop["snr_loss"] <= 0.07
    assert s_prop["false_alarms"] <= 0.1 * s_plain["false_alarms"]


def test_training_resumes_from_a_checkpoint(tmp_path):
    """30 Adam steps straight equal 15 steps, a checkpoint written and read back,
    and 15 more, bit for bit (the batch schedule is a function of the step and
    the gradient is summed over the CTAs in a fixed order)."""
    t = torch()
    rng = np.random.default_rng(11)
    X = t.from_numpy(rng.normal(size=(2048, 256)).astype(np.float32)).cuda()
    y = t.from_numpy((rng.random(2048) < 0.5).astype(np.float32)).cuda()
    X[y > 0.5, 100:120] += 2.0
    p0 = t.from_numpy(spd_synth.net_init_params(5)).cuda()
    pa = p0.clone()
    la, ma, va = P.train(pa, X, y, steps=30, batch=256, lr=3e-3, seed=4)
    pb = p0.clone()
    lb, mb, vb = P.train(pb, X, y, steps=15, batch=256, lr=3e-3, seed=4)
    P.save_checkpoint(tmp_path / "c.ckpt", pb, mb, vb, step=15, seed=4)
    pc, mc, vc, step, seed = P.load_checkpoint(tmp_path / "c.ckpt")
    lc, _, _ = P.train(pc, X, y, steps=30 - step, batch=256, lr=3e-3, seed=seed, m=mc, v=vc, step0=step)
    assert la[:15] == lb and la[15:] == lc
    assert t.equal(pa, pc) and t.equal(ma, mc) and t.equal(va, vc)
