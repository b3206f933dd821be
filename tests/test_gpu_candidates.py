"""Candidate selection on the GPU (threshold + peak finding) through the C ABI.

The rule decides integers from floats, so both sides take the decision on the
same float32 SNRs: the oracle's rule is run on the GPU's Y and the record lists
must be identical (bit-exact).  The fused spd_search must equal spd_execute
followed by spd_candidates.
"""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, run_gpu, torch

pytestmark = pytest.mark.gpu


def _gpu_cands(plan, Y, W, thr, R, ws, cap):
    t = torch()
    out = t.zeros(max(cap, 1) * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.candidates(plan, Y, W, thr, R, out if cap > 0 else None, cnt, ws)
    t.cuda.synchronize()
    n = int(cnt.item())
    return n, spd.records(out, min(n, cap))


def _setup(name="ig1", s_end=2048, ndm=5, nt=70001, seed=11, n_pulses=12):
    x = spd_synth.gaussian_noise(ndm, nt, seed, dtype=np.float64)
    tab = spd_synth.pulse_table(n_pulses, ndm, nt, seed + 3, width_range=(1, 1000), snr_range=(8, 25),
                                min_gap=4096)
    spd_synth.inject(x, tab)
    x = x.astype(np.float32)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    Yh, Wh, dev = run_gpu(plan, x, 0.0, 1.0, return_ws=True)
    return plan, x, Yh, Wh, dev, tab


@pytest.mark.parametrize("R", [0, 1, 5, 64])
@pytest.mark.parametrize("thr", [3.0, 5.0])
def test_candidates_match_oracle_rule_on_gpu_snr(R, thr):
    plan, x, Yh, Wh, (Y, W, ws, *_), _ = _setup()
    w, _ = plan.widths()
    n, rec = _gpu_cands(plan, Y, W, thr, R, ws, cap=1 << 20)
    no, rows, starts, widx, snr = oracle.candidates(Yh.astype(np.float64), Wh.astype(np.int32), thr, R)
    assert n == no
    assert np.array_equal(rec["row"], rows) and np.array_equal(rec["start"], starts)
    assert np.array_equal(rec["width_idx"], widx) and np.array_equal(rec["snr"], snr.astype(np.float32))
    assert np.array_equal(rec["width"], w[rec["width_idx"]])


def test_truncation_keeps_first_records_and_true_count():
    plan, x, Yh, Wh, (Y, W, ws, *_), _ = _setup()
    n_all, rec_all = _gpu_cands(plan, Y, W, 3.0, 0, ws, cap=1 << 20)
    assert n_all > 20
    n, rec = _gpu_cands(plan, Y, W, 3.0, 0, ws, cap=17)
    assert n == n_all and len(rec) == 17 and np.array_equal(rec, rec_all[:17])
    n0, _ = _gpu_cands(plan, Y, W, 3.0, 0, ws, cap=0)
    assert n0 == n_all


def test_candidates_status_reports_overflow_synchronously():
    # the candidate call itself returns SPD_OK; spd_candidates_status waits for the
    # stream and turns a count above cap into SPD_ERR_BUFFER_TOO_SMALL
    t = torch()
    plan, x, Yh, Wh, (Y, W, ws, *_), _ = _setup()
    out = t.zeros(17 * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.candidates(plan, Y, W, 3.0, 0, out, cnt, ws)
    stream = t.cuda.current_stream().cuda_stream
    with pytest.raises(spd.SpdError) as e:
        spd.spd_candidates_status(cnt.data_ptr(), 17, stream)
    assert e.value.status == 5  # SPD_ERR_BUFFER_TOO_SMALL
    n = int(cnt.item())
    assert n > 17 and spd.spd_candidates_status(cnt.data_ptr(), n, stream) == n


@pytest.mark.parametrize("name,s_end", [("ig1", 8192), ("bd16", 8192), ("exh", 256), ("ig3", 512)])
def test_fused_search_equals_execute_then_candidates(name, s_end):
    t = torch()
    plan, x, Yh, Wh, (Y, W, ws, mu_d, sg_d, xv), tab = _setup(name, s_end, ndm=4, nt=50000)
    n1, rec1 = _gpu_cands(plan, Y, W, 6.0, 2, ws, cap=4096)
    Y2 = t.empty_like(Y)
    W2 = t.empty_like(W)
    out = t.zeros(4096 * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.search(plan, xv, mu_d, sg_d, Y2, W2, 6.0, 2, out, cnt, ws)
    t.cuda.synchronize()
    n2 = int(cnt.item())
    assert n2 == n1 and np.array_equal(spd.records(out, min(n2, 4096)), rec1)
    assert t.equal(Y2[:, :plan.nt], Y[:, :plan.nt]) and t.equal(W2[:, :plan.nt], W[:, :plan.nt])
    # every injected pulse (SNR >= 8) gives a candidate close to it
    for p in tab:
        near = (rec1["row"] == p["row"]) & (np.abs(rec1["start"] - p["start"]) <= p["width"] + 64)
        assert near.any(), p


def test_no_candidates_when_threshold_above_everything():
    plan, x, Yh, Wh, (Y, W, ws, *_), _ = _setup()
    n, rec = _gpu_cands(plan, Y, W, 1e9, 1, ws, cap=16)
    assert n == 0 and len(rec) == 0


@pytest.mark.parametrize("name,s_end,table", [("exh", 256, False), ("bd16", 4096, True), ("ig1", 4096, False),
                                              ("dit", 4096, False), ("ig3", 2048, False), ("bd8", 2048, False)])
def test_fewer_starts_than_samples(name, s_end, table):
    """spd_plan_set_starts: the first n_starts starts get exactly the outputs of a
    plan over every start, later starts are not written, and the candidates equal
    the full plan's away from the new row end."""
    t = torch()
    ndm, nt, ns, R = 3, 50000, 30001, 2
    x = spd_synth.gaussian_noise(ndm, nt, 31, dtype=np.float64)
    tab = spd_synth.pulse_table(6, ndm, nt, 32, width_range=(1, 300), snr_range=(7.0, 20.0))
    spd_synth.inject(x, tab, 1.0)
    xd = t.from_numpy(x.astype(np.float32)).cuda()
    full = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    part = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    if name != "exh":
        for pl in (full, part):
            spd.spd_plan_set_segment(pl, 16384)  # several segments per row
    spd.spd_plan_set_starts(part, ns)
    if table:
        nw = len(full.widths()[0])
        mu, sg = t.empty((ndm, nw), device="cuda"), t.empty((ndm, nw), device="cuda")
        ws0 = t.empty(full.workspace_size(), dtype=t.uint8, device="cuda")
        spd.noise_stats(full, xd, mu, sg, ws0)
    else:
        mu, sg = t.zeros(ndm, device="cuda"), t.ones(ndm, device="cuda")
    mode = 1 if table else 0
    res = []
    for pl in (full, part):
        Y = t.full((ndm, nt), -12345.0, device="cuda")
        W = t.full((ndm, nt), 777, dtype=t.int16, device="cuda")
        ws = t.empty(pl.workspace_size(), dtype=t.uint8, device="cuda")
        out = t.empty(8192 * 24, dtype=t.uint8, device="cuda")
        cnt = t.zeros(1, dtype=t.int64, device="cuda")
        spd.search(pl, xd, mu, sg, Y, W, 5.0, R, out, cnt, ws, noise_mode=mode)
        k = int(cnt.item())
        assert k <= 8192
        res.append((Y.cpu().numpy(), W.cpu().numpy(), spd.records(out, k).copy()))
    (Yf, Wf, rf), (Yp, Wp, rp) = res
    assert np.array_equal(Yp[:, :ns], Yf[:, :ns]) and np.array_equal(Wp[:, :ns], Wf[:, :ns])
    assert np.all(Yp[:, ns:] == -12345.0) and np.all(Wp[:, ns:] == 777)
    near_end = lambda r: r["start"] >= ns - R
    assert not np.any(rp["start"] >= ns)
    assert np.array_equal(rp[~near_end(rp)], rf[(rf["start"] < ns) & ~near_end(rf)])
    assert len(rp) >= 1 and len(rf) >= len(rp)
