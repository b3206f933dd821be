"""Parity of the CUDA search (through the C ABI) with the FP64 oracle.

Bar: |Y_gpu - Y_oracle| <= 1e-5 * max(|Y_oracle|, 1) at every start; the width
index is exact wherever the oracle's best SNR beats its second best by more
than that tolerance, and elsewhere the GPU's width must reach the maximum within
the tolerance.  Sizes span several tiles and a ragged tail.
"""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, RTOL, assert_parity, oracle_grid, recompute_snr, run_gpu, torch

pytestmark = pytest.mark.gpu


def _data(ndm, nt, seed, pulses=True, mu=0.0, sigma=1.0, max_w=300):
    x = spd_synth.gaussian_noise(ndm, nt, seed, mu=mu, sigma=sigma, dtype=np.float64)
    if pulses and nt > max_w + 2:
        n = max(1, ndm * 2)
        tab = spd_synth.pulse_table(n, ndm, nt, seed + 1, width_range=(1, min(max_w, nt - 1)),
                                    snr_range=(6.0, 30.0))
        spd_synth.inject(x, tab, sigma)
    return x.astype(np.float32)


def _check(plan, x, mu, sigma, ctx, **kw):
    Yg, Wg = run_gpu(plan, x, mu, sigma, **kw)
    g = oracle_grid(plan)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, mu, sigma)
    nt = x.shape[1]
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx=ctx)
    # every chosen width is eligible and reaches the maximum within the tolerance
    snr, ok = recompute_snr(x, mu, sigma, g.L, g.Ls, Wg)
    assert ok.all(), ctx
    assert np.all(np.abs(snr - Yo) <= RTOL * np.maximum(np.abs(Yo), 1.0) * 2), ctx
    return Yg, Wg


CASES = [
    # name, s_end, ndm, nt  (IGRID/BoxDIT tiles are 16384 starts; exhaustive 2048)
    ("exh", 256, 3, 9001), ("exh", 64, 2, 4099), ("exh", 1, 2, 513), ("exh", 1000, 2, 5000),
    ("bd8", 8192, 3, 40000), ("bd16", 8192, 2, 40001), ("bd32", 8192, 2, 36003),
    ("bd8", 60, 2, 20000), ("bd16", 300, 2, 18000), ("bd32", 33, 2, 5000), ("bd32", 2000, 2, 33000),
    # BoxDIT: every top level kind -- fine only (top 0..3), first coarse level (K = 8: with
    # remainder blocks; K = 16: aligned; K = 32: base of K - 2 blocks), deepest levels, and
    # rows longer than one 131072-start segment
    ("bd32", 20, 2, 3000), ("bd16", 100, 2, 6000), ("bd8", 200, 2, 17000), ("bd32", 700, 2, 20000),
    ("bd8", 20000, 2, 140000), ("bd32", 20000, 2, 50000), ("bd16", 30000, 1, 140001),
    ("dit", 8192, 3, 40000), ("ig0p2", 4096, 2, 30000), ("ig1p2", 4096, 2, 30000),
    ("ig1", 8192, 3, 50000), ("ig1", 6, 2, 3000), ("ig1", 20, 2, 17000), ("ig1", 5000, 2, 33000),
    ("ig2p4", 4096, 2, 30000), ("ig2", 8192, 3, 40003), ("ig2", 12, 2, 5000),
    ("ig3p8", 4096, 2, 30000), ("ig3", 8192, 2, 40000), ("ig3", 100, 2, 9000),
    # row stride = 4 (mod 8): W rows are only 8-byte aligned on odd rows
    ("ig1", 512, 5, 3900), ("ig2", 8192, 3, 20004), ("bd16", 1000, 3, 20004), ("exh", 200, 3, 6004),
]


@pytest.mark.parametrize("name,s_end,ndm,nt", CASES, ids=["%s-%d-%dx%d" % c for c in CASES])
def test_parity_random(name, s_end, ndm, nt):
    x = _data(ndm, nt, 100 + nt % 97)
    mu = np.linspace(-0.5, 0.5, ndm)
    sigma = np.linspace(0.8, 1.6, ndm)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    _check(plan, x, mu, sigma, "%s s_end=%d" % (name, s_end))


@pytest.mark.parametrize("name", ["exh", "bd32", "ig1", "ig3", "dit"])
@pytest.mark.parametrize("nt", [1, 2, 3, 5, 37, 130])
def test_tiny_rows(name, nt):
    s_end = 64 if name != "exh" else 16
    x = _data(2, nt, 7 + nt, pulses=False)
    plan = spd.spd_plan_create(ndm=2, nt=nt, **ALGOS[name](s_end))
    Yg, Wg = _check(plan, x, 0.0, 1.0, "%s nt=%d" % (name, nt))
    assert np.array_equal(Wg[:, -1], [0, 0])  # the last sample only has width 1


@pytest.mark.parametrize("name", ["bd16", "ig2", "exh"])
def test_row_stride_padding_untouched(name):
    ndm, nt, ld = 3, 20001, 20008
    x = _data(ndm, nt, 3)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, ld=ld, **ALGOS[name](2000 if name != "exh" else 100))
    Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
    assert np.all(Yg[:, nt:] == -12345.0)
    assert np.all(Wg[:, nt:].view(np.int16) == np.int16(54321 - 65536))
    g = oracle_grid(plan)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx=name)


@pytest.mark.parametrize("name", ["bd8", "ig1", "exh"])
def test_unaligned_pointer_scalar_path(name):
    # an x/Y/W base that is not 16-byte aligned takes the scalar load/store path
    ndm, nt = 2, 20000
    x = _data(ndm, nt, 5)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](4096 if name != "exh" else 128))
    Yg, Wg = run_gpu(plan, x, 0.2, 1.3, x_offset=1)
    g = oracle_grid(plan)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, 0.2, 1.3)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx=name)


@pytest.mark.parametrize("name", ["exh", "bd32", "ig1", "ig3", "dit"])
def test_all_zero_input_ties_to_smallest_width(name):
    ndm, nt = 2, 20000
    x = np.zeros((ndm, nt), np.float32)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](1024 if name != "exh" else 50))
    Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
    assert np.all(Yg == 0.0) and np.all(Wg == 0)


@pytest.mark.parametrize("name,s_end", [("bd32", 8000), ("ig1", 8192), ("exh", 256), ("ig3", 8192)])
def test_matched_pulse_recovers_true_snr(name, s_end):
    # Sec. 4.3 / Appendix A: a noise-free rectangular pulse of amplitude C/sqrt(S)
    # matched by a grid width at an eligible start gives exactly SNR C.
    nt = 40000
    plan = spd.spd_plan_create(ndm=1, nt=nt, **ALGOS[name](s_end))
    w, s = plan.widths()
    for S, Lsp in zip(w[:: max(1, len(w) // 12)], s[:: max(1, len(w) // 12)]):
        if S > 8192:
            continue
        t0 = int(Lsp) * ((1000 + int(Lsp) - 1) // int(Lsp))
        x = np.zeros((1, nt), np.float32)
        x[0, t0:t0 + S] = np.float32(10.0 / np.sqrt(S))
        Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
        assert abs(Yg[0, t0] - 10.0) < 1e-4, (name, S)
        assert w[Wg[0, t0]] == S, (name, S, w[Wg[0, t0]])


def test_sec43_pulse_detected_at_start_100():
    # Sec. 4.3: width-20 pulse starting at sample 100, BoxDIT with maximum width 8000:
    # found at start 100 (centre 110) with width 20.
    nt = 20000
    x = spd_synth.gaussian_noise(1, nt, 43, dtype=np.float64) * 0.0
    x[0, 100:120] += 8.0 / np.sqrt(20)
    plan = spd.spd_plan_create(ndm=1, nt=nt, **ALGOS["bd32"](8000))
    Yg, Wg = run_gpu(plan, x.astype(np.float32), 0.0, 1.0)
    w, _ = plan.widths()
    s = int(np.argmax(Yg[0]))
    assert s == 100 and w[Wg[0, s]] == 20 and s + 10 == 110


@pytest.mark.parametrize("name", ["bd8", "bd32", "ig1", "ig2", "ig3", "dit"])
def test_sliding_pulse_within_appendix_bounds(name):
    # Sec. 4.1 measurement on the GPU: one series per pulse shift; max over the
    # series of the highest RSNR equals Eq. RSNRmax, the minimum is >= Eq. RSNRmin.
    s_end = 512
    plan0 = spd.spd_plan_create(ndm=1, nt=100, **ALGOS[name](s_end))
    g = oracle_grid(plan0)
    n_shift = int(g.Ls.max())
    t0 = 2048
    nt = t0 + n_shift + 2 * s_end + 700
    for S in (1, 3, 8, 20, 45, 100, 128, 300):
        x = spd_synth.sliding_pulse_rows(S, n_shift, t0, nt, C=1.0, dtype=np.float32)
        plan = spd.spd_plan_create(ndm=n_shift, nt=nt, **ALGOS[name](s_end))
        Yg, _ = run_gpu(plan, x, 0.0, 1.0)
        best = Yg.max(axis=1).astype(np.float64)
        bmax, bmin = oracle.rsnr_bounds(g, S, 1.0)
        assert abs(best.max() - bmax) < 1e-5, (name, S, best.max(), bmax)
        assert best.min() >= bmin - 1e-5, (name, S, best.min(), bmin)


EXPLICIT = {
    "bd8": lambda: oracle.grid_boxdit(8, 512),
    "ig2": lambda: oracle.grid_igrid(2, 8, 1024),
    "sparse": lambda: oracle.Grid([1, 3, 5, 10, 50, 200, 999], [1, 1, 2, 4, 8, 32, 64]),
}


@pytest.mark.parametrize("name", list(EXPLICIT))
@pytest.mark.parametrize("table", [False, True])
def test_explicit_grid_parity(name, table):
    """spd_plan_create_grid: a caller-given width set with per-width separations
    against the oracle's search of the same grid (several tiles, ragged tail)."""
    g = EXPLICIT[name]()
    ndm, nt = 3, 20011
    x = spd_synth.gaussian_noise(ndm, nt, 71, dtype=np.float64)
    tab = spd_synth.pulse_table(6, ndm, nt, 72, width_range=(1, 400), snr_range=(7.0, 25.0))
    spd_synth.inject(x, tab, 1.0)
    plan = spd.spd_plan_create_grid(g.L, g.Ls, ndm=ndm, nt=nt)
    if table:
        rng = np.random.default_rng(73)
        L = g.L.astype(np.float64)
        mu = 0.1 * L[None, :] + rng.normal(0, 0.05, (ndm, 1)) * L[None, :]
        sg = np.sqrt(L)[None, :] * rng.uniform(0.9, 1.3, (ndm, 1))
        Yg, Wg = run_gpu(plan, x.astype(np.float32), mu, sg, noise_mode=1)
        Yo, Wo, Y2o = oracle.search(x, g, mu, sg, noise_mode=1)
    else:
        Yg, Wg = run_gpu(plan, x.astype(np.float32), 0.0, 1.0)
        Yo, Wo, Y2o = oracle.search(x, g)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="explicit %s" % name)
