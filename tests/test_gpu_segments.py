"""Segment seams of the streaming kernels against the FP64 oracle.

A BoxDIT or IGRID plan splits each row into segments searched by separate CTAs,
each reading the widest boxcar past its end again (the halo).  With
spd_plan_set_segment(plan, 16384) a row of 70 000 - 140 000 samples crosses five to
nine seams, so every grid's halo, segment start and backwards chunk walk is
compared element by element with the oracle (Eq. boxcar, Eq. SNRlong), with white
and with table noise.  Pulses of up to 4 000 samples are placed across the seams.
The exhaustive kernel has no segments; its 2 048-start tiles are crossed by the
same rows.
"""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, assert_parity, oracle_grid, recompute_snr, run_gpu, RTOL

pytestmark = pytest.mark.gpu

SEG = 16384
GRIDS = ["bd8", "bd16", "bd32", "dit", "ig0p2", "ig1p2", "ig1", "ig2p4", "ig2", "ig3p8", "ig3"]
CASES = [(g, 8192, 140000) for g in GRIDS] + [(g, 1500, 70001) for g in GRIDS]


def _series(ndm, nt, seed):
    x = spd_synth.gaussian_noise(ndm, nt, seed, dtype=np.float64)
    # pulses straddling the seams (a start shortly before a multiple of the segment)
    seams = np.arange(SEG, nt - 4100, SEG)
    rows, starts, widths, snrs = [], [], [], []
    g = np.random.default_rng(seed + 1)
    for k, b in enumerate(seams):
        w = int([3, 40, 700, 4000][k % 4])
        rows.append(k % ndm)
        starts.append(int(b - w // 2 - g.integers(0, 3)))
        widths.append(w)
        snrs.append(float(g.uniform(8.0, 25.0)))
    tab = np.zeros(len(rows), spd_synth.PULSE_DTYPE)
    tab["row"], tab["start"], tab["width"], tab["snr"] = rows, starts, widths, snrs
    spd_synth.inject(x, tab, 1.0)
    return x


def _tables(widths, ndm, seed):
    L = np.asarray(widths, np.float64)[None, :]
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, (ndm, 1))
    muL = (0.05 * L + 0.3 * np.sqrt(L) * u).astype(np.float32)
    sgL = (np.linspace(0.9, 1.4, ndm).reshape(-1, 1) * L ** 0.6).astype(np.float32)
    return muL, sgL


@pytest.mark.parametrize("noise", ["white", "table"])
@pytest.mark.parametrize("name,s_end,nt", CASES, ids=["%s-%d-%d" % c for c in CASES])
def test_segment_seams_parity(name, s_end, nt, noise):
    ndm = 2
    x = _series(ndm, nt, 500 + nt % 101 + len(name))
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    spd.spd_plan_set_segment(plan, SEG)
    g = oracle_grid(plan)
    assert g.L[-1] <= 2 * SEG  # the widest boxcar reaches past the next seam
    if noise == "white":
        mu = np.array([0.2, -0.1])
        sg = np.array([1.1, 0.9])
        xs = x * sg.reshape(-1, 1) + mu.reshape(-1, 1)
        xs = xs.astype(np.float32)
        Yg, Wg = run_gpu(plan, xs, mu, sg)
        Yo, Wo, Y2o = oracle.search(xs.astype(np.float64), g, mu, sg)
    else:
        mu, sg = _tables(g.L, ndm, nt)
        xs = x.astype(np.float32)
        Yg, Wg = run_gpu(plan, xs, mu, sg, noise_mode=1)
        Yo, Wo, Y2o = oracle.search(xs.astype(np.float64), g, mu.astype(np.float64), sg.astype(np.float64),
                                    noise_mode=1)
    ctx = "%s s_end=%d nt=%d %s, %d segments" % (name, s_end, nt, noise, -(-nt // SEG))
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx=ctx)
    if noise == "white":
        snr, ok = recompute_snr(xs, mu, sg, g.L, g.Ls, Wg)
        assert ok.all(), ctx
        assert np.all(np.abs(snr - Yo) <= 2 * RTOL * np.maximum(np.abs(Yo), 1.0)), ctx


@pytest.mark.parametrize("noise", ["white", "table"])
def test_exhaustive_tile_seams_parity(noise):
    ndm, nt = 2, 70001
    x = _series(ndm, nt, 909)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS["exh"](300))
    g = oracle_grid(plan)
    xs = x.astype(np.float32)
    if noise == "white":
        Yg, Wg = run_gpu(plan, xs, 0.0, 1.0)
        Yo, Wo, Y2o = oracle.search(xs.astype(np.float64), g)
    else:
        mu, sg = _tables(g.L, ndm, 3)
        Yg, Wg = run_gpu(plan, xs, mu, sg, noise_mode=1)
        Yo, Wo, Y2o = oracle.search(xs.astype(np.float64), g, mu.astype(np.float64), sg.astype(np.float64),
                                    noise_mode=1)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="exh %s" % noise)
