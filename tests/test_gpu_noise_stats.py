"""spd_noise_stats (Sec. 4.5 mean and standard deviation with outlier rejection at
power-of-two decimations, interpolated per width) against the FP64 oracle, and
the table it produces driving a table-noise search."""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, assert_parity, oracle_grid, run_gpu, torch

pytestmark = pytest.mark.gpu


def _nlev(lend):
    n = 1
    while n < 16 and (1 << (n - 1)) < lend:
        n += 1
    return n


def _rows(ndm, nt, seed, spikes=0.002):
    x = spd_synth.gaussian_noise(ndm, nt, seed, dtype=np.float64)
    x = x * np.linspace(0.8, 1.5, ndm)[:, None] + np.linspace(-1.0, 2.0, ndm)[:, None]
    rng = np.random.default_rng(seed)
    for r in range(ndm):
        idx = rng.choice(nt, int(spikes * nt), replace=False)
        x[r, idx] += rng.uniform(8.0, 40.0, idx.size)  # impulsive interference
    return x


def _gpu_table(plan, stored, thr, passes):
    t = torch()
    ndm, nt = stored.shape
    host = t.from_numpy(np.ascontiguousarray(stored).view(np.int16) if stored.dtype == np.uint16
                        else np.ascontiguousarray(stored))
    x = host.cuda()
    nw = len(plan.widths()[0])
    mu = t.empty((ndm, nw), dtype=t.float32, device="cuda")
    sg = t.empty((ndm, nw), dtype=t.float32, device="cuda")
    ws = t.empty(plan.workspace_size(), dtype=t.uint8, device="cuda")
    spd.noise_stats(plan, x, mu, sg, ws, outlier_sigma=thr, max_passes=passes)
    spd.spd_sync_status(plan, t.cuda.current_stream().cuda_stream)
    return mu.cpu().numpy().astype(np.float64), sg.cpu().numpy().astype(np.float64)


def _oracle_table(plan, vals, thr, passes):
    w, _ = plan.widths()
    m, s, n = oracle.msd_levels(vals, _nlev(int(w[-1])), thr=thr, max_passes=passes)
    return oracle.msd_table(m, s, n, w)


def _close(g, o, ctx):
    (gm, gs), (om, os_) = g, o
    assert np.all(np.abs(gs - os_) <= 2e-5 * np.maximum(os_, 1e-6)), (ctx, np.max(np.abs(gs - os_) / os_))
    assert np.all(np.abs(gm - om) <= 2e-5 * (np.abs(om) + os_)), (ctx, np.max(np.abs(gm - om)))


CASES = [("ig1", 8192, 3, 100003, 2.0, 10), ("bd16", 2000, 2, 50001, 3.0, 10), ("exh", 100, 2, 30000, 2.0, 4),
         ("ig3", 8192, 2, 5000, 2.0, 10), ("dit", 32768, 1, 300000, 2.5, 20), ("ig1", 8192, 2, 70000, 0.0, 1)]


@pytest.mark.parametrize("name,s_end,ndm,nt,thr,passes", CASES, ids=["%s-%d-%dx%d-t%g-p%d" % c for c in CASES])
def test_noise_stats_parity(name, s_end, ndm, nt, thr, passes):
    x = _rows(ndm, nt, 700 + nt % 71)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    _close(_gpu_table(plan, x.astype(np.float32), thr, passes),
           _oracle_table(plan, x.astype(np.float32).astype(np.float64), thr, passes), name)


# 60001 samples: rows loaded into registers; 60000: 16-byte rows, staged by bulk copies
@pytest.mark.parametrize("nt", [60001, 60000])
@pytest.mark.parametrize("dtype,code", [("f16", spd.SPD_F16), ("bf16", spd.SPD_BF16), ("u8", spd.SPD_U8)])
def test_noise_stats_dtypes(dtype, code, nt):
    ndm = 2
    x = spd_synth.gaussian_noise(ndm, nt, 31, dtype=np.float64)
    stored, vals = spd_synth.quantize(x if dtype == "u8" else 0.5 + 1.2 * x, dtype)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, dtype=code, **ALGOS["ig1"](4096))
    _close(_gpu_table(plan, stored, 2.0, 10), _oracle_table(plan, vals, 2.0, 10), dtype)


# short rows: a single sample, fewer samples than one 256-sample warp step, and the
# step and 2048-sample chunk boundaries; ld = nt loads into registers, ld a multiple
# of 4 (16-byte rows) takes bulk copies for the whole steps and plain loads for the rest
@pytest.mark.parametrize("aligned", [False, True], ids=["ld=nt", "ld16B"])
@pytest.mark.parametrize("nt", [1, 3, 255, 256, 257, 2047, 2049, 4097])
def test_noise_stats_short_rows(nt, aligned):
    ndm, ld = 3, ((nt + 3) // 4) * 4 if aligned else nt
    xf = _rows(ndm, ld, 900 + nt).astype(np.float32)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, ld=ld, **ALGOS["exh"](16))
    _close(_gpu_table(plan, xf, 2.0, 10), _oracle_table(plan, xf[:, :nt].astype(np.float64), 2.0, 10),
           "nt %d ld %d" % (nt, ld))


def test_noise_stats_table_drives_table_search():
    # spikes inflate a plain deviation; the rejected estimate gives the search its noise table
    ndm, nt = 2, 80000
    x = _rows(ndm, nt, 91, spikes=0.003)
    tab = spd_synth.pulse_table(4, ndm, nt, 92, width_range=(1, 300), snr_range=(8.0, 20.0))
    spd_synth.inject(x, tab, 1.0)
    xf = x.astype(np.float32)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS["bd8"](4096))
    gm, gs = _gpu_table(plan, xf, 2.0, 10)
    om, os_ = _oracle_table(plan, xf.astype(np.float64), 2.0, 10)
    _close((gm, gs), (om, os_), "table")
    Yg, Wg = run_gpu(plan, xf, gm.astype(np.float32), gs.astype(np.float32), noise_mode=1)
    Yo, Wo, Y2o = oracle.search(xf.astype(np.float64), oracle_grid(plan), gm.astype(np.float32).astype(np.float64),
                                gs.astype(np.float32).astype(np.float64), noise_mode=1)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="msd table search")
