"""The search at the benchmark workloads' full sizes, in the launch configuration
bench.py times.

* exhaustive_small (64 x 65,536, widths 1..256): full element-wise parity.
* ska_mid (4,096 x 1,048,576, IGRID IG(1) / BoxDIT BD-32, S_end = 8192): parity on
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


@pytest.mark.parametrize("name", ["ig1", "bd32"])
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
