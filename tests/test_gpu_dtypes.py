"""Reduced-precision inputs (f16, bf16, u8): the CUDA search on the stored
samples against the FP64 oracle on the values those samples hold, with the same
bar as float32 input.  Sizes span several segments and a ragged tail; the
scalar path (rows not 16-byte aligned) is covered too."""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, assert_parity, oracle_grid, run_gpu

pytestmark = pytest.mark.gpu

DT = {"f16": spd.SPD_F16, "bf16": spd.SPD_BF16, "u8": spd.SPD_U8}


def _stored(ndm, nt, seed, dtype):
    x = spd_synth.gaussian_noise(ndm, nt, seed, dtype=np.float64)
    tab = spd_synth.pulse_table(2 * ndm, ndm, nt, seed + 1, width_range=(1, min(300, nt - 2)),
                                snr_range=(6.0, 25.0))
    spd_synth.inject(x, tab, 1.0)
    if dtype != "u8":
        x = 0.2 + 1.3 * x  # mean 0.2, deviation 1.3 in stored units
        return spd_synth.quantize(x, dtype) + ((0.2, 1.3),)
    stored, vals = spd_synth.quantize(x, dtype)
    return stored, vals, (spd_synth.U8_OFFSET, spd_synth.U8_SCALE)


CASES = [
    ("exh", 128, 2, 9001), ("bd8", 8192, 2, 40000), ("bd32", 4096, 2, 36003),
    ("ig1", 8192, 3, 50000), ("ig1", 20, 2, 17000), ("ig3", 4096, 2, 30000), ("dit", 8192, 2, 40000),
    ("ig1", 8192, 1, 140001),
]


@pytest.mark.parametrize("dtype", ["f16", "bf16", "u8"])
@pytest.mark.parametrize("name,s_end,ndm,nt", CASES, ids=["%s-%d-%dx%d" % c for c in CASES])
def test_dtype_parity(dtype, name, s_end, ndm, nt):
    stored, vals, (mu, sigma) = _stored(ndm, nt, 500 + nt % 83, dtype)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, dtype=DT[dtype], **ALGOS[name](s_end))
    Yg, Wg = run_gpu(plan, stored, mu, sigma)
    Yo, Wo, Y2o = oracle.search(vals, oracle_grid(plan), mu, sigma)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="%s %s" % (dtype, name))


@pytest.mark.parametrize("dtype", ["f16", "bf16", "u8"])
@pytest.mark.parametrize("name", ["exh", "bd16", "ig2"])
def test_dtype_scalar_path(dtype, name):
    # rows of ld * sample size not a multiple of 16 bytes, base one sample off
    ndm, nt, ld = 3, 20001, 20003
    stored, vals, (mu, sigma) = _stored(ndm, nt, 9, dtype)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, ld=ld, dtype=DT[dtype],
                               **ALGOS[name](2000 if name != "exh" else 100))
    Yg, Wg = run_gpu(plan, stored, mu, sigma, x_offset=1)
    Yo, Wo, Y2o = oracle.search(vals, oracle_grid(plan), mu, sigma)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="%s %s scalar" % (dtype, name))


# error of each stored type against the FP64 oracle on the original (unquantised)
# series: quantisation error, reported (pytest -s) and bounded by the type's step
ERR_BOUNDS = {"f32": (1e-5, 1e-6, 0.999), "f16": (5e-3, 5e-4, 0.99), "bf16": (4e-2, 4e-3, 0.95),
              "u8": (0.2, 0.03, 0.9)}


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16", "u8"])
def test_dtype_error_against_fp64_original(dtype):
    ndm, nt = 4, 131072
    x = spd_synth.gaussian_noise(ndm, nt, 77, dtype=np.float64)
    tab = spd_synth.pulse_table(8, ndm, nt, 78, width_range=(1, 2000), snr_range=(6.0, 15.0), min_gap=9000)
    spd_synth.inject(x, tab, 1.0)
    if dtype == "f32":
        stored, mu, sigma, code = x.astype(np.float32), 0.0, 1.0, spd.SPD_F32
    else:
        stored, _ = spd_synth.quantize(x, dtype)
        mu, sigma = (spd_synth.U8_OFFSET, spd_synth.U8_SCALE) if dtype == "u8" else (0.0, 1.0)
        code = DT[dtype]
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, dtype=code, **ALGOS["ig1"](8192))
    Yg, Wg = run_gpu(plan, stored, mu, sigma)
    Yo, Wo, Y2o = oracle.search(x, oracle_grid(plan), 0.0, 1.0)
    rel = np.abs(Yg.astype(np.float64) - Yo) / np.maximum(np.abs(Yo), 1.0)
    clear = (Yo - Y2o) > 0.05
    agree = float(np.mean(Wg[clear] == Wo[clear]))
    print("\n%s vs FP64 original: max %.3g, p99.9 %.3g, mean %.3g relative SNR error; width agreement %.5f "
          "(%d starts with a clear winner)" % (dtype, rel.max(), np.quantile(rel, 0.999), rel.mean(), agree,
                                               int(clear.sum())))
    mx, mean, ag = ERR_BOUNDS[dtype]
    assert np.quantile(rel, 0.999) <= mx and rel.mean() <= mean and agree >= ag
