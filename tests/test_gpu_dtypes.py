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
