"""Table noise (spd_noise mode 1): per-row, per-width mu_L and sigma_L (Eq. SNRlong
with caller-supplied statistics instead of Eq. whitenoise), GPU against the FP64
oracle's table mode, element by element, with the same bar as white noise."""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, assert_parity, oracle_grid, run_gpu

pytestmark = pytest.mark.gpu


def _data(ndm, nt, seed, mu, sigma):
    x = spd_synth.gaussian_noise(ndm, nt, seed, dtype=np.float64)
    x = x * np.asarray(sigma).reshape(-1, 1) + np.asarray(mu).reshape(-1, 1)
    tab = spd_synth.pulse_table(2 * ndm, ndm, nt, seed + 1, width_range=(1, min(300, nt - 2)),
                                snr_range=(6.0, 30.0))
    spd_synth.inject(x, tab, float(np.mean(sigma)))
    return x.astype(np.float32)


def _tables(widths, mu, sigma, alpha, offset, seed):
    """mu_L = L mu_r + offset * sqrt(L) u_r, sigma_L = sigma_r L^alpha (alpha 0.5: white)."""
    L = np.asarray(widths, np.float64)[None, :]
    mu = np.asarray(mu, np.float64).reshape(-1, 1)
    sigma = np.asarray(sigma, np.float64).reshape(-1, 1)
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, (mu.shape[0], 1))
    muL = (L * mu + offset * np.sqrt(L) * u).astype(np.float32)
    sgL = (sigma * L ** alpha).astype(np.float32)
    return muL, sgL


CASES = [
    ("exh", 200, 2, 9001), ("bd8", 8192, 2, 40000), ("bd16", 2000, 2, 20001),
    ("bd32", 8192, 2, 36003), ("bd32", 700, 2, 20000), ("bd32", 20, 2, 3000),
    ("ig1", 8192, 3, 50000), ("ig1", 20, 2, 17000), ("ig2", 12, 2, 5000),
    ("ig3", 4096, 2, 30000), ("dit", 8192, 2, 40000),
]


@pytest.mark.parametrize("name,s_end,ndm,nt", CASES, ids=["%s-%d-%dx%d" % c for c in CASES])
def test_table_noise_parity(name, s_end, ndm, nt):
    mu = np.linspace(-0.4, 0.6, ndm)
    sigma = np.linspace(0.9, 1.7, ndm)
    x = _data(ndm, nt, 300 + nt % 89, mu, sigma)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    w, _ = plan.widths()
    muL, sgL = _tables(w, mu, sigma, alpha=0.6, offset=0.3, seed=nt)  # red-noise-like growth
    Yg, Wg = run_gpu(plan, x, muL, sgL, noise_mode=1)
    g = oracle_grid(plan)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, muL.astype(np.float64),
                                sgL.astype(np.float64), noise_mode=1)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="%s table" % name)


@pytest.mark.parametrize("name", ["exh", "bd8", "ig1", "ig3"])
def test_white_table_equals_white_mode(name):
    ndm, nt = 2, 30000
    mu, sigma = np.array([0.3, -0.2]), np.array([1.2, 0.7])
    x = _data(ndm, nt, 77, mu, sigma)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](4096 if name != "exh" else 128))
    w, _ = plan.widths()
    muL, sgL = _tables(w, mu, sigma, alpha=0.5, offset=0.0, seed=1)
    Yt, Wt = run_gpu(plan, x, muL, sgL, noise_mode=1)
    Yw, Ww = run_gpu(plan, x, mu, sigma)
    g = oracle_grid(plan)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, mu, sigma)
    assert_parity(Yt, Wt, Yo, Wo, Y2o, nt, ctx="%s white table" % name)
    assert_parity(Yw, Ww, Yo, Wo, Y2o, nt, ctx="%s white" % name)
    assert np.allclose(Yt, Yw, rtol=1e-5, atol=1e-5)
