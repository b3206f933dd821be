"""Pins of the oracle's search (definition form O1 and the paper's step forms O2).

All CPU only.  Pins: pure-Python brute force on tiny inputs, the closed-form SNR
of a matched rectangular pulse (Sec. 2.1 and Appendix A), a boxcar missing the
pulse gives SNR 0, the Sec. 4.3 example, and O1 == O2 on random data.
"""
import math

import numpy as np
import pytest

import oracle
import spd_synth


def _rand(ndm, nt, seed):
    return spd_synth.gaussian_noise(ndm, nt, seed, dtype=np.float64)


@pytest.mark.parametrize("grid", [
    ("exh", lambda: oracle.grid_exhaustive(9)),
    ("bd4", lambda: oracle.grid_boxdit(4, 30)),
    ("ig1", lambda: oracle.grid_igrid(1, 4, 24)),
    ("ig2", lambda: oracle.grid_igrid(2, 8, 17)),
    ("dit", lambda: oracle.grid_igrid(0, 1, 32)),
], ids=lambda g: g[0])
def test_brute_force_equals_definition(grid):
    g = grid[1]()
    x = _rand(2, 97, 11)
    mu, sigma = np.array([0.3, -1.0]), np.array([1.5, 0.7])
    Y, W, _ = oracle.search(x, g, mu, sigma)
    Yl, Wl, _ = oracle.search(x, g, mu, sigma, literal=True)
    for r in range(2):
        Yb, Wb = oracle.brute_search(x[r], g.L, g.Ls, mu[r], sigma[r])
        np.testing.assert_allclose(Y[r], Yb, rtol=0, atol=1e-12)
        np.testing.assert_allclose(Yl[r], Yb, rtol=0, atol=1e-12)
        assert np.array_equal(W[r], Wb) and np.array_equal(Wl[r], Wb)


@pytest.mark.parametrize("S", [1, 3, 7, 16, 33, 64, 100, 200])
def test_matched_pulse_closed_form(S):
    # A rectangular pulse of amplitude C/sqrt(S) (Eq. amplitudenormalization) with
    # mu = 0, sigma = 1 gives exactly C for the boxcar that covers it
    # (Appendix A, best case S = L).  Every other boxcar gives less.
    C, t, nt = 10.0, 300, 900
    x = np.zeros((1, nt))
    x[0, t:t + S] = C / math.sqrt(S)
    g = oracle.grid_exhaustive(256)
    Y, W, _ = oracle.search(x, g)
    assert abs(Y[0, t] - C) < 1e-12
    assert g.L[W[0, t]] == S
    assert np.all(Y[0, np.arange(nt) != t] < C - 1e-9)


def test_boxcar_missing_pulse_gives_zero():
    # Appendix A: a boxcar that does not intersect the pulse sums to zero, SNR 0.
    x = np.zeros((1, 500))
    x[0, 400:410] = 3.0
    g = oracle.grid_exhaustive(32)
    Y, W, _ = oracle.search(x, g)
    far = np.arange(0, 400 - 32)
    assert np.all(Y[0, far] == 0.0) and np.all(W[0, far] == 0)  # ties -> smallest width


def test_sec43_pulse_at_100(paper_values):
    # Sec. 4.3: width-20 rectangular pulse starting at sample 100 is found by a
    # width-20 boxcar; boxcars are indexed by their first sample (Eq. boxcar), so
    # the reported centre is start + width/2 = 110.
    S, t0 = paper_values["e4_width"], paper_values["e4_start"]
    C = 8.0
    x = np.zeros((1, 2 * 8192 + 400))
    x[0, t0:t0 + S] = C / math.sqrt(S)
    # BoxDIT BD-32 with the maximum search width of the Sec. 4.3 runs.
    g = oracle.grid_boxdit(32, paper_values["e4_search_width"])
    Y, W, _ = oracle.search(x, g)
    s = int(np.argmax(Y[0]))
    assert s == t0 and g.L[W[0, s]] == S and abs(Y[0, s] - C) < 1e-12
    assert s + g.L[W[0, s]] // 2 == paper_values["e4_detect"]
    Yb, Wl = oracle.boxdit_steps(x, 32, paper_values["e4_search_width"])
    assert int(np.argmax(Yb[0])) == t0 and Wl[0, t0] == S


@pytest.mark.parametrize("k,s_end,nt", [(4, 100, 513), (8, 300, 1000), (16, 200, 700),
                                        (32, 1000, 2100), (8, 50, 37), (4, 500, 300)])
def test_boxdit_paper_form_equals_definition(k, s_end, nt):
    x = _rand(3, nt, 5 + k)
    mu, sigma = np.array([0.0, 0.5, -2.0]), np.array([1.0, 2.0, 0.5])
    g = oracle.grid_boxdit(k, s_end)
    Y, W, _ = oracle.search(x, g, mu, sigma)
    Yp, Wl = oracle.boxdit_steps(x, k, s_end, mu, sigma)
    np.testing.assert_allclose(Yp, Y, rtol=0, atol=1e-11)
    assert np.array_equal(g.L[W], Wl)


@pytest.mark.parametrize("k,s_end,nt", [((2, 4, 6), 300, 700), ((12,), 400, 901), ((6, 2), 100, 333),
                                        ((2,), 1000, 1500), ((10, 4, 14, 2), 250, 64)])
def test_boxdit_per_iteration_paper_form_equals_definition(k, s_end, nt):
    # Alg. 1 with L^i_max changing per iteration (Sec. 3.1): the shifted decimation by
    # L^i_max / D per iteration against the definition on the grid of the width formula.
    x = _rand(3, nt, 77 + len(k))
    mu, sigma = np.array([0.0, 0.5, -2.0]), np.array([1.0, 2.0, 0.5])
    g = oracle.grid_boxdit(list(k), s_end)
    Y, W, _ = oracle.search(x, g, mu, sigma)
    Yp, Wl = oracle.boxdit_steps(x, list(k), s_end, mu, sigma)
    np.testing.assert_allclose(Yp, Y, rtol=0, atol=1e-11)
    assert np.array_equal(g.L[W], Wl)


def test_boxdit_per_iteration_brute_force():
    # literal running sums over the grid (no prefix sums) on a tiny row
    x = _rand(2, 97, 5)
    g = oracle.grid_boxdit([6, 2, 4], 60)
    Y, W, _ = oracle.search(x, g, literal=True)
    Yp, Wl = oracle.boxdit_steps(x, [6, 2, 4], 60)
    np.testing.assert_allclose(Yp, Y, rtol=0, atol=1e-11)
    assert np.array_equal(g.L[W], Wl)


@pytest.mark.parametrize("d,P,s_end,nt", [(0, 1, 256, 700), (1, 4, 300, 1025), (2, 8, 200, 999),
                                          (3, 16, 400, 1300), (1, 2, 64, 200), (2, 4, 100, 77),
                                          (1, 4, 5000, 600)])
def test_igrid_paper_form_equals_definition(d, P, s_end, nt):
    x = _rand(3, nt, 40 + d)
    mu, sigma = np.array([0.0, 0.25, 1.0]), np.array([1.0, 3.0, 0.25])
    g = oracle.grid_igrid(d, P, s_end)
    Y, W, _ = oracle.search(x, g, mu, sigma)
    Yp, Wl = oracle.igrid_steps(x, d, P, s_end, mu, sigma)
    np.testing.assert_allclose(Yp, Y, rtol=0, atol=1e-11)
    assert np.array_equal(g.L[W], Wl)


def test_table_noise_mode_matches_white():
    # Table mode with mu_L = L mu, sigma_L = sqrt(L) sigma must equal white mode (Eq. whitenoise).
    g = oracle.grid_igrid(1, 4, 64)
    x = _rand(2, 300, 3)
    mu, sigma = np.array([0.1, -0.4]), np.array([1.2, 0.9])
    Y, W, _ = oracle.search(x, g, mu, sigma)
    muL = mu[:, None] * g.L[None, :]
    sgL = sigma[:, None] * np.sqrt(g.L[None, :].astype(float))
    Yt, Wt, _ = oracle.search(x, g, muL, sgL, noise_mode=1)
    np.testing.assert_allclose(Yt, Y, rtol=1e-13, atol=1e-13)
    assert np.array_equal(Wt, W)


def test_end_of_row_only_complete_boxcars():
    # Reading of the paper: width L is used at s only if s + L <= nt.  The last
    # sample only sees width 1.
    g = oracle.grid_exhaustive(16)
    x = _rand(1, 50, 9)
    Y, W, _ = oracle.search(x, g)
    assert W[0, -1] == 0 and abs(Y[0, -1] - x[0, -1]) < 1e-13
    for s in range(50):
        assert s + g.L[W[0, s]] <= 50


def test_second_best_reported():
    g = oracle.grid_exhaustive(4)
    x = np.array([[1.0, 1.0, -5.0, 0.0, 0.0]])
    Y, W, Y2 = oracle.search(x, g)
    # at s = 0: widths 1,2,3,4 -> 1, 2/sqrt2, -3/sqrt3, -3/2
    assert abs(Y[0, 0] - math.sqrt(2)) < 1e-15 and W[0, 0] == 1 and Y2[0, 0] == 1.0
