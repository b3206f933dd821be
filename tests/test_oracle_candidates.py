"""Pins of the candidate rule (threshold + local maximum), CPU only."""
import numpy as np

import oracle


def _brute(Y, thr, R):
    out = []
    for r in range(Y.shape[0]):
        for s in range(Y.shape[1]):
            v = Y[r, s]
            if v < thr:
                continue
            ok = all(v > Y[r, q] for q in range(max(0, s - R), s))
            ok = ok and all(v >= Y[r, q] for q in range(s + 1, min(Y.shape[1], s + R + 1)))
            if ok:
                out.append((r, s))
    return out


def test_candidates_match_brute_force():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((5, 400)) * 2.0
    Y[1, 50:55] = 7.0  # plateau: the leftmost wins
    for R in (0, 1, 2, 5):
        n, rows, starts, w, snr = oracle.candidates(Y, None, thr=1.5, R=R)
        want = _brute(Y, 1.5, R)
        assert n == len(want) and list(zip(rows, starts)) == want
        assert np.all(snr == Y[rows, starts])
    n, rows, starts, _, _ = oracle.candidates(Y, None, thr=6.5, R=3)
    assert (1, 50) in list(zip(rows, starts)) and (1, 51) not in list(zip(rows, starts))


def test_radius_zero_is_plain_threshold():
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((3, 1000))
    n, rows, starts, _, _ = oracle.candidates(Y, None, thr=1.0, R=0)
    want = np.argwhere(Y >= 1.0)
    assert n == len(want) and np.array_equal(np.stack([rows, starts], 1), want)


def test_overflow_keeps_first_records():
    Y = np.full((2, 50), 10.0)
    n, rows, starts, _, _ = oracle.candidates(Y, None, thr=1.0, R=0, cap=7)
    assert n == 100 and list(starts) == list(range(7)) and set(rows) == {0}
