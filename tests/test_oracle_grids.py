"""Pins of the oracle's width grids against what the paper prints (CPU only)."""
import numpy as np
import pytest

import oracle
from conftest import read_table


def test_boxdit_worked_example():
    # Sec. 3.1 worked example (L^i_max = 4): golden file holds the two printed groups.
    want = read_table("boxdit_lmax4.txt")
    g = oracle.grid_boxdit(4, 12)
    assert [[int(a), int(b)] for a, b in zip(g.L, g.Ls)] == want


def test_boxdit_per_iteration_lmax():
    # Sec. 3.1: BoxDIT's maximum width may differ from iteration to iteration; the
    # golden grid is evaluated by hand from the width formula (see its header).
    want = read_table("boxdit_lmax_per_iter.txt")
    g = oracle.grid_boxdit([2, 4, 6], 45)
    assert [[int(a), int(b)] for a, b in zip(g.L, g.Ls)] == want
    # a list whose entries are all k is the uniform grid; n_iter counts iterations
    for k in (2, 6, 8, 10):
        for n_iter in (0, 3):
            u = oracle.grid_boxdit(k, 700, n_iter)
            v = oracle.grid_boxdit([k, k, k], 700, n_iter)
            assert np.array_equal(u.L, v.L) and np.array_equal(u.Ls, v.Ls)
    g = oracle.grid_boxdit([4, 2], 1, 3)  # exactly three iterations: 1..4 | 6, 8 | 12, 16
    assert list(g.L) == [1, 2, 3, 4, 6, 8, 12, 16] and list(g.Ls) == [1] * 4 + [2] * 2 + [4] * 2


def test_igrid_table1_depths():
    # Table 1: widths produced from base 16 by depth d.  In the IG(d) grid the step
    # whose base width is 16 must produce exactly that row.
    for row in read_table("igrid_table1.txt"):
        d, widths = row[0], row[1:]
        g = oracle.grid_igrid(d, max(1, 2 ** (d + 1)), 4096)
        step = [int(w) for w in g.L if 16 <= w < 32]
        assert step == widths, (d, step, widths)


def test_igrid_step_count_to_8192(paper_values):
    # 14 IGRID steps reach L_end = 8192; a step is one decimation level (base 2^i).
    for d, P in ((1, 4), (2, 8), (3, 16)):
        g = oracle.grid_igrid(d, P, paper_values["l_end_performance"])
        steps = {int(np.log2(w)) for w in g.L}
        assert len(steps) == paper_values["igrid_steps_to_8192"]
        assert int(g.L[-1]) == paper_values["l_end_performance"]


def test_dit_is_powers_of_two():
    # Alg. 3: DIT produces widths 2^i with separation equal to the width.
    g = oracle.grid_igrid(0, 1, 1 << 12)
    assert list(g.L) == [1 << i for i in range(13)]
    assert list(g.Ls) == list(g.L)


def test_igrid_separation_is_base_over_layers():
    # Sec. 3.2: P layers give separation 2^i / P.
    g = oracle.grid_igrid(2, 8, 8192)
    for w, s in zip(g.L, g.Ls):
        base = 1 << int(np.log2(w))
        assert s == max(1, base // 8)


def test_boxdit_width_formula_and_nearest_longer():
    # Alg. 1: iteration i adds widths L^{i-1}_MAX + 2^i m with separation 2^i; the last
    # width is the first one >= S_end (Sec. 3, definition of L_end).
    for k in (8, 16, 32):
        g = oracle.grid_boxdit(k, 8192)
        assert g.L[-1] >= 8192 and g.L[-2] < 8192
        assert np.all(np.diff(g.L) > 0)
        for w, s in zip(g.L, g.Ls):
            i = int(np.log2(s))
            lmax_prev = k * (2 ** i - 1)
            assert (w - lmax_prev) % s == 0 and 1 <= (w - lmax_prev) // s <= k


def test_exhaustive():
    g = oracle.grid_exhaustive(256)
    assert list(g.L) == list(range(1, 257)) and set(g.Ls) == {1}


def test_invalid_parameters_rejected():
    with pytest.raises(ValueError):
        oracle.grid_boxdit(3, 100)  # L^i_max must be divisible by D = 2 (Sec. 3.1)
    with pytest.raises(ValueError):
        oracle.grid_boxdit([4, 6, 5], 100)  # ... in every iteration
    with pytest.raises(ValueError):
        oracle.grid_igrid(1, 3, 100)  # layers must be a power of two
