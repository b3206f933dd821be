"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
entry point declared in include/spd.h, validates plans, and its width grids
equal the oracle's (two independent restatements of the paper)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "spd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spd_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = spd.load_library()
    names = _declared()
    assert "spd_execute" in names and "spd_search" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_candidates_status_validates_before_any_device_work():
    lib = spd.load_library()
    total = ctypes.c_int64(-7)
    assert lib.spd_candidates_status(None, 10, ctypes.byref(total), None) == 1  # NULL count
    assert lib.spd_candidates_status(ctypes.c_void_p(8), -1, ctypes.byref(total), None) == 1  # cap < 0
    assert lib.spd_candidates_status(ctypes.c_void_p(12), 0, None, None) == 1  # misaligned
    assert total.value == -7


def test_version_and_status_strings():
    assert spd.spd_version() == "0.1"
    for s in range(8):
        assert spd.spd_status_string(s)
    assert spd.spd_status_string(0) == "ok"


GRIDS = [
    ("exh256", dict(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=256), lambda: oracle.grid_exhaustive(256)),
    ("exh1", dict(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=1), lambda: oracle.grid_exhaustive(1)),
] + [
    ("bd%d_%d" % (k, s), dict(algo=spd.SPD_ALGO_BOXDIT, s_end=s, boxdit_lmax=k),
     (lambda k=k, s=s: oracle.grid_boxdit(k, s)))
    for k in (2, 6, 8, 12, 16, 32, 64) for s in (1, 5, 32, 33, 100, 8192, 20000)
    if not (k == 64 and s == 20000)  # 576 widths: above the 512 a plan may hold
] + [
    ("ig%d_%d_%d" % (d, P, s), dict(algo=spd.SPD_ALGO_IGRID, s_end=s, igrid_depth=d, igrid_layers=P),
     (lambda d=d, P=P, s=s: oracle.grid_igrid(d, P, s)))
    for d, P in ((0, 1), (0, 2), (1, 2), (1, 4), (2, 4), (2, 8), (3, 8), (3, 16))
    for s in (1, 3, 7, 16, 31, 100, 8192, 30000)
]


@pytest.mark.parametrize("name,kw,og", GRIDS, ids=[g[0] for g in GRIDS])
def test_plan_widths_equal_oracle_grid(name, kw, og):
    plan = spd.spd_plan_create(ndm=4, nt=100000, **kw)
    w, s = plan.widths()
    g = og()
    assert np.array_equal(w, g.L) and np.array_equal(s, g.Ls)
    assert plan.workspace_size() > 0


@pytest.mark.parametrize("kw", [
    dict(algo=spd.SPD_ALGO_BOXDIT, s_end=100, boxdit_lmax=7),
    dict(algo=spd.SPD_ALGO_BOXDIT, s_end=100, boxdit_lmax=0),
    dict(algo=spd.SPD_ALGO_BOXDIT, s_end=100, boxdit_lmax=258),
    dict(algo=spd.SPD_ALGO_BOXDIT, s_end=20000, boxdit_lmax=64),  # 576 widths
    dict(algo=spd.SPD_ALGO_IGRID, s_end=100, igrid_depth=1, igrid_layers=3),
    dict(algo=spd.SPD_ALGO_IGRID, s_end=100, igrid_depth=2, igrid_layers=2),
    dict(algo=spd.SPD_ALGO_IGRID, s_end=100, igrid_depth=4, igrid_layers=16),
    dict(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=0),
    dict(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=5000),
    dict(algo=spd.SPD_ALGO_IGRID, s_end=40000, igrid_depth=1, igrid_layers=4),
    dict(algo=7, s_end=10),
])
def test_invalid_plans_rejected(kw):
    with pytest.raises(spd.SpdError) as e:
        spd.spd_plan_create(ndm=4, nt=1000, **kw)
    assert e.value.status == 1


def test_bad_shapes_and_dtypes():
    with pytest.raises(spd.SpdError) as e:
        spd.spd_plan_create(spd.SPD_ALGO_IGRID, 64, ndm=4, nt=100, ld=50, igrid_depth=1, igrid_layers=4)
    assert e.value.status == 1
    with pytest.raises(spd.SpdError) as e:
        spd.spd_plan_create(spd.SPD_ALGO_IGRID, 64, ndm=0, nt=100, igrid_depth=1, igrid_layers=4)
    assert e.value.status == 1
    for dt in (spd.SPD_F32, spd.SPD_F16, spd.SPD_BF16, spd.SPD_U8):
        spd.spd_plan_create(spd.SPD_ALGO_IGRID, 64, ndm=4, nt=100, igrid_depth=1, igrid_layers=4,
                            dtype=dt)
    with pytest.raises(spd.SpdError) as e:
        spd.spd_plan_create(spd.SPD_ALGO_IGRID, 64, ndm=4, nt=100, igrid_depth=1, igrid_layers=4,
                            dtype=4)
    assert e.value.status == 1


def test_execute_rejects_x_misaligned_for_its_dtype():
    plan = spd.spd_plan_create(spd.SPD_ALGO_IGRID, 64, ndm=4, nt=1000, igrid_depth=1, igrid_layers=4,
                               dtype=spd.SPD_F16)
    with pytest.raises(spd.SpdError) as e:
        spd.spd_execute(plan, 4097, 4096, 4096, 4096, 4096, 4096, 1 << 30)
    assert e.value.status == 1


def test_execute_validates_before_launch():
    # NULL pointers and a missing workspace are rejected synchronously, no GPU touched.
    plan = spd.spd_plan_create(spd.SPD_ALGO_IGRID, 64, ndm=4, nt=1000, igrid_depth=1, igrid_layers=4)
    with pytest.raises(spd.SpdError) as e:
        spd.spd_execute(plan, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.status == 1
    with pytest.raises(spd.SpdError) as e:
        spd.spd_execute(plan, 4096, 4096, 4096, 4096, 4096, 0, 0)
    assert e.value.status == 4  # workspace too small
    with pytest.raises(spd.SpdError) as e:
        spd.spd_candidates(plan, 4096, 4096, 6.0, 65, 0, 0, 4096, 0, 0, 0)
    assert e.value.status == 1  # radius above the maximum
    with pytest.raises(spd.SpdError) as e:
        spd.spd_execute(plan, 4096, 4096, 4096, 4096, 4096, 4096, 1 << 30, noise_mode=2)
    assert e.value.status == 1  # noise modes are 0 (white) and 1 (table)
    with pytest.raises(spd.SpdError) as e:
        spd.spd_execute(plan, 4096, 4098, 4096, 4096, 4096, 4096, 1 << 30, noise_mode=1)
    assert e.value.status == 1  # misaligned noise table


def test_widths_buffer_too_small():
    plan = spd.spd_plan_create(spd.SPD_ALGO_BOXDIT, 8192, ndm=1, nt=100, boxdit_lmax=32)
    lib = spd.load_library()
    n = ctypes.c_int32()
    buf = np.zeros(10, np.int32)
    st = lib.spd_plan_widths(ctypes.c_void_p(plan.handle), buf.ctypes.data, None, 10, ctypes.byref(n))
    assert st == 5 and n.value == 257


def test_batch_validation():
    A = spd.SPD_ALGO_BOXDIT
    b = spd.spd_batch_create(A, 4096, [1024, 1024, 768, 512, 256],
                             [2097152, 1048576, 524288, 262144, 131072], boxdit_lmax=16)
    assert b.workspace_size() > 0
    b.set_segment(65536)
    b.set_wait_ns(10 ** 6)
    for bad in (1000, 16384 + 8192, 0, 1 << 25):
        with pytest.raises(spd.SpdError) as e:
            b.set_segment(bad)
        assert e.value.status == 1
    with pytest.raises(spd.SpdError) as e:
        b.set_wait_ns(-1)
    assert e.value.status == 1
    with pytest.raises(spd.SpdError) as e:  # exhaustive grids are not batched
        spd.spd_batch_create(spd.SPD_ALGO_EXHAUSTIVE, 64, [1], [100])
    assert e.value.status == 2
    for ndm, nt, ld in (([1] * 9, [100] * 9, None), ([0], [100], None), ([1], [100], [50])):
        with pytest.raises(spd.SpdError) as e:
            spd.spd_batch_create(A, 64, ndm, nt, ld, boxdit_lmax=8)
        assert e.value.status == 1
    # execute validates before any launch: NULL range pointers, small workspace
    with pytest.raises(spd.SpdError) as e:
        spd.spd_batch_execute(b, [0] * 5, [0] * 5, [0] * 5, [0] * 5, [0] * 5, 4096, 1 << 30)
    assert e.value.status == 1
    with pytest.raises(spd.SpdError) as e:
        spd.spd_batch_execute(b, [4096] * 5, [4096] * 5, [4096] * 5, [4096] * 5, [4096] * 5, 4096, 16)
    assert e.value.status == 4


@pytest.mark.parametrize("lmax,s_end,n_iter", [([2, 4, 6], 45, 0), ([6, 2], 3000, 0), ([32, 16, 8], 8192, 0),
                                              ([8], 1, 10), ([12], 1, 6), ([4, 2], 1, 3), ([64, 2], 9000, 0)])
def test_per_iteration_boxdit_plan_equals_oracle_grid(lmax, s_end, n_iter):
    plan = spd.spd_plan_create_boxdit(lmax, s_end, ndm=2, nt=50000, n_iter=n_iter)
    w, s = plan.widths()
    g = oracle.grid_boxdit(lmax, s_end, n_iter)
    assert np.array_equal(w, g.L) and np.array_equal(s, g.Ls)
    assert plan.workspace_size() > 0


def test_per_iteration_boxdit_plan_rules():
    for lmax, n_iter in (([3], 0), ([4, 5], 0), ([0], 0), ([260], 0), ([], 0), ([8], 25), ([8], -1),
                         ([2] * 25, 0)):
        with pytest.raises(spd.SpdError) as e:
            spd.spd_plan_create_boxdit(lmax if lmax else np.zeros(0, np.int32), 100, ndm=2, nt=1000,
                                       n_iter=n_iter)
        assert e.value.status == 1, (lmax, n_iter)
    # widest width above 32768 or more than 512 widths
    for lmax, s_end in (([2], 40000), ([256], 1000)):
        with pytest.raises(spd.SpdError):
            spd.spd_plan_create_boxdit(lmax, s_end, ndm=2, nt=1000)
    # the general kernel takes tiles of 2048, 4096 or 8192 starts as its segment
    plan = spd.spd_plan_create_boxdit([6, 2], 1000, ndm=2, nt=1 << 20)
    for seg in (2048, 4096, 8192):
        spd.spd_plan_set_segment(plan, seg)
    for seg in (1024, 16384, 3000):
        with pytest.raises(spd.SpdError) as e:
            spd.spd_plan_set_segment(plan, seg)
        assert e.value.status == 1
    wide = spd.spd_plan_create_boxdit([2], 30000, ndm=2, nt=1 << 20)
    spd.spd_plan_set_segment(wide, 8192)  # 8192 starts + a 32766-sample halo still fit in 227 KB


def test_two_kernel_form_workspace():
    """General BoxDIT plans above level 4 keep x^4, the level-3 bases and the first
    kernel's SNR and width index at every 16th start of every row in the workspace
    (3 floats and a u16 per 16 samples, rounded up to whole first-kernel tiles);
    plans up to level 4 need none."""
    ndm, nt = 3, 100000
    low = spd.spd_plan_create_boxdit([6], 20, ndm=ndm, nt=nt)     # widths up to 42: levels 0-2
    high = spd.spd_plan_create_boxdit([6], 8192, ndm=ndm, nt=nt)  # levels 0-10
    base = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=8192, ndm=ndm, nt=nt, boxdit_lmax=16)
    assert low.workspace_size() == base.workspace_size()
    for seg in (2048, 4096, 8192):
        spd.spd_plan_set_segment(high, seg)
        ldh = -(-nt // seg) * (seg // 16)
        assert high.workspace_size() - base.workspace_size() >= (3 * 4 + 2) * ndm * ldh
        assert high.workspace_size() - base.workspace_size() < (3 * 4 + 2) * ndm * ldh + 512


def test_proposal_rules():
    kw = dict(algo=spd.SPD_ALGO_IGRID, s_end=4096, igrid_depth=1, igrid_layers=4)
    p = spd.spd_proposal_create(ndm=4, nt=1 << 16, max_blocks=10, **kw)
    assert p.workspace_size() > 0 and len(p.widths()[0]) == len(oracle.grid_igrid(1, 4, 4096))
    for bad, status in ((dict(nt=5000), 1), (dict(nt=4095), 1), (dict(dtype=spd.SPD_U8), 2),
                        (dict(s_end=30000), 2), (dict(peak_radius=65), 1), (dict(max_blocks=0), 1),
                        (dict(ndm=0), 1)):
        a = dict(ndm=4, nt=1 << 16, max_blocks=10, **kw)
        a.update(bad)
        with pytest.raises(spd.SpdError) as e:
            spd.spd_proposal_create(**a)
        assert e.value.status == status, bad
    lib = spd.load_library()
    # argument checks come before any device work
    import ctypes
    nb = ctypes.c_int64(7)
    assert lib.spd_propose_search(None, 256, 256, None, ctypes.c_float(0), ctypes.c_float(6), 256, 1, 256,
                                  ctypes.byref(nb), 256, 1 << 30, None) == 1
    assert nb.value == 0
    ws = p.workspace_size()
    nz = spd._binding._Noise(0, 256, 256)
    h = ctypes.c_void_p(p.handle)
    assert lib.spd_propose_search(h, 256, 256, ctypes.byref(nz), ctypes.c_float(0), ctypes.c_float(6), 256, 1,
                                  256, None, 256, ws - 1, None) == 4  # workspace too small
    assert lib.spd_propose_search(h, 256, 256, ctypes.byref(nz), ctypes.c_float(float("nan")),
                                  ctypes.c_float(6), 256, 1, 256, None, 256, ws, None) == 1
    assert lib.spd_propose_search(h, 256, 256, ctypes.byref(nz), ctypes.c_float(0), ctypes.c_float(6), 256, 1,
                                  260, None, 256, ws, None) == 1  # misaligned count
    # block search: more ids than the proposal holds, misaligned ids, short workspace
    assert lib.spd_search_blocks(h, 256, ctypes.byref(nz), 256, 11, ctypes.c_float(6), 256, 1, 256, 256, ws,
                                 None) == 5
    assert lib.spd_search_blocks(h, 256, ctypes.byref(nz), 260, 3, ctypes.c_float(6), 256, 1, 256, 256, ws,
                                 None) == 1
    assert lib.spd_search_blocks(h, 256, ctypes.byref(nz), 256, 3, ctypes.c_float(6), 256, 1, 256, 256, ws - 1,
                                 None) == 4


def test_plan_segment_rules():
    plan = spd.spd_plan_create(spd.SPD_ALGO_IGRID, 32768, ndm=1, nt=1 << 20, igrid_depth=0, igrid_layers=1)
    with pytest.raises(spd.SpdError):
        spd.spd_plan_set_segment(plan, 16384)  # DIT up to 32768 has a level of 2^15: segments of 2^15
    spd.spd_plan_set_segment(plan, 32768)
    ex = spd.spd_plan_create(spd.SPD_ALGO_EXHAUSTIVE, 64, ndm=1, nt=1000)
    with pytest.raises(spd.SpdError):
        spd.spd_plan_set_segment(ex, 16384)


def test_net_select_and_gather_validate_before_launch():
    lib = spd.load_library()
    # u8 has no -inf code to pad with
    assert lib.spd_net_gather(4096, spd.SPD_U8, 1, 4096, 4096, 4096, 1, 4096, 0, 4096, 4096, 4096, None) == 2
    # output row shorter than the copied width; misaligned output; bad dtype
    assert lib.spd_net_gather(4096, spd.SPD_F16, 1, 4096, 4096, 4096, 1, 4096, 0, 4096, 4096, 4000, None) == 1
    assert lib.spd_net_gather(4096, spd.SPD_F16, 1, 4096, 4096, 4096, 1, 4096, 0, 4096, 4104, 4096, None) == 1
    assert lib.spd_net_gather(4096, 7, 1, 4096, 4096, 4096, 1, 4096, 0, 4096, 4096, 4096, None) == 1
    # f16 rows of 4100 samples are not 16-byte multiples
    assert lib.spd_net_gather(4096, spd.SPD_F16, 1, 4096, 4096, 4096, 1, 4096, 0, 4096, 4096, 4100, None) == 1
    assert lib.spd_net_gather(4096, spd.SPD_F16, 1, 4096, 4096, 4096, 1, 4096, -1, 4096, 4096, 4096, None) == 1
    assert lib.spd_net_select(4096, 16, ctypes.c_float(float("nan")), 4096, 16, 4096, None) == 1
    assert lib.spd_net_select(4096, 16, ctypes.c_float(0.0), None, 16, 4096, None) == 1
    assert lib.spd_net_select(4096, -1, ctypes.c_float(0.0), 4096, 16, 4096, None) == 1


def test_torch_helpers_refuse_short_outputs():
    """The torch-level helpers check every [ndm][ld] buffer before the C call
    (the C calls take bare pointers)."""
    torch = pytest.importorskip("torch")
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=64, boxdit_lmax=8, ndm=2, nt=1000, ld=1024)
    x = torch.zeros((2, 1024))
    ws = torch.zeros(16, dtype=torch.uint8)
    with pytest.raises(spd.SpdError) as e:
        spd.execute(plan, x, torch.zeros(2), torch.ones(2), torch.zeros((2, 1000)), torch.zeros((2, 1024), dtype=torch.int16), ws)
    assert e.value.status == 5
    with pytest.raises(spd.SpdError):
        spd.search(plan, x[:, :1000], torch.zeros(2), torch.ones(2), torch.zeros((2, 1024)),
                   torch.zeros((2, 1024), dtype=torch.int16), 6.0, 1, None, torch.zeros(1, dtype=torch.int64), ws)


def test_plan_set_starts_rules():
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_IGRID, s_end=4096, igrid_depth=1, igrid_layers=4, ndm=2, nt=50000)
    spd.spd_plan_set_starts(plan, 1)
    spd.spd_plan_set_starts(plan, 50000)
    for bad in (0, -5, 50001):
        with pytest.raises(spd.SpdError) as e:
            spd.spd_plan_set_starts(plan, bad)
        assert e.value.status == 1
    exh = spd.spd_plan_create(algo=spd.SPD_ALGO_EXHAUSTIVE, s_end=64, ndm=1, nt=9000)
    spd.spd_plan_set_starts(exh, 4097)


def test_explicit_grid_rules():
    ok = spd.spd_plan_create_grid([1, 3, 5, 10, 50, 200], [1, 1, 2, 4, 8, 32], ndm=2, nt=5000)
    w, s = ok.widths()
    assert w.tolist() == [1, 3, 5, 10, 50, 200] and s.tolist() == [1, 1, 2, 4, 8, 32]
    bad = [([2, 3], [1, 1]),            # width 1 must come first
           ([1, 3], [2, 1]),            # width 1 at every start
           ([1, 5, 5], [1, 1, 1]),      # strictly increasing
           ([1, 5, 4], [1, 1, 1]),
           ([1, 6], [1, 3]),            # separations are powers of two
           ([1, 5000], [1, 1]),         # at most 4096
           (list(range(1, 514)), [1] * 513)]  # at most 512 widths
    for widths, seps in bad:
        with pytest.raises(spd.SpdError) as e:
            spd.spd_plan_create_grid(widths, seps, ndm=2, nt=5000)
        assert e.value.status == 1, (widths[:4], seps[:4])
    # an explicit grid equal to a built-in one has the same table
    g = oracle.grid_boxdit(8, 512)
    pl = spd.spd_plan_create_grid(g.L, g.Ls, ndm=1, nt=4096)
    assert np.array_equal(pl.widths()[0], g.L) and np.array_equal(pl.widths()[1], g.Ls)


def test_ordered_gradient_workspace_rules():
    lib = spd.load_library()
    need = spd.spd_net_gradient_workspace_size()
    assert need == 4 * 1024 * (4817 + 1)
    assert lib.spd_net_gradient_ordered(4096, 4096, 4096, 8, 4096, 4096, 4096, need - 4, None) == 4
    assert lib.spd_net_gradient_ordered(4096, 4096, 4096, 8, 4096, 4096, None, need, None) == 1
    assert lib.spd_net_gradient_ordered(4096, 4096, 4096, 0, 4096, 4096, 4096, need, None) == 1
