"""The general BoxDIT kernel (any even L^i_max, uniform or per iteration; Alg. 1
and Sec. 3.1) against the FP64 oracle, with the bar of the other parity tests.

Cases span several 2048/4096-start tiles with ragged tails, top levels whose
unit exceeds the tile (positions in every second or fourth tile only), a top
level cut short by the nearest-longer rule and full iterations counted by
n_iter, table noise, every input type, the scalar (unaligned) path, evaluated
starts below nt, the batched search and the candidate step that reads the
kernel's tile maxima."""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, RTOL, assert_parity, oracle_grid, recompute_snr, run_gpu, torch

pytestmark = pytest.mark.gpu


def _data(ndm, nt, seed, max_w=300, mu=0.0, sigma=1.0):
    x = spd_synth.gaussian_noise(ndm, nt, seed, mu=mu, sigma=sigma, dtype=np.float64)
    if nt > max_w + 2:
        tab = spd_synth.pulse_table(2 * ndm, ndm, nt, seed + 1, width_range=(1, min(max_w, nt - 1)),
                                    snr_range=(6.0, 30.0))
        spd_synth.inject(x, tab, sigma)
    return x.astype(np.float32)


def _check(plan, x, mu, sigma, ctx, **kw):
    Yg, Wg = run_gpu(plan, x, mu, sigma, **kw)
    g = oracle_grid(plan)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, mu, sigma)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, x.shape[1], ctx=ctx)
    snr, ok = recompute_snr(x, mu, sigma, g.L, g.Ls, Wg)
    assert ok.all(), ctx
    assert np.all(np.abs(snr - Yo) <= 2 * RTOL * np.maximum(np.abs(Yo), 1.0)), ctx
    return Yg, Wg


UNIFORM = [
    # k, s_end, ndm, nt
    (2, 8192, 2, 40001), (4, 8192, 2, 30000), (6, 8192, 2, 40003), (10, 8192, 2, 36000),
    (12, 8192, 3, 40000), (24, 8192, 2, 33001), (64, 8192, 2, 40000), (128, 1500, 2, 21000),
    (2, 20000, 1, 140001),   # top level 13: unit 8192 > tile, positions every 2nd / 4th tile
    (12, 30000, 1, 100000),  # widest widths near the limit (tiles of 2048)
    (6, 5, 2, 5000), (12, 1, 2, 4100), (2, 3, 2, 9000), (14, 300, 2, 9001),
]


@pytest.mark.parametrize("k,s_end,ndm,nt", UNIFORM, ids=["k%d-%d-%dx%d" % c for c in UNIFORM])
def test_uniform_lmax_parity(k, s_end, ndm, nt):
    x = _data(ndm, nt, 300 + k + nt % 89)
    mu = np.linspace(-0.5, 0.5, ndm)
    sigma = np.linspace(0.8, 1.6, ndm)
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=s_end, ndm=ndm, nt=nt, boxdit_lmax=k)
    g = oracle_grid(plan)
    ref = oracle.grid_boxdit(k, s_end)
    assert np.array_equal(g.L, ref.L) and np.array_equal(g.Ls, ref.Ls)
    _check(plan, x, mu, sigma, "k=%d s_end=%d" % (k, s_end))


PER_ITER = [
    # lmax list, s_end, n_iter, ndm, nt
    ((2, 4, 6), 8192, 0, 2, 40000), ((6, 2), 3000, 0, 2, 20001), ((32, 16, 8), 8192, 0, 2, 40000),
    ((64, 2), 9000, 0, 2, 30000), ((8, 8, 8, 8, 16), 8192, 0, 2, 33333), ((4, 6, 8, 10, 12), 5000, 0, 2, 25000),
    ((12,), 1, 6, 2, 30000), ((2, 30), 1, 9, 2, 33000), ((8,), 1, 10, 2, 20000),
    # the second of the two kernels with many block counts per level, the first with few, and the reverse
    ((2, 2, 2, 2, 64), 8192, 0, 2, 40000), ((128, 2, 2, 2, 2, 32), 6000, 0, 2, 30000),
]


@pytest.mark.parametrize("lmax,s_end,n_iter,ndm,nt", PER_ITER,
                         ids=["%s-%d-%d-%dx%d" % (("_".join(map(str, c[0])),) + c[1:]) for c in PER_ITER])
def test_per_iteration_lmax_parity(lmax, s_end, n_iter, ndm, nt):
    x = _data(ndm, nt, 600 + len(lmax) + nt % 71)
    plan = spd.spd_plan_create_boxdit(list(lmax), s_end, ndm=ndm, nt=nt, n_iter=n_iter)
    g = oracle_grid(plan)
    ref = oracle.grid_boxdit(list(lmax), max(s_end, 1), n_iter)
    assert np.array_equal(g.L, ref.L) and np.array_equal(g.Ls, ref.Ls)
    _check(plan, x, 0.3, 1.2, "lmax=%s n_iter=%d" % (lmax, n_iter))


@pytest.mark.parametrize("nt", [1, 2, 3, 37, 130, 4095, 4097])
def test_tiny_and_tile_edge_rows(nt):
    x = _data(2, nt, 11 + nt, max_w=30)
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=64, ndm=2, nt=nt, boxdit_lmax=6)
    Yg, Wg = _check(plan, x, 0.0, 1.0, "nt=%d" % nt)
    assert np.array_equal(Wg[:, nt - 1], [0, 0])  # the last sample only has width 1


@pytest.mark.parametrize("nt", [1, 37, 4097, 16385, 33000])
def test_two_kernel_form_short_rows(nt):
    # a plan above level 4 on rows shorter than its widest boxcars, than one
    # first-kernel tile or than one second-kernel tile (32 768 starts)
    x = _data(2, nt, 31 + nt, max_w=300)
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=2000, ndm=2, nt=nt, boxdit_lmax=6)
    assert oracle_grid(plan).L[-1] > 16 * 6  # widths above level 4
    _check(plan, x, 0.0, 1.0, "nt=%d" % nt)


@pytest.mark.parametrize("name", ["bd2", "bd12", "bd64"])
def test_table_noise_parity(name):
    ndm, nt = 3, 30001
    x = _data(ndm, nt, 41)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](8192))
    g = oracle_grid(plan)
    L = g.L.astype(np.float64)[None, :]
    u = np.random.default_rng(5).uniform(-1.0, 1.0, (ndm, 1))
    muL = (0.05 * L + 0.3 * np.sqrt(L) * u).astype(np.float32)
    sgL = (np.linspace(0.9, 1.4, ndm).reshape(-1, 1) * L ** 0.6).astype(np.float32)
    Yg, Wg = run_gpu(plan, x, muL, sgL, noise_mode=1)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, muL.astype(np.float64), sgL.astype(np.float64),
                                noise_mode=1)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx=name + " table")


@pytest.mark.parametrize("dtype", [spd.SPD_F16, spd.SPD_BF16, spd.SPD_U8])
@pytest.mark.parametrize("offset", [0, 1])
def test_input_types_and_scalar_path(dtype, offset):
    name = {spd.SPD_F16: "f16", spd.SPD_BF16: "bf16", spd.SPD_U8: "u8"}[dtype]
    ndm, nt = 2, 20001
    x = spd_synth.gaussian_noise(ndm, nt, 77, dtype=np.float64)
    tab = spd_synth.pulse_table(4, ndm, nt, 78, width_range=(1, 300), snr_range=(6.0, 25.0))
    spd_synth.inject(x, tab, 1.0)
    if name == "u8":
        stored, vals = spd_synth.quantize(x, name)
        mu, sigma = spd_synth.U8_OFFSET, spd_synth.U8_SCALE
    else:
        stored, vals = spd_synth.quantize(0.2 + 1.3 * x, name)
        mu, sigma = 0.2, 1.3
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=4000, ndm=ndm, nt=nt, boxdit_lmax=10,
                               dtype=dtype)
    Yg, Wg = run_gpu(plan, stored, mu, sigma, x_offset=offset)
    Yo, Wo, Y2o = oracle.search(vals, oracle_grid(plan), mu, sigma)
    assert_parity(Yg, Wg, Yo, Wo, Y2o, nt, ctx="%s offset %d" % (name, offset))


def test_row_stride_and_evaluated_starts():
    ndm, nt, ld, ns = 3, 20001, 20008, 12345
    x = _data(ndm, nt, 3)
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=2000, ndm=ndm, nt=nt, ld=ld, boxdit_lmax=6)
    spd.spd_plan_set_starts(plan, ns)
    Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
    assert np.all(Yg[:, ns:] == -12345.0)  # neither the starts past n_starts nor the padding are written
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), oracle_grid(plan))
    assert_parity(Yg[:, :ns], Wg[:, :ns], Yo[:, :ns], Wo[:, :ns], Y2o[:, :ns], ns, ctx="n_starts")


@pytest.mark.parametrize("segment", [2048, 4096, 8192])
def test_two_kernel_form_tiles(segment):
    """A plan above level 4 runs levels 0-3 on tiles of 2048, 4096 or 8192
    starts, then levels 4.. on the series x^4 in tiles of 2048 level-4 positions
    (32 768 starts): rows of four such tiles and a ragged fifth, with fewer
    evaluated starts than samples."""
    ndm, nt, ns = 2, 150001, 140003
    x = _data(ndm, nt, 17 + segment)
    plan = spd.spd_plan_create_boxdit([2, 4, 6, 8, 10, 12], 8192, ndm=ndm, nt=nt)
    spd.spd_plan_set_segment(plan, segment)
    spd.spd_plan_set_starts(plan, ns)
    Yg, Wg = run_gpu(plan, x, 0.1, 0.9)
    assert np.all(Yg[:, ns:] == -12345.0)
    Yo, Wo, Y2o = oracle.search(x.astype(np.float64), oracle_grid(plan), 0.1, 0.9)
    assert_parity(Yg[:, :ns], Wg[:, :ns], Yo[:, :ns], Wo[:, :ns], Y2o[:, :ns], ns, ctx="tile %d" % segment)


def test_all_zero_input_ties_to_smallest_width():
    x = np.zeros((2, 20000), np.float32)
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=1024, ndm=2, nt=20000, boxdit_lmax=12)
    Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
    assert np.all(Yg == 0.0) and np.all(Wg == 0)


def test_matched_pulse_recovers_true_snr():
    # a noise-free pulse of amplitude C / sqrt(S) matched by a grid width at an
    # eligible start gives exactly SNR C (Sec. 4.3, Appendix A)
    nt = 40000
    plan = spd.spd_plan_create_boxdit([4, 6, 10], 8192, ndm=1, nt=nt)
    w, s = plan.widths()
    for S, Lsp in zip(w[::5], s[::5]):
        t0 = int(Lsp) * ((1000 + int(Lsp) - 1) // int(Lsp))
        x = np.zeros((1, nt), np.float32)
        x[0, t0:t0 + S] = np.float32(10.0 / np.sqrt(S))
        Yg, Wg = run_gpu(plan, x, 0.0, 1.0)
        assert abs(Yg[0, t0] - 10.0) < 1e-4, S
        assert w[Wg[0, t0]] == S, (S, w[Wg[0, t0]])


def test_candidates_from_tile_maxima():
    # the candidate step skips tiles by the kernel's tile maxima: it must give
    # exactly the oracle's rule applied to the kernel's own SNRs
    t = torch()
    ndm, nt = 3, 50001
    x = _data(ndm, nt, 21)
    plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=8192, ndm=ndm, nt=nt, boxdit_lmax=12)
    Yg, Wg, (Y, W, ws, mu_d, sg_d, xv) = run_gpu(plan, x, 0.0, 1.0, return_ws=True)
    cap = 1 << 16
    out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    for thr in (5.0, 8.0):
        spd.candidates(plan, Y, W, thr, 1, out, cnt, ws, use_tile_max=True)
        t.cuda.synchronize()
        n = int(cnt.item())
        rec = spd.records(out, min(n, cap))
        no, rows, starts, widx, snr = oracle.candidates(Yg.astype(np.float64), Wg.astype(np.int32), thr, 1)
        assert n == no and n > 0
        assert np.array_equal(rec["row"], rows) and np.array_equal(rec["start"], starts)
        assert np.array_equal(rec["width_idx"], widx) and np.array_equal(rec["snr"], snr.astype(np.float32))


def test_batch_agrees_with_per_range_search():
    """The batched search runs every level in one kernel per tile; a per-range
    search of a plan above level 4 runs the two-kernel form, which takes the
    levels from 4 on with tasks of several positions.  Both meet the oracle; their
    SNRs differ at most by the low 3 mantissa bits that carry a window rank."""
    t = torch()
    shapes = [(3, 50000), (2, 25001), (1, 140001)]
    xs = [_data(a, b, 950 + i) for i, (a, b) in enumerate(shapes)]
    b = spd.spd_batch_create(spd.SPD_ALGO_BOXDIT, 8192, [a for a, _ in shapes], [n for _, n in shapes],
                             boxdit_lmax=12)
    dx = [t.from_numpy(x).cuda() for x in xs]
    ys = [t.full(x.shape, -7.0, dtype=t.float32, device="cuda") for x in xs]
    wis = [t.zeros(x.shape, dtype=t.int16, device="cuda") for x in xs]
    mus = [t.zeros(x.shape[0], device="cuda") for x in xs]
    sgs = [t.ones(x.shape[0], device="cuda") for x in xs]
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws)
    spd.spd_batch_status(b, ws.data_ptr(), t.cuda.current_stream().cuda_stream)
    for r, x in enumerate(xs):
        plan = spd.spd_plan_create(algo=spd.SPD_ALGO_BOXDIT, s_end=8192, ndm=x.shape[0], nt=x.shape[1],
                                   boxdit_lmax=12)
        Ys, Ws = run_gpu(plan, x, 0.0, 1.0)
        Yb, Wb = ys[r].cpu().numpy(), wis[r].cpu().numpy().view(np.uint16)
        g = oracle_grid(plan)
        Yo, Wo, Y2o = oracle.search(x.astype(np.float64), g, 0.0, 1.0)
        assert_parity(Yb, Wb, Yo, Wo, Y2o, x.shape[1], ctx="batched, range %d" % r)
        fin = np.isfinite(Ys)
        assert np.array_equal(np.isfinite(Yb), fin), r
        assert np.all(np.abs(Yb[fin] - Ys[fin]) <= 2.0 ** -19 * np.abs(Ys[fin])), r
