"""Batched search (spd_batch_*): several DM ranges of different shapes in one
persistent launch give what a search per range gives (same kernels), match the
oracle, do not depend on the segment length, replay from a CUDA graph, and the
bounded ready-flag wait reports SPD_ERR_TIMEOUT without harming the context."""
import numpy as np
import pytest

import oracle
import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, assert_parity, oracle_grid, run_gpu, torch

pytestmark = pytest.mark.gpu

SHAPES = [(3, 50000), (2, 25001), (4, 12500), (1, 140001)]


def _ranges(seed):
    out = []
    for i, (ndm, nt) in enumerate(SHAPES):
        x = spd_synth.gaussian_noise(ndm, nt, seed + i, dtype=np.float64)
        tab = spd_synth.pulse_table(2 * ndm, ndm, nt, seed + 50 + i, width_range=(1, 300), snr_range=(7.0, 25.0))
        spd_synth.inject(x, tab, 1.0)
        out.append(x.astype(np.float32))
    return out


def _alloc(t, xs):
    dx = [t.from_numpy(x).cuda() for x in xs]
    ys = [t.full(x.shape, -7.0, dtype=t.float32, device="cuda") for x in xs]
    ws_ = [t.zeros(x.shape, dtype=t.int16, device="cuda") for x in xs]
    mus = [t.zeros(x.shape[0], device="cuda") for x in xs]
    sgs = [t.ones(x.shape[0], device="cuda") for x in xs]
    return dx, ys, ws_, mus, sgs


def _batch(name, s_end):
    kw = ALGOS[name](s_end)
    algo = kw.pop("algo")
    kw.pop("s_end")
    return spd.spd_batch_create(algo, s_end, [a for a, _ in SHAPES], [b for _, b in SHAPES], **kw)


@pytest.mark.parametrize("name,s_end", [("bd16", 4096), ("ig1", 8192), ("bd8", 60), ("dit", 8192)])
def test_batch_equals_per_range_search_and_oracle(name, s_end):
    t = torch()
    xs = _ranges(900)
    b = _batch(name, s_end)
    dx, ys, wis, mus, sgs = _alloc(t, xs)
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws)
    spd.spd_batch_status(b, ws.data_ptr(), t.cuda.current_stream().cuda_stream)
    for r, x in enumerate(xs):
        plan = spd.spd_plan_create(ndm=x.shape[0], nt=x.shape[1], **ALGOS[name](s_end))
        Ys, Ws = run_gpu(plan, x, 0.0, 1.0)
        assert np.array_equal(ys[r].cpu().numpy(), Ys), (name, r)
        assert np.array_equal(wis[r].cpu().numpy().view(np.uint16), Ws), (name, r)
    # one range against the oracle
    r = 1
    plan = spd.spd_plan_create(ndm=xs[r].shape[0], nt=xs[r].shape[1], **ALGOS[name](s_end))
    Yo, Wo, Y2o = oracle.search(xs[r].astype(np.float64), oracle_grid(plan))
    assert_parity(ys[r].cpu().numpy(), wis[r].cpu().numpy().view(np.uint16), Yo, Wo, Y2o, xs[r].shape[1], ctx=name)


def test_batch_segment_lengths_and_candidates():
    t = torch()
    xs = _ranges(910)
    b = _batch("bd16", 4096)
    dx, ys, wis, mus, sgs = _alloc(t, xs)
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    ref = None
    for seg in (16384, 32768, 131072, 262144):
        b.set_segment(seg)
        spd.batch_execute(b, dx, ys, wis, mus, sgs, ws)
        t.cuda.synchronize()
        got = [y.cpu().numpy().copy() for y in ys]
        if ref is None:
            ref = got
        for a, c in zip(ref, got):
            assert np.allclose(a, c, rtol=1e-6, atol=1e-6), seg
    # candidates of one range from the batch workspace's tile maxima
    r = 3
    cap = 4096
    out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
    cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.spd_batch_candidates(b, r, ys[r].data_ptr(), wis[r].data_ptr(), 6.0, 1, out.data_ptr(), cap,
                             cnt.data_ptr(), ws.data_ptr(), ws.numel(), 1, t.cuda.current_stream().cuda_stream)
    t.cuda.synchronize()
    n = int(cnt.item())
    rec = spd.records(out, min(n, cap))
    Yh = ys[r].cpu().numpy().astype(np.float64)
    ref_n = oracle.candidates(Yh, None, 6.0, 1, cap=cap)[0]
    assert n == ref_n


def test_batch_graph_replay():
    t = torch()
    xs = _ranges(920)
    b = _batch("ig1", 8192)
    dx, ys, wis, mus, sgs = _alloc(t, xs)
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    s = t.cuda.Stream()
    with t.cuda.stream(s):
        spd.batch_execute(b, dx, ys, wis, mus, sgs, ws, stream=s)  # first call outside the capture
    s.synchronize()
    ref = [y.cpu().numpy().copy() for y in ys]
    for y in ys:
        y.fill_(0.0)
    g = t.cuda.CUDAGraph()
    with t.cuda.graph(g, stream=s):
        spd.batch_execute(b, dx, ys, wis, mus, sgs, ws, stream=s)
    g.replay()
    t.cuda.synchronize()
    for a, y in zip(ref, ys):
        assert np.array_equal(a, y.cpu().numpy())


def test_batch_ready_flags_and_bounded_wait():
    t = torch()
    xs = _ranges(930)
    b = _batch("bd8", 2000)
    dx, ys, wis, mus, sgs = _alloc(t, xs)
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    st = t.cuda.current_stream().cuda_stream
    ready = [t.ones(1, dtype=t.int32, device="cuda") for _ in xs]
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws, readys=ready)
    spd.spd_batch_status(b, ws.data_ptr(), st)  # every flag set: no wait, status OK
    ref = [y.cpu().numpy().copy() for y in ys]
    # range 2's flag is never set: its wait runs out after 50 ms, the others finish
    b.set_wait_ns(50 * 10 ** 6)
    ready[2].zero_()
    for y in ys:
        y.fill_(-7.0)
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws, readys=ready)
    with pytest.raises(spd.SpdError) as e:
        spd.spd_batch_status(b, ws.data_ptr(), st)
    assert e.value.status == 6  # SPD_ERR_TIMEOUT
    for r, y in enumerate(ys):
        if r == 2:
            assert np.all(y.cpu().numpy() == -7.0)  # skipped: left unwritten
        else:
            assert np.array_equal(y.cpu().numpy(), ref[r])
    # the context is still usable
    ready[2].fill_(1)
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws, readys=ready)
    spd.spd_batch_status(b, ws.data_ptr(), st)
    assert np.array_equal(ys[2].cpu().numpy(), ref[2])


def test_batch_flags_set_while_the_search_waits():
    """Ranges copied in after the persistent search was launched: a copy stream
    uploads each range and then sets its ready flag with a 4-byte copy; the
    units of each range start when they see the flag, and the outputs equal the
    search of data already in place."""
    t = torch()
    xs = _ranges(950)
    b = _batch("bd16", 4096)
    dx, ys, wis, mus, sgs = _alloc(t, xs)
    ws = t.empty(b.workspace_size(), dtype=t.uint8, device="cuda")
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws)
    ref = [y.cpu().numpy().copy() for y in ys]
    hs = [t.from_numpy(x).pin_memory() for x in xs]
    for d in dx:
        d.zero_()
    for y in ys:
        y.fill_(-7.0)
    flags = t.zeros(len(xs), dtype=t.int32, device="cuda")
    one = t.ones(1, dtype=t.int32).pin_memory()
    b.set_wait_ns(5 * 10 ** 9)
    main, cs = t.cuda.current_stream(), t.cuda.Stream()
    t.cuda.synchronize()
    spd.batch_execute(b, dx, ys, wis, mus, sgs, ws, readys=[flags[r:r + 1] for r in range(len(xs))], stream=main)
    with t.cuda.stream(cs):
        for r, (h, d) in enumerate(zip(hs, dx)):
            d.copy_(h, non_blocking=True)
            flags[r:r + 1].copy_(one, non_blocking=True)
    cs.synchronize()
    spd.spd_batch_status(b, ws.data_ptr(), main.cuda_stream)
    for r, y in enumerate(ys):
        assert np.array_equal(y.cpu().numpy(), ref[r]), r
