"""spd_candidates_static: the candidate step without a caller-provided workspace.

Some callers cannot allocate device memory at the point where they select
candidates (a real-time pipeline that reserved its memory at start-up, a C
caller with no allocator for scratch space); this entry point keeps its scratch
in a fixed array inside the library.  Its records and count must equal those of
spd_candidates (which uses the workspace) exactly, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import ALGOS, run_gpu, torch

pytestmark = pytest.mark.gpu


def _records(out, n, cap):
    return spd.records(out, min(n, cap))


@pytest.mark.parametrize("name,s_end,thr,radius", [("ig1", 4096, 4.0, 1), ("bd16", 2000, 3.5, 0),
                                                   ("exh", 128, 4.5, 3)])
def test_static_scratch_candidates_equal_workspace_version(name, s_end, thr, radius):
    t = torch()
    ndm, nt = 6, 70001
    x = spd_synth.gaussian_noise(ndm, nt, 3141, dtype=np.float64)
    tab = spd_synth.pulse_table(10, ndm, nt, 3142, width_range=(1, 500), snr_range=(8, 20), min_gap=2048)
    spd_synth.inject(x, tab)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS[name](s_end))
    _, _, (Y, W, ws, *_ ) = run_gpu(plan, x.astype(np.float32), 0.0, 1.0, return_ws=True)
    cap = 1 << 16
    stream = t.cuda.current_stream().cuda_stream
    ref_out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
    ref_cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.candidates(plan, Y, W, thr, radius, ref_out, ref_cnt, ws)
    t.cuda.synchronize()
    n_ref = int(ref_cnt.item())
    assert n_ref > 0
    ref = _records(ref_out, n_ref, cap)
    for _ in range(2):  # the scratch keeps the previous call's contents; results must not depend on it
        out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
        cnt = t.full((1,), -1, dtype=t.int64, device="cuda")
        spd.spd_candidates_static(plan, Y.data_ptr(), W.data_ptr(), thr, radius, out.data_ptr(), cap,
                                  cnt.data_ptr(), stream)
        spd.spd_sync_status(plan, stream)
        n = int(cnt.item())
        assert n == n_ref
        assert np.array_equal(_records(out, n, cap), ref)


def test_static_scratch_at_its_maximum():
    """262,144 candidate tiles, the static maximum: one tile per short row, so the
    array's group sums and offsets past the first group and the scan's carry
    across passes of 1,024 groups are all used; records and count equal
    spd_candidates', on two calls in a row."""
    t = torch()
    ndm, nt = 262144, 64
    x = spd_synth.gaussian_noise(ndm, nt, 2718, dtype=np.float32)
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, **ALGOS["ig1"](8))
    _, _, (Y, W, ws, *_) = run_gpu(plan, x, 0.0, 1.0, return_ws=True)
    cap = 1 << 21
    stream = t.cuda.current_stream().cuda_stream
    ref_out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
    ref_cnt = t.zeros(1, dtype=t.int64, device="cuda")
    spd.candidates(plan, Y, W, 2.5, 1, ref_out, ref_cnt, ws)
    t.cuda.synchronize()
    n_ref = int(ref_cnt.item())
    assert 10000 < n_ref <= cap
    ref = _records(ref_out, n_ref, cap)
    assert ref["row"].max() > 250000  # records from the last groups of tiles
    for _ in range(2):
        out = t.zeros(cap * 24, dtype=t.uint8, device="cuda")
        cnt = t.full((1,), -1, dtype=t.int64, device="cuda")
        spd.spd_candidates_static(plan, Y.data_ptr(), W.data_ptr(), 2.5, 1, out.data_ptr(), cap,
                                  cnt.data_ptr(), stream)
        spd.spd_sync_status(plan, stream)
        assert int(cnt.item()) == n_ref
        assert np.array_equal(_records(out, n_ref, cap), ref)


def test_static_scratch_rejects_plans_beyond_its_size():
    # 262,144 candidate tiles of 16,384 starts is the static maximum
    plan = spd.spd_plan_create(ndm=262145, nt=16, **ALGOS["ig1"](8))
    with pytest.raises(spd.SpdError) as e:
        spd.spd_candidates_static(plan, 4096, 4096, 6.0, 1, 4096, 1, 4096, 0)
    assert e.value.status == 2
