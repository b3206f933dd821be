"""Host logic of the proposal workload (no GPU): the 1/f generator and its
boxcar-variance formula, block pulse tables, many-pulse injection, zero-DM
spikes, and the candidate/pulse bookkeeping of the proposal module."""
import numpy as np
import pytest

import spd_synth
from paper_1910_08324_gb300 import proposal as P

torch = pytest.importorskip("torch")


def test_red_noise_is_unit_variance_with_the_stated_boxcar_variance():
    nt = 1 << 15
    x = spd_synth.device_red_noise(128, nt, 5, device="cpu").double().numpy()
    assert np.allclose(x.std(axis=1, ddof=1), 1.0, atol=1e-6)
    c = np.concatenate([np.zeros((x.shape[0], 1)), np.cumsum(x, axis=1)], axis=1)
    for L in (1, 8, 256, 2048):
        emp = (c[:, L:] - c[:, :-L]).var()
        ref = spd_synth.red_boxcar_var([L], nt, device="cpu")[0]
        assert abs(emp / ref - 1.0) < 0.1, (L, emp, ref)
    # alpha = 0 is white noise without its mean (no DC bin): an L-sum has variance
    # L - L^2 / nt (up to the weight of the single Nyquist bin)
    L = np.array([1, 7, 100, 5000])
    assert np.allclose(spd_synth.red_boxcar_var(L, nt, alpha=0.0, device="cpu"), L - L * L / nt, rtol=2e-4)


def test_matched_amplitudes_reduce_to_white_noise():
    tab = spd_synth.pulse_table(20, 4, 1 << 14, 3, width_range=(1, 512))
    a = spd_synth.proposal_amplitudes(tab, 1 << 14, red=False, device="cpu")
    assert np.allclose(a, tab["snr"] / np.sqrt(tab["width"]))
    ar = spd_synth.proposal_amplitudes(tab, 1 << 14, red=True, device="cpu")
    assert np.all(ar >= a)


def test_block_pulses_lie_inside_their_blocks():
    p = spd_synth.block_pulses(16, 1 << 16, 4096, 9, frac=0.5)
    assert 0.3 * 256 < len(p) < 0.7 * 256
    assert np.all(p["start"] // 4096 == (p["start"] + p["width"] - 1) // 4096)
    assert np.all((p["width"] >= 1) & (p["width"] <= 2048)) and np.all((p["snr"] >= 5) & (p["snr"] <= 20))
    assert len(np.unique(p["row"] * 16 + p["start"] // 4096)) == len(p)


def test_inject_many_equals_a_loop():
    x = torch.zeros(5, 10000, dtype=torch.float32)
    tab = spd_synth.pulse_table(12, 5, 10000, 3, width_range=(1, 300), min_gap=10)
    amp = np.linspace(1, 2, 12)
    spd_synth.device_inject_many(x, tab, amp=amp, rows_per_chunk=2)
    ref = np.zeros((5, 10000))
    for p, a in zip(tab, amp):
        ref[p["row"], p["start"]:p["start"] + p["width"]] += a
    assert np.abs(x.numpy() - ref).max() < 1e-6


def test_zero_dm_spikes_hit_every_row_at_the_same_samples():
    x, sig = spd_synth.proposal_series(3, 1 << 14, 4, device="cpu", red=False, spike_frac=1e-2)
    idx = spd_synth.zero_dm_spikes(1 << 14, 1e-2, 4 + 104729)
    assert sig == 1.0 and len(idx) == round(1e-2 * (1 << 14))
    assert np.all(x[:, torch.as_tensor(idx)].numpy() > 5.0)


def _rec(rows, starts, widths, snrs):
    r = np.zeros(len(rows), P.B.CANDIDATE_DTYPE)
    r["row"], r["start"], r["width"], r["snr"] = rows, starts, widths, snrs
    return r


def test_match_label_and_score():
    pulses = np.zeros(3, spd_synth.PULSE_DTYPE)
    pulses["row"], pulses["start"], pulses["width"], pulses["snr"] = [0, 0, 1], [100, 9000, 5000], [10, 400, 64], 8
    rec = _rec([0, 0, 0, 1, 1, 1], [95, 9300, 9010, 5000, 5100, 30000], [12, 4000, 300, 64, 64, 1], [7, 9, 8, 10, 11, 6])
    best, hit = P.match_pulses(rec, pulses)
    # start 95 within [90, 110], width 12 within 4x of 10; 9300 misses on width; 5100 is past 5000 + 64
    assert np.allclose(best, [7, 8, 10]) and hit.tolist() == [True, False, True, True, False, False]
    y = P.label_blocks(rec, pulses, 2, 1 << 15)
    assert np.nonzero(y)[0].tolist() == [0, 2, 8 + 1]
    s = P.score(rec, pulses, np.array([8.0, 16.0, 5.0]), 2, 1 << 15)
    assert s["judge_found"] == 2 and s["recall"] == 1.0
    assert abs(s["snr_loss"] - np.mean([1 - 7 / 8, 1 - 8 / 16])) < 1e-12
    # quiet blocks: row 1 block 7 (30000) holds no pulse and precedes none; row 0's blocks 0, 1, 2 are busy
    assert s["false_alarms"] == 1


def test_batch_schedule_is_a_function_of_the_step():
    n, b = 1000, 128
    per_epoch = n // b
    seen = np.concatenate([P.batch_indices(n, b, 7, k, device="cpu").numpy() for k in range(per_epoch)])
    assert len(np.unique(seen)) == per_epoch * b  # an epoch never repeats a block
    late = P.batch_indices(n, b, 7, 3 * per_epoch + 2, device="cpu").numpy()
    P.batch_indices(n, b, 7, 0, device="cpu")  # another epoch in between
    assert np.array_equal(P.batch_indices(n, b, 7, 3 * per_epoch + 2, device="cpu").numpy(), late)
    assert not np.array_equal(P.batch_indices(n, b, 8, 2, device="cpu").numpy(),
                              P.batch_indices(n, b, 7, 2, device="cpu").numpy())


def test_checkpoint_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    vec = [torch.from_numpy(rng.normal(size=4817).astype(np.float32)) for _ in range(3)]
    path = tmp_path / "net.ckpt"
    P.save_checkpoint(path, *vec, step=1234, seed=99)
    p2, m2, v2, step, seed = P.load_checkpoint(path, device="cpu")
    assert step == 1234 and seed == 99
    for a, b in zip(vec, (p2, m2, v2)):
        assert torch.equal(a, b)
    assert path.stat().st_size == 8 + 24 + 3 * 4 * 4817
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(100))
    with pytest.raises(ValueError):
        P.load_checkpoint(bad, device="cpu")
