"""Proposal network on the GPU against its FP64 definition (oracle.net): logits,
gradients and Adam steps; the x16 decimation; and a short training run that
must learn to separate blocks holding a pulse from noise blocks."""
import numpy as np
import pytest

import paper_1910_08324_gb300 as spd
import spd_synth
from gpu_util import torch
from oracle import net

pytestmark = pytest.mark.gpu


def _blocks(n, seed, pulse_frac=0.5):
    """Decimated-domain blocks: N(0,1) plus, in a fraction, a boxcar pulse."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 256))
    y = (rng.random(n) < pulse_frac).astype(np.float32)
    for i in np.nonzero(y)[0]:
        w = int(rng.integers(1, 40))
        s = int(rng.integers(0, 256 - w))
        X[i, s:s + w] += rng.uniform(1.5, 4.0)
    return X.astype(np.float32), y


def _params(seed):
    th = net.init_params(seed)
    th[net.N_PARAMS - 17:net.N_PARAMS - 1] = np.random.default_rng(seed).normal(0.0, 0.5, 16)
    return th.astype(np.float32)


def test_forward_logits_match_oracle():
    t = torch()
    X, _ = _blocks(64, 1)
    th = _params(2)
    lg = t.empty(64, device="cuda")
    spd.net_forward(t.from_numpy(th).cuda(), t.from_numpy(X).cuda(), lg)
    g = lg.cpu().numpy()
    o = np.array([net.forward(th.astype(np.float64), x)[0] for x in X])
    assert np.all(np.abs(g - o) <= 1e-2 * np.maximum(1.0, np.abs(o))), np.max(np.abs(g - o))


def test_gradient_matches_oracle():
    t = torch()
    X, y = _blocks(16, 3)
    th = _params(4)
    G = t.empty(net.N_PARAMS, device="cuda")
    L = t.empty(1, device="cuda")
    spd.net_gradient(t.from_numpy(th).cuda(), t.from_numpy(X).cuda(), t.from_numpy(y).cuda(), G, L)
    lo, go = net.batch_gradient(th.astype(np.float64), X.astype(np.float64), y)
    gg = G.cpu().numpy() / 16
    assert abs(L.item() / 16 - lo) <= 1e-2 * max(1.0, abs(lo))
    assert np.linalg.norm(gg - go) <= 3e-2 * np.linalg.norm(go), (np.linalg.norm(gg - go), np.linalg.norm(go))
    # the head gradient is exact up to FP32 rounding
    assert np.allclose(gg[-17:], go[-17:], rtol=2e-2, atol=1e-4)


def test_adam_step_matches_oracle():
    t = torch()
    rng = np.random.default_rng(5)
    th = rng.normal(size=net.N_PARAMS).astype(np.float32)
    g = rng.normal(size=net.N_PARAMS).astype(np.float32)
    m = rng.normal(size=net.N_PARAMS).astype(np.float32) * 0.1
    v = np.abs(rng.normal(size=net.N_PARAMS)).astype(np.float32) * 0.01
    P, M, V, Gd = (t.from_numpy(a.copy()).cuda() for a in (th, m, v, g * 8))
    spd.net_adam(P, M, V, Gd, 8, 1e-3, 3)
    tho, mo, vo = net.adam(th.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                           g.astype(np.float64), 3, 1e-3)
    assert np.allclose(P.cpu().numpy(), tho, rtol=1e-5, atol=1e-6)
    assert np.allclose(M.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
    assert np.allclose(V.cpu().numpy(), vo, rtol=1e-5, atol=1e-8)


@pytest.mark.parametrize("dtype,code", [("f32", spd.SPD_F32), ("f16", spd.SPD_F16), ("u8", spd.SPD_U8)])
def test_decimation(dtype, code):
    t = torch()
    ndm, nt = 3, 4096 * 3 + 16 * 5
    x = spd_synth.gaussian_noise(ndm, nt, 6, dtype=np.float64)
    stored, vals = spd_synth.quantize(x if dtype == "u8" else 0.3 + 1.1 * x, dtype)
    mu, sg = ((spd_synth.U8_OFFSET, spd_synth.U8_SCALE) if dtype == "u8" else (0.3, 1.1))
    host = t.from_numpy(np.ascontiguousarray(stored))
    d = t.empty((ndm, nt // 16), device="cuda")
    spd.net_decimate(host.cuda(), t.full((ndm,), mu, device="cuda"), t.full((ndm,), sg, device="cuda"), d, dtype=code)
    ref = (vals[:, : (nt // 16) * 16].reshape(ndm, -1, 16).sum(axis=2) - 16 * mu) / (4 * sg)
    assert np.allclose(d.cpu().numpy(), ref, rtol=1e-5, atol=1e-4)


def test_training_separates_pulse_blocks():
    t = torch()
    X, y = _blocks(4096, 7)
    Xv, yv = _blocks(1024, 8)
    th = net.init_params(9)
    P = t.from_numpy(th).cuda()
    M = t.zeros_like(P)
    V = t.zeros_like(P)
    G = t.empty_like(P)
    L = t.empty(1, device="cuda")
    Xd, yd = t.from_numpy(X).cuda(), t.from_numpy(y).cuda()
    losses = []
    bs = 256
    for step in range(1, 201):
        i0 = ((step - 1) * bs) % len(X)
        spd.net_gradient(P, Xd[i0:i0 + bs], yd[i0:i0 + bs], G, L)
        spd.net_adam(P, M, V, G, bs, 3e-3, step)
        losses.append(L.item() / bs)
    lg = t.empty(len(Xv), device="cuda")
    spd.net_forward(P, t.from_numpy(Xv).cuda(), lg)
    acc = np.mean((lg.cpu().numpy() > 0) == (yv > 0.5))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:20]), (losses[:5], losses[-5:])
    assert acc > 0.9, acc


def test_ordered_gradient_equals_atomic_sum_and_repeats():
    t = torch()
    X, y = _blocks(3000, 13)
    th = _params(14)
    P_, Xd, yd = t.from_numpy(th).cuda(), t.from_numpy(X).cuda(), t.from_numpy(y).cuda()
    G1, L1 = t.empty(net.N_PARAMS, device="cuda"), t.empty(1, device="cuda")
    spd.net_gradient(P_, Xd, yd, G1, L1)
    ws = t.empty(spd.spd_net_gradient_workspace_size(), dtype=t.uint8, device="cuda")
    G2, L2 = t.empty_like(G1), t.empty_like(L1)
    G3, L3 = t.empty_like(G1), t.empty_like(L1)
    spd.net_gradient_ordered(P_, Xd, yd, G2, L2, ws)
    spd.net_gradient_ordered(P_, Xd, yd, G3, L3, ws)
    assert t.equal(G2, G3) and t.equal(L2, L3)  # the ordered sum repeats exactly
    assert t.allclose(G1, G2, rtol=1e-4, atol=1e-6) and t.allclose(L1, L2, rtol=1e-5)
