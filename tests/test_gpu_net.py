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


# Element-wise bounds of the network parity.  Both sides round the same
# quantities to bf16 at the same points; the GPU sums in FP32, the oracle in
# FP64.  An FP32 sum of the 9- to 144-term convolutions differs from FP64 by a
# few 1e-7 relative, which moves a bf16 rounding (one bf16 ulp, 2^-8 relative)
# only when the sum lies within that distance of a rounding boundary: a few
# activations in 10^4.  One such flip moves a logit by at most ~1e-4 of its
# scale and a summed gradient entry by ~1e-4 of its tensor's scale, so the bounds
# are 1e-3 relative plus 1e-3 of the largest entry of the same parameter tensor
# (a norm bound would hide one wrong weight gradient; these do not).
LOGIT_RTOL = 1e-3
GRAD_RTOL, GRAD_SCALE_TOL = 1e-3, 1e-3


def _tensor_slices():
    o = 0
    for name, shp in net.SHAPES:
        n = int(np.prod(shp))
        yield name, slice(o, o + n)
        o += n


def test_forward_logits_match_oracle():
    t = torch()
    X, _ = _blocks(256, 1)
    th = _params(2)
    lg = t.empty(len(X), device="cuda")
    spd.net_forward(t.from_numpy(th).cuda(), t.from_numpy(X).cuda(), lg)
    g = lg.cpu().numpy().astype(np.float64)
    o = np.array([net.forward(th.astype(np.float64), x)[0] for x in X])
    err = np.abs(g - o) / np.maximum(1.0, np.abs(o))
    print("\nlogits: max rel err %.3g, 99th pct %.3g" % (err.max(), np.percentile(err, 99)))
    assert np.all(err <= LOGIT_RTOL), err.max()


@pytest.mark.parametrize("ordered", [False, True])
def test_gradient_matches_oracle_elementwise(ordered):
    t = torch()
    X, y = _blocks(16, 3)
    th = _params(4)
    G = t.empty(net.N_PARAMS, device="cuda")
    L = t.empty(1, device="cuda")
    P_, Xd, yd = t.from_numpy(th).cuda(), t.from_numpy(X).cuda(), t.from_numpy(y).cuda()
    if ordered:
        ws = t.empty(spd.spd_net_gradient_workspace_size(), dtype=t.uint8, device="cuda")
        spd.net_gradient_ordered(P_, Xd, yd, G, L, ws)
    else:
        spd.net_gradient(P_, Xd, yd, G, L)
    lo, go = net.batch_gradient(th.astype(np.float64), X.astype(np.float64), y)
    gg = G.cpu().numpy().astype(np.float64) / 16
    assert abs(L.item() / 16 - lo) <= 1e-5 * max(1.0, abs(lo))
    for name, sl in _tensor_slices():
        a, b = gg[sl], go[sl]
        tol = GRAD_RTOL * np.abs(b) + GRAD_SCALE_TOL * np.abs(b).max()
        err = np.abs(a - b)
        print("%s: max err %.3g of scale %.3g (bound %.3g)" % (name, err.max(), np.abs(b).max(), tol.min()))
        assert np.all(err <= tol), (name, int(np.argmax(err - tol)), float(err.max()), float(np.abs(b).max()))


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


@pytest.mark.parametrize("dtype,code", [("f32", spd.SPD_F32), ("f16", spd.SPD_F16), ("bf16", spd.SPD_BF16),
                                        ("u8", spd.SPD_U8)])
@pytest.mark.parametrize("nt", [4096 * 3 + 16 * 5, 4096 * 3 + 16 * 5 + 7])
def test_decimation_matches_oracle(dtype, code, nt):
    """net_decimate_kernel against oracle.net.decimate (FP64, from its definition),
    element by element, on the stored values of every input type; rows with a
    ragged tail (dropped) and per-row mu, sigma.  The GPU sums 16 exactly
    converted samples in FP32: |error| <= 16 ulp of the block sum."""
    t = torch()
    ndm = 3  # nt: 16-byte rows (vector loads) and rows of a ragged length (element loads)
    x = spd_synth.gaussian_noise(ndm, nt, 6, dtype=np.float64)
    if dtype == "u8":
        stored, vals = spd_synth.quantize(x, dtype)
        mu = np.full(ndm, spd_synth.U8_OFFSET, np.float64)
        sg = np.full(ndm, spd_synth.U8_SCALE, np.float64) * np.array([1.0, 0.9, 1.2])
    else:
        mu = np.array([0.3, -1.0, 2.0])
        sg = np.array([1.1, 0.6, 2.5])
        stored, vals = spd_synth.quantize(mu[:, None] + sg[:, None] * x, dtype)
    host = t.from_numpy(np.ascontiguousarray(stored).view(np.int16) if stored.dtype == np.uint16
                        else np.ascontiguousarray(stored))
    d = t.empty((ndm, nt // 16), device="cuda")
    spd.net_decimate(host.cuda(), t.from_numpy(mu.astype(np.float32)).cuda(),
                     t.from_numpy(sg.astype(np.float32)).cuda(), d, dtype=code)
    ref = net.decimate(vals, mu.astype(np.float32), sg.astype(np.float32))
    blocksum = np.abs(vals[:, : (nt // 16) * 16]).reshape(ndm, -1, 16).sum(axis=2)
    tol = (16 * 2.0 ** -23 * (blocksum + 16 * np.abs(mu)[:, None]) / (4 * sg[:, None]) + 2.0 ** -22 * np.abs(ref))
    err = np.abs(d.cpu().numpy() - ref)
    assert np.all(err <= tol + 1e-7), (float(err.max()), float((err / (tol + 1e-7)).max()))


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
