"""Seeded synthetic inputs for single-pulse detection.

Both the CUDA path's tests/bench and the CPU oracle take their inputs from here,
so this module holds no step of the search itself: it only draws noise and
injects pulses.

Signal model (Sec. 2.1 of the paper, "idealized signal model"): white Gaussian
noise of mean ``mu`` and deviation ``sigma`` plus rectangular pulses of width
``S`` whose amplitude is ``SNR * sigma / sqrt(S)`` (Eq. amplitudenormalization
with C = SNR), so that a boxcar matching the pulse exactly recovers ``SNR``.

Randomness: numpy's counter-based Philox generator for host arrays, torch's
Philox-based CUDA generator for device arrays; every entry point takes an
explicit seed.  Workload seeds are ``SEED_BASE + k``.

Workloads (synthetic stand-ins: the paper's SKA-MID-like data is an instrument
rate, not a downloadable set):
  * exhaustive_small: 64 DM trials x 65,536 samples, N(0,1), eight pulses of
    widths {1,3,7,16,33,64,100,200} and SNR 10.
  * ska_mid: 4,096 DM trials x 1,048,576 samples at 64 us, N(0,1), 500 pulses,
    widths log-uniform in 1..4096, SNR uniform in 6..20.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1910083240

PULSE_DTYPE = np.dtype([("row", np.int64), ("start", np.int64), ("width", np.int64),
                        ("snr", np.float64)])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def gaussian_noise(ndm: int, nt: int, seed: int, mu: float = 0.0, sigma: float = 1.0,
                   dtype=np.float32) -> np.ndarray:
    """``ndm x nt`` white Gaussian noise drawn on the host."""
    g = rng(seed)
    x = g.standard_normal((ndm, nt), dtype=np.float64)
    x *= sigma
    x += mu
    return x.astype(dtype, copy=False)


def pulse_table(n: int, ndm: int, nt: int, seed: int, widths=None, snrs=None,
                width_range=(1, 4096), log_uniform: bool = True, snr_range=(6.0, 20.0),
                min_gap: int = 0) -> np.ndarray:
    """Random pulse truth table ``(row, start, width, snr)``, sorted by (row, start).

    ``widths``/``snrs`` fix the values (cycled); otherwise widths are drawn
    log-uniformly (or uniformly) in ``width_range`` and SNRs uniformly in
    ``snr_range``.  Pulses of one row are at least ``min_gap + width`` apart and
    lie completely inside the row.
    """
    g = rng(seed)
    out = np.zeros(n, PULSE_DTYPE)
    placed: dict[int, list[tuple[int, int]]] = {}
    for i in range(n):
        if widths is not None:
            w = int(widths[i % len(widths)])
        elif log_uniform:
            lo, hi = math.log(width_range[0]), math.log(width_range[1] + 1)
            w = int(min(width_range[1], max(width_range[0], math.floor(math.exp(g.uniform(lo, hi))))))
        else:
            w = int(g.integers(width_range[0], width_range[1] + 1))
        snr = float(snrs[i % len(snrs)]) if snrs is not None else float(g.uniform(*snr_range))
        for _ in range(10000):
            r = int(g.integers(0, ndm))
            if nt - w <= 0:
                raise ValueError("pulse wider than the series")
            s = int(g.integers(0, nt - w + 1))
            ok = all(s + w + min_gap <= a or a + b + min_gap <= s for a, b in placed.get(r, []))
            if ok:
                placed.setdefault(r, []).append((s, w))
                break
        else:
            raise RuntimeError("could not place pulse %d" % i)
        out[i] = (r, s, w, snr)
    out.sort(order=("row", "start"))
    return out


def pulse_amplitude(width, snr, sigma=1.0):
    """Per-sample amplitude of a rectangular pulse of true SNR ``snr`` (Eq. amplitudenormalization)."""
    return snr * sigma / math.sqrt(width)


def inject(x: np.ndarray, table: np.ndarray, sigma: float = 1.0) -> np.ndarray:
    """Add the rectangular pulses of ``table`` to the host array ``x`` in place."""
    for p in table:
        a = pulse_amplitude(int(p["width"]), float(p["snr"]), sigma)
        r, s, w = int(p["row"]), int(p["start"]), int(p["width"])
        seg = x[r, s:s + w].astype(np.float64) + a
        x[r, s:s + w] = seg.astype(x.dtype)
    return x


def sliding_pulse_rows(S: int, n_shift: int, t0: int, nt: int, C: float = 1.0,
                       dtype=np.float64) -> np.ndarray:
    """Noise-free series, one per shift: row k holds a pulse [t0 + k, t0 + k + S).

    This is the test data of Sec. 4.1 (each pulse shift in its own series).
    """
    x = np.zeros((n_shift, nt), dtype=np.float64)
    a = pulse_amplitude(S, C)
    for k in range(n_shift):
        x[k, t0 + k:t0 + k + S] = a
    return x.astype(dtype)


# ----------------------------------------------------------------------------- workloads
def exhaustive_small(seed: int = SEED_BASE + 1, dtype=np.float32):
    """64 x 65,536 N(0,1) with eight SNR-10 pulses of widths {1,3,7,16,33,64,100,200}."""
    ndm, nt = 64, 65536
    x = gaussian_noise(ndm, nt, seed, dtype=np.float64)
    tab = pulse_table(8, ndm, nt, seed + 7, widths=[1, 3, 7, 16, 33, 64, 100, 200],
                      snrs=[10.0], min_gap=2 * 256)
    inject(x, tab)
    return x.astype(dtype), tab


SKA_MID = dict(ndm=4096, nt=1 << 20, t_samp=64e-6, n_pulses=500, width_range=(1, 4096),
               snr_range=(6.0, 20.0), s_end=8192)


def ska_mid_pulses(seed: int = SEED_BASE + 2, ndm: int = SKA_MID["ndm"], nt: int = SKA_MID["nt"],
                   n: int = SKA_MID["n_pulses"], min_gap: int = 2 * 9216):
    """The 500-pulse truth table of the SKA-MID-shaped workload."""
    return pulse_table(n, ndm, nt, seed, width_range=SKA_MID["width_range"],
                       snr_range=SKA_MID["snr_range"], min_gap=min_gap)


def device_noise(ndm: int, nt: int, seed: int, device="cuda", mu: float = 0.0,
                 sigma: float = 1.0, out=None):
    """``ndm x nt`` float32 N(mu, sigma^2) drawn on the device with a seeded torch generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    if out is None:
        out = torch.empty((ndm, nt), dtype=torch.float32, device=device)
    # fill row blocks so that the temporary memory stays bounded
    step = max(1, (1 << 28) // max(nt, 1))
    for r0 in range(0, ndm, step):
        blk = out[r0:r0 + step]
        torch.randn(blk.shape, generator=g, device=device, dtype=torch.float32, out=blk)
        if sigma != 1.0:
            blk.mul_(sigma)
        if mu != 0.0:
            blk.add_(mu)
    return out


def device_inject(x, table, sigma: float = 1.0):
    """Add the pulses of ``table`` to a device tensor ``x`` ([ndm, >= nt]) in place."""
    for p in table:
        a = pulse_amplitude(int(p["width"]), float(p["snr"]), sigma)
        r, s, w = int(p["row"]), int(p["start"]), int(p["width"])
        x[r, s:s + w] += a
    return x


# ---------------------------------------------------------------- reduced-precision inputs
# Storage types of the input samples (spd_dtype order) and their u8 digitisation.
U8_OFFSET, U8_SCALE = 128.0, 16.0  # u8 = clip(round_half_even(128 + 16 v), 0, 255) for N(0,1) v


def quantize(x: np.ndarray, dtype: str):
    """Store float samples as ``dtype`` ('f32', 'f16', 'bf16' or 'u8').

    Returns ``(stored, values)``: ``stored`` is the numpy array to upload (bf16
    as its uint16 bit patterns), ``values`` the float64 value of every stored
    sample (what a search of the stored data sees).  f16 and bf16 round to
    nearest even; u8 maps v to clip(round_half_even(128 + 16 v), 0, 255), so its
    noise statistics are mu = 128 mu_v, sigma = 16 sigma_v in stored units.
    """
    x = np.asarray(x)
    if dtype == "f32":
        s = x.astype(np.float32)
        return s, s.astype(np.float64)
    if dtype == "f16":
        s = x.astype(np.float16)
        return s, s.astype(np.float64)
    if dtype == "bf16":
        b = np.ascontiguousarray(x.astype(np.float32)).view(np.uint32)
        r = ((b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)).astype(np.uint16)
        vals = (r.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
        return r, vals
    if dtype == "u8":
        v = np.clip(np.rint(U8_OFFSET + U8_SCALE * np.asarray(x, np.float64)), 0, 255).astype(np.uint8)
        return v, v.astype(np.float64)
    raise ValueError("unknown dtype %r" % dtype)


def device_quantize(x, dtype: str):
    """Device counterpart of ``quantize`` for torch tensors (float32 in, stored type out;
    bf16 as torch.bfloat16).  Same rounding rules."""
    import torch
    if dtype == "f32":
        return x.float()
    if dtype == "f16":
        return x.half()
    if dtype == "bf16":
        return x.bfloat16()
    if dtype == "u8":
        return torch.clamp(torch.round(U8_OFFSET + U8_SCALE * x), 0, 255).to(torch.uint8)
    raise ValueError("unknown dtype %r" % dtype)


# ---------------------------------------------------------------- non-white inputs (proposal workload)
def device_red_noise(ndm: int, nt: int, seed: int, device="cuda", alpha: float = 1.0):
    """1/f^alpha noise (power spectrum proportional to f^-alpha) per row, shaped in the
    Fourier domain from seeded white noise and scaled to unit variance per row."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((ndm, nt), dtype=torch.float32, device=device)
    f = torch.fft.rfftfreq(nt, device=device)
    shape = torch.zeros_like(f)
    shape[1:] = f[1:] ** (-alpha / 2.0)
    step = max(1, (1 << 25) // max(nt, 1))
    for r0 in range(0, ndm, step):
        n = min(step, ndm - r0)
        w = torch.randn((n, nt), generator=g, device=device, dtype=torch.float32)
        v = torch.fft.irfft(torch.fft.rfft(w, dim=1) * shape, n=nt, dim=1)
        out[r0:r0 + n] = v / v.std(dim=1, keepdim=True)
    return out


def zero_dm_spikes(nt: int, frac: float, seed: int) -> np.ndarray:
    """Time indices of impulsive zero-DM interference: the same samples in every row."""
    n = int(round(frac * nt))
    return np.sort(rng(seed).choice(nt, n, replace=False)) if n > 0 else np.zeros(0, np.int64)


def proposal_series(ndm: int, nt: int, seed: int, device="cuda", red: bool = True, spike_frac: float = 1e-3,
                    spike_amp: float = 10.0):
    """Float32 rows of white N(0,1) + (red) unit-variance 1/f noise + zero-DM spikes of spike_amp
    noise deviations at spike_frac of the time samples.  Returns (x, sigma): the noise deviation
    (sqrt(2) with red noise) in which pulse amplitudes and SNRs are stated."""
    x = device_noise(ndm, nt, seed, device=device)
    sigma = 1.0
    if red:
        x += device_red_noise(ndm, nt, seed + 7919, device=device)
        sigma = math.sqrt(2.0)
    idx = zero_dm_spikes(nt, spike_frac, seed + 104729)
    if len(idx):
        import torch
        x[:, torch.as_tensor(idx, device=device)] += spike_amp * sigma
    return x, sigma


def device_inject_many(x, table, sigma: float = 1.0, amp=None, rows_per_chunk: int = 64):
    """Add many rectangular pulses to a float32 device tensor ``x`` [ndm, nt] in place:
    +a at each start and -a one past each end in an FP64 difference array, prefix-summed
    along time (row chunks bound the temporary memory).  ``amp``: per-pulse
    amplitudes; default the white-noise amplitude snr * sigma / sqrt(width)."""
    import torch
    if len(table) == 0:
        return x
    ndm, nt = x.shape
    dev = x.device
    r = torch.as_tensor(table["row"].astype(np.int64), device=dev)
    s = torch.as_tensor(table["start"].astype(np.int64), device=dev)
    w = torch.as_tensor(table["width"].astype(np.int64), device=dev)
    if amp is None:
        amp = table["snr"] * sigma / np.sqrt(table["width"].astype(np.float64))
    a = torch.as_tensor(np.asarray(amp, np.float64), device=dev)
    order = np.argsort(table["row"], kind="stable")
    rows_sorted = table["row"][order].astype(np.int64)
    order_d = torch.as_tensor(order, device=dev)
    for r0 in range(0, ndm, rows_per_chunk):
        n = min(rows_per_chunk, ndm - r0)
        i0, i1 = np.searchsorted(rows_sorted, [r0, r0 + n])
        if i1 == i0:
            continue
        sel = order_d[i0:i1]
        d = torch.zeros(n * (nt + 1), dtype=torch.float64, device=dev)
        rr = r[sel] - r0
        d.index_add_(0, rr * (nt + 1) + s[sel], a[sel])
        d.index_add_(0, rr * (nt + 1) + s[sel] + w[sel], -a[sel])
        x[r0:r0 + n] += torch.cumsum(d.view(n, nt + 1), dim=1)[:, :nt].to(x.dtype)
    return x


def block_pulses(ndm: int, nt: int, block: int, seed: int, frac: float = 0.5,
                 width_range=(1, 2048), snr_range=(5.0, 20.0)) -> np.ndarray:
    """Pulse table with one pulse, in a random ``frac`` of the ``block``-sample blocks,
    lying wholly inside its block: widths log-uniform in ``width_range``, SNRs uniform
    in ``snr_range``.  Sorted by (row, start)."""
    g = rng(seed)
    nb = nt // block
    hit = np.nonzero(g.random(ndm * nb) < frac)[0]
    n = len(hit)
    lo, hi = math.log(width_range[0]), math.log(width_range[1] + 1)
    w = np.clip(np.floor(np.exp(g.uniform(lo, hi, n))), width_range[0], width_range[1]).astype(np.int64)
    off = np.floor(g.random(n) * (block - w + 1)).astype(np.int64)
    out = np.zeros(n, PULSE_DTYPE)
    out["row"] = hit // nb
    out["start"] = (hit % nb) * block + off
    out["width"] = w
    out["snr"] = g.uniform(snr_range[0], snr_range[1], n)
    return out


def red_boxcar_var(widths, nt: int, alpha: float = 1.0, device="cuda") -> np.ndarray:
    """Expected variance of an L-sample sum of the unit-variance 1/f^alpha noise of
    ``device_red_noise``, for each L in ``widths``: the power p_k of frequency bin k
    (proportional to k^-alpha over k = 1..nt/2, summing to one) times the boxcar's
    power gain (sin(pi k L / nt) / sin(pi k / nt))^2, summed over k."""
    import torch
    u = np.unique(np.asarray(widths, np.int64))
    k = torch.arange(1, nt // 2 + 1, device=device, dtype=torch.float64)
    p = k ** (-alpha)
    p /= p.sum()
    th = math.pi * k / nt
    s2 = torch.sin(th) ** 2
    out = torch.empty(len(u), dtype=torch.float64, device=device)
    for i in range(0, len(u), 32):
        L = torch.as_tensor(u[i:i + 32], device=device, dtype=torch.float64)
        g = torch.sin(th[None, :] * L[:, None]) ** 2 / s2[None, :]
        out[i:i + 32] = (g * p[None, :]).sum(dim=1)
    return out.cpu().numpy()[np.searchsorted(u, np.asarray(widths, np.int64))]


def proposal_amplitudes(table, nt: int, red: bool = True, device="cuda") -> np.ndarray:
    """Per-sample amplitudes that give each pulse of ``table`` its SNR against the
    noise of ``proposal_series`` at the pulse's own width: unit white noise plus,
    with ``red``, unit-variance 1/f noise, so a w-sample sum has variance
    w + red_boxcar_var(w)."""
    w = table["width"].astype(np.float64)
    var = w + (red_boxcar_var(table["width"], nt, device=device) if red and len(table) else 0.0)
    return table["snr"] * np.sqrt(var) / w


# ---------------------------------------------------------------- proposal network weights
# Parameter layout of the proposal network (float32 vector): W1[16][9], b1[16],
# W2[16][16][9], b2[16], W3[16][16][9], b3[16], W4[16], b4.
NET_SHAPES = [("W1", (16, 1, 9)), ("b1", (16,)), ("W2", (16, 16, 9)), ("b2", (16,)), ("W3", (16, 16, 9)),
              ("b3", (16,)), ("W4", (16,)), ("b4", (1,))]


def net_init_params(seed: int) -> np.ndarray:
    """Seeded He-style initial weights of the proposal network (normal, deviation
    sqrt(2 / fan-in) for the weights; zero biases), float32 in the layout above."""
    g = np.random.default_rng(int(seed))
    parts = []
    for name, shp in NET_SHAPES:
        if name.startswith("W"):
            fan_in = shp[1] * shp[2] if len(shp) == 3 else shp[0]
            parts.append(g.normal(0.0, math.sqrt(2.0 / fan_in), shp).reshape(-1))
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    return np.concatenate(parts).astype(np.float32)
