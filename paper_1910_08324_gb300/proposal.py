"""Block proposals: a full-resolution search restricted to the blocks that a
trained network flags.

A block is 4096 input samples of one row; the network reads it as 256
samples after an x16 decimation.  ``flag_blocks`` decimates the series and
scores every block (``spd_net_decimate``, ``spd_net_forward``).
``search_flagged`` then searches the flagged blocks at full resolution
(``propose_and_search`` runs both as one C-ABI call, ``spd_propose_search``,
with the same geometry and the record map on the device).  Each flagged block
is copied into one compact series, together with

* the ``radius`` samples before it, so that the peak test of its first start
  sees its left neighbours;
* the ``radius`` starts after it (the right-hand neighbours of its peak test)
  and the samples that a boxcar starting at any of these can reach (up to the
  plan's widest width).

Samples past the row's ends are -inf, the same value the kernels use past a
row's end, so boxcars that would need them never count.  The compact series
is searched with one plan and the row's noise statistics.  Candidates that
start inside a block are then mapped back to (row, start).

``train`` fits the network with the gradient and Adam kernels, and
``label_blocks`` makes its labels.  A block is positive iff it holds the
start of an injected pulse that the plain search recovers.  ``match_pulses``
is the shared yardstick: it pairs candidates with injected pulses.

All arithmetic on samples runs in the library's kernels.  This module only
orders the calls, moves blocks with torch indexing and does host bookkeeping
on candidate lists.
"""
from __future__ import annotations

import functools

import numpy as np

from . import _binding as B

BLOCK = 4096      # input samples per block
DECIMATION = 16   # the network reads BLOCK / DECIMATION = 256 samples per block


def flag_blocks(params, x, mu, sigma, dtype: int = B.SPD_F32, threshold: float = 0.0, stream=None):
    """Logits [ndm, nt // 4096] of the blocks of ``x`` ([ndm, nt], nt a multiple of
    4096, stored as ``dtype``; ``mu``/``sigma`` float32 [ndm]) and the mask
    logit > threshold."""
    import torch
    ndm, nt = x.shape
    if nt % BLOCK:
        raise ValueError("the series length must be a multiple of %d" % BLOCK)
    d = torch.empty((ndm, nt // DECIMATION), dtype=torch.float32, device=x.device)
    B.net_decimate(x, mu, sigma, d, dtype=dtype, stream=stream)
    logits = torch.empty(ndm * (nt // BLOCK), dtype=torch.float32, device=x.device)
    B.net_forward(params, d.view(-1, BLOCK // DECIMATION), logits, stream=stream)
    logits = logits.view(ndm, nt // BLOCK)
    return logits, logits > threshold


def decimated_blocks(x, mu, sigma, dtype: int = B.SPD_F32, stream=None):
    """The network's input: float32 [ndm * nt / 4096, 256] decimated blocks of ``x``."""
    import torch
    ndm, nt = x.shape
    d = torch.empty((ndm, nt // DECIMATION), dtype=torch.float32, device=x.device)
    B.net_decimate(x, mu, sigma, d, dtype=dtype, stream=stream)
    return d.view(-1, BLOCK // DECIMATION)


def plan_geometry(grid: dict):
    """(widest width, largest start separation) of a plan grid (``spd_plan_create``
    keywords without the shape)."""
    return _geometry(tuple(sorted(grid.items())))


@functools.lru_cache(maxsize=64)
def _geometry(key):
    p = B.spd_plan_create(ndm=1, nt=1 << 16, **dict(key))
    try:
        w, sep = p.widths()
        return int(w[-1]), int(sep.max())
    finally:
        p.close()


def select_blocks(logits, threshold: float = 0.0, stream=None):
    """Device list (int64, increasing) of the ids row * blocks_per_row + block of
    the blocks whose logit exceeds ``threshold`` (``spd_net_select``)."""
    import torch
    flat = logits.reshape(-1)
    ids = torch.empty(flat.numel(), dtype=torch.int64, device=flat.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=flat.device)
    B.net_select(flat, threshold, ids, cnt, stream=stream)
    return ids[:int(cnt.item())]


def gather_blocks(x, ids, left: int, right: int, dtype: int, ld_align: int = 64, stream=None):
    """Compact copy of the blocks ``ids`` (``spd_net_gather``): [n, ld] rows holding
    ``left`` samples before each block, the block and ``right`` samples after it
    (-inf outside the series); ``ld`` rounds the row length up to ``ld_align``
    samples so that rows stay 16-byte aligned.  Returns (rows, row length)."""
    import torch
    width = left + BLOCK + right
    ld = -(-width // ld_align) * ld_align
    out = torch.empty((ids.numel(), ld), dtype=x.dtype, device=x.device)
    B.net_gather(x, ids, ids.numel(), BLOCK, left, width, out, dtype=dtype, stream=stream)
    return out, width


def search_flagged(x, ids, mu, sigma, grid: dict, threshold: float = 6.0, radius: int = 1,
                   cap: int = 1 << 22, noise_mode: int = 0, stream=None):
    """Search the blocks ``ids`` (``select_blocks``) of ``x`` ([ndm, nt]) with the
    plan grid ``grid`` (``spd_plan_create`` keywords: algo, s_end, boxdit_lmax,
    ..., dtype): one ``spd_search_blocks`` call (gather, search, candidates with
    the record map, on the device).  ``mu``/``sigma`` are the full series'
    statistics: [ndm] (white) or [ndm, n_widths] of the same grid (``noise_mode``
    1).  The context before a block is a whole number of the grid's largest
    start separation, so every level's starts fall where they fall in a search
    of the whole row and each block gets the outputs the plain search gives it.
    Returns the candidate records (numpy, rows and starts of ``x``, sorted by row
    and start)."""
    import torch
    n = ids.numel()
    if n == 0:
        return np.zeros(0, B.CANDIDATE_DTYPE)
    lend, sep = plan_geometry(grid)
    if BLOCK % sep:
        raise ValueError("grid start separation %d does not divide the %d-sample block" % (sep, BLOCK))
    prop, ws = _proposal(grid, x, radius, need=n)
    out = torch.empty(cap * B.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device=x.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=x.device)
    B.search_blocks(prop, x, mu, sigma, ids.contiguous(), out, cnt, ws, threshold, noise_mode=noise_mode,
                    stream=stream)
    k = int(cnt.item())
    if k > cap:
        raise B.SpdError(5, "search_flagged: %d candidates exceed cap %d" % (k, cap))
    return B.records(out, k).copy()


_PROPOSALS = {}  # (grid, shape, radius, device) -> (spd_proposal, its workspace)


def _proposal(grid: dict, x, radius: int, need: int = 0):
    import torch
    ndm, nt = x.shape
    key = (tuple(sorted(grid.items())), ndm, nt, x.stride(0), radius, str(x.device))
    e = _PROPOSALS.get(key)
    if e is None or e[0].max_blocks < need:
        total = ndm * (nt // BLOCK)
        mb = min(total, max(need, 4096, total // 16))
        prop = B.spd_proposal_create(ndm=ndm, nt=nt, ld=x.stride(0), peak_radius=radius, max_blocks=mb, **grid)
        e = (prop, torch.empty(prop.workspace_size(), dtype=torch.uint8, device=x.device))
        _PROPOSALS[key] = e
    return e


def propose_and_search(params, x, mu_tab, sigma_tab, grid: dict, logit_threshold: float = 0.0,
                       threshold: float = 6.0, radius: int = 1, cap: int = 1 << 22, stream=None):
    """The proposal path through one C-ABI call (``spd_propose_search``):
    decimate and score every block, select those above ``logit_threshold`` and
    search them with per-width noise tables ``mu_tab``, ``sigma_tab`` ([ndm,
    n_widths] of ``grid``; the network reads the width-1 entries); records come
    back in the series' (row, start).  The proposal object and its workspace are
    kept per shape and grid (room for 1/16 of the blocks, grown when more are
    flagged).  Returns (records, number of searched blocks)."""
    import torch
    out = torch.empty(cap * B.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device=x.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=x.device)
    prop, ws = _proposal(grid, x, radius)
    try:
        nb = B.propose_search(prop, params, x, mu_tab, sigma_tab, out, cnt, ws, logit_threshold, threshold,
                              noise_mode=1, stream=stream)
    except B.SpdError as err:
        if err.status != 5:
            raise
        prop, ws = _proposal(grid, x, radius, need=err.n_blocks)  # more blocks flagged than it holds
        nb = B.propose_search(prop, params, x, mu_tab, sigma_tab, out, cnt, ws, logit_threshold, threshold,
                              noise_mode=1, stream=stream)
    k = int(cnt.item())
    if k > cap:
        raise B.SpdError(5, "propose_and_search: %d candidates exceed cap %d" % (k, cap))
    return B.records(out, k).copy(), nb


def score(rec, pulses, snr_judge, ndm: int, nt: int, judge_threshold: float = 6.0):
    """Detection figures of candidate records against injected pulses whose SNR
    under the ideal search is ``snr_judge`` (``pulse_snr`` with the exhaustive
    grid): recall of the pulses the ideal search finds (SNR >= judge_threshold),
    overall and by width class; the mean SNR loss 1 - SNR / ideal SNR of the
    recalled ones; and the false alarms, candidates starting in quiet blocks
    (neither the block nor the next one holds a pulse, so no boxcar starting
    there reaches a pulse)."""
    best, _ = match_pulses(rec, pulses)
    found = snr_judge >= judge_threshold
    det = found & (best > 0)
    bpr = nt // BLOCK
    busy = np.zeros(ndm * bpr + 1, bool)
    b = pulses["row"].astype(np.int64) * bpr + pulses["start"] // BLOCK
    busy[b] = True
    busy[(b - 1)[pulses["start"] // BLOCK > 0]] = True  # the block before, in the same row
    cb = rec["row"].astype(np.int64) * bpr + rec["start"] // BLOCK
    out = {"pulses": int(len(pulses)), "judge_found": int(found.sum()),
           "recall": float(det.sum() / max(found.sum(), 1)),
           "snr_loss": float(np.mean(1.0 - best[det] / snr_judge[det])) if det.any() else float("nan"),
           "false_alarms": int((~busy[cb]).sum()), "candidates": int(len(rec))}
    for lo, hi in ((1, 16), (16, 256), (256, 1 << 30)):
        s = found & (pulses["width"] >= lo) & (pulses["width"] < hi)
        out["recall_w%d_%d" % (lo, min(hi, 4096))] = float(det[s].sum() / max(s.sum(), 1))
    return out


def match_pulses(rec, pulses, width_ratio: float = 4.0):
    """Pair candidate records with injected pulses.  A candidate matches a pulse
    (row, start s0, width w) when it lies in the same row, starts in
    [s0 - w, s0 + w] and its width lies within a factor ``width_ratio`` of w.
    Returns (best matched SNR per pulse, 0 where none; bool per candidate: it
    matches some pulse)."""
    best = np.zeros(len(pulses), np.float64)
    hit = np.zeros(len(rec), bool)
    if len(rec) == 0 or len(pulses) == 0:
        return best, hit
    span = np.int64(1) << 40
    key = rec["row"].astype(np.int64) * span + rec["start"].astype(np.int64)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    pr = pulses["row"].astype(np.int64)
    ps = pulses["start"].astype(np.int64)
    pw = pulses["width"].astype(np.int64)
    lo = np.searchsorted(ks, pr * span + np.maximum(ps - pw, 0), side="left")
    hi = np.searchsorted(ks, pr * span + ps + pw, side="right")
    cnt = hi - lo
    tot = int(cnt.sum())
    if tot == 0:
        return best, hit
    pid = np.repeat(np.arange(len(pulses)), cnt)
    first = np.repeat(lo - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt)
    cid = order[first + np.arange(tot)]
    cw = rec["width"][cid].astype(np.float64)
    ok = (cw <= width_ratio * pw[pid]) & (cw * width_ratio >= pw[pid])
    np.maximum.at(best, pid[ok], rec["snr"][cid[ok]].astype(np.float64))
    hit[cid[ok]] = True
    return best, hit


def label_blocks(rec, pulses, ndm: int, nt: int):
    """Block labels [ndm * nt / 4096] (float32): 1 iff the block holds the start of
    a pulse that some candidate of ``rec`` recovers (``match_pulses``)."""
    y = np.zeros(ndm * (nt // BLOCK), np.float32)
    best, _ = match_pulses(rec, pulses)
    found = best > 0
    y[pulses["row"][found] * (nt // BLOCK) + pulses["start"][found] // BLOCK] = 1.0
    return y


_PERM_CACHE: dict = {}  # the permutation of the epoch last used (key, tensor)


def batch_indices(n: int, batch: int, seed: int, step: int, device=None):
    """Block indices of training step ``step`` (counting from 0): the steps of an
    epoch take consecutive slices of a permutation of the n blocks drawn from a
    generator seeded with (seed, epoch), so the schedule is a function of the
    step alone and a resumed run sees the batches an uninterrupted one would."""
    import torch
    per_epoch = max(n // batch, 1)
    epoch, k = divmod(step, per_epoch)
    key = (n, int(seed), epoch, str(device))
    perm = _PERM_CACHE.get("perm") if _PERM_CACHE.get("key") == key else None
    if perm is None:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) * 1000003 + epoch)
        perm = torch.randperm(n, generator=g, device=device)
        _PERM_CACHE["key"], _PERM_CACHE["perm"] = key, perm
    return perm[k * batch:(k + 1) * batch]


def train(params, X, y, steps: int, batch: int = 512, lr: float = 3e-3, seed: int = 0, m=None, v=None,
          step0: int = 0, stream=None):
    """Steps step0 .. step0 + steps - 1 of Adam on mini-batches of the decimated
    blocks ``X`` (float32 [n, 256]) with labels ``y`` (float32 [n])
    (``batch_indices``); updates ``params`` (and the moments ``m``, ``v``) in
    place.  Returns (mean loss of each step as a host list, m, v)."""
    import torch
    dev = params.device
    m = torch.zeros_like(params) if m is None else m
    v = torch.zeros_like(params) if v is None else v
    G = torch.empty_like(params)
    L = torch.empty(1, dtype=torch.float32, device=dev)
    ws = torch.empty(B.spd_net_gradient_workspace_size(), dtype=torch.uint8, device=dev)
    n = X.shape[0]
    losses = torch.empty(steps, dtype=torch.float32, device=dev)
    for i in range(steps):
        idx = batch_indices(n, batch, seed, step0 + i, device=dev)
        xb = X[idx].contiguous()
        yb = y[idx].contiguous()
        B.net_gradient_ordered(params, xb, yb, G, L, ws, stream=stream)  # deterministic: runs repeat exactly
        B.net_adam(params, m, v, G, idx.numel(), lr, step0 + i + 1, stream=stream)
        losses[i] = L[0] / idx.numel()
    return losses.cpu().tolist(), m, v


# checkpoints of training: magic, version, parameter count, step, seed, then the
# parameters and the two Adam moments as float32 (little-endian throughout)
_CKPT_MAGIC = b"SPDNETCK"
_CKPT_VERSION = 1


def save_checkpoint(path, params, m, v, step: int, seed: int):
    """Write the training state (weights, Adam moments, next step, schedule
    seed) to ``path`` as one flat binary file (atomically: a temporary file
    renamed over it)."""
    import os
    import struct
    arrs = [np.ascontiguousarray(t.detach().float().cpu().numpy(), dtype="<f4") for t in (params, m, v)]
    if not (arrs[0].size == arrs[1].size == arrs[2].size):
        raise ValueError("parameter and moment vectors differ in size")
    tmp = str(path) + ".tmp"
    with open(tmp, "wb") as f:
        f.write(_CKPT_MAGIC + struct.pack("<IIqq", _CKPT_VERSION, arrs[0].size, int(step), int(seed)))
        for a in arrs:
            f.write(a.tobytes())
    os.replace(tmp, path)


def load_checkpoint(path, device="cuda"):
    """(params, m, v, step, seed) from ``save_checkpoint``'s file, the vectors as
    float32 tensors on ``device``; ValueError for a file of another format."""
    import struct
    import torch
    with open(path, "rb") as f:
        raw = f.read()
    head = len(_CKPT_MAGIC) + struct.calcsize("<IIqq")
    if len(raw) < head or raw[:len(_CKPT_MAGIC)] != _CKPT_MAGIC:
        raise ValueError("not a proposal-network checkpoint: %s" % path)
    version, n, step, seed = struct.unpack("<IIqq", raw[len(_CKPT_MAGIC):head])
    if version != _CKPT_VERSION or len(raw) != head + 12 * n:
        raise ValueError("checkpoint %s: version %d, %d bytes for %d parameters" % (path, version, len(raw), n))
    vecs = [torch.from_numpy(np.frombuffer(raw, dtype="<f4", count=n, offset=head + 4 * n * i).copy()).to(device)
            for i in range(3)]
    return vecs[0], vecs[1], vecs[2], int(step), int(seed)


def pulse_snr(x, pulses, mu, sigma, grid: dict, noise_mode: int = 1, width_ratio: float = 4.0, stream=None):
    """SNR that a search with the plan grid ``grid`` measures for each injected
    pulse of ``x``: the largest output SNR over starts in [s0 - w, s0 + w] whose
    best width lies within a factor ``width_ratio`` of w (0 where none).  A
    window from s0 - w, rounded down to the grid's largest start separation, to
    past s0 + w, with the samples its boxcars reach, is gathered for each pulse
    (``spd_net_gather``) and all windows are searched with one plan; ``mu`` and
    ``sigma`` are the full series' statistics as in ``search_flagged``.  With the
    exhaustive grid this is the ideal search's SNR of the pulse."""
    import torch
    if len(pulses) == 0:
        return np.zeros(0)
    ndm, nt = x.shape
    dev = x.device
    dtype = grid.get("dtype", B.SPD_F32)
    lend, sep = plan_geometry(grid)
    wmax = int(pulses["width"].max())
    nst = 2 * wmax + 1 + sep
    width = nst + lend
    ld = -(-width // 64) * 64
    a0 = (np.maximum(pulses["start"] - pulses["width"], 0) // sep).astype(np.int64)  # window start / sep
    bpr = -(-nt // sep)
    ids = torch.as_tensor(pulses["row"].astype(np.int64) * bpr + a0, device=dev)
    xs = torch.empty((len(pulses), ld), dtype=x.dtype, device=dev)
    B.net_gather(x, ids, len(pulses), sep, 0, width, xs, dtype=dtype, stream=stream)
    rows = torch.as_tensor(pulses["row"].astype(np.int64), device=dev)
    plan = B.spd_plan_create(ndm=len(pulses), nt=width, ld=ld, **grid)
    try:
        Y = torch.empty(xs.shape, dtype=torch.float32, device=dev)  # outputs share the row stride
        W = torch.empty(xs.shape, dtype=torch.int16, device=dev)
        ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device=dev)
        B.execute(plan, xs, mu[rows].contiguous(), sigma[rows].contiguous(), Y, W, ws, stream=stream,
                  noise_mode=noise_mode)
        wt = torch.as_tensor(plan.widths()[0].astype(np.float64), device=dev)
    finally:
        plan.close()
    off = torch.as_tensor(pulses["start"] - pulses["width"] - a0 * sep, device=dev)  # window index of s0 - w
    pw = torch.as_tensor(pulses["width"].astype(np.float64), device=dev)
    j = torch.arange(nst, device=dev)[None, :]
    cw = wt[torch.clamp(W[:, :nst].long() & 0xFFFF, max=len(wt) - 1)]
    sel = ((j >= off[:, None]) & (j <= off[:, None] + 2 * pw[:, None]) & (cw <= width_ratio * pw[:, None])
           & (cw * width_ratio >= pw[:, None]))
    y = torch.where(sel, Y[:, :nst].double(), torch.zeros_like(cw))
    return torch.clamp(y.max(dim=1).values, min=0.0).cpu().numpy()
