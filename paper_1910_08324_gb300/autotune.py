"""Launch-shape autotuner for the streaming searches (plans and batches).

A CTA of the BoxDIT/IGRID kernels searches one segment of a row; the segment
length trades the re-read of the widest boxcar after each segment (shorter
segments re-read more) against the number of CTAs (longer segments give fewer,
and a ragged last wave).  A batched search also sets how many persistent CTAs
share an SM (fewer leave each CTA more of the SM's issue slots and caches,
more hide more latency).  ``tune_segment`` times each candidate segment length,
``tune_launch`` each (segment, CTAs per SM) pair, with a caller-supplied timing
function; the fastest is kept and cached in a JSON file keyed by the search's
description (grid, dtype, range shapes), so a later run with the same key
reuses it without timing.  A CTA's thread count (256) and starts per thread (8)
are not tuned: one CTA step covers a 2 048-sample chunk, 8 starts per thread,
and the kernels' level layout (which thread owns which coarse position, which
warp builds levels 9 to 11) is built on that chunk.  The general BoxDIT kernel
(any other L^i_max) is the exception: its starts per CTA, a tile of
``BOXDIT_GENERAL_TILES``, are what ``spd_plan_set_segment`` sets for its plans,
and ``tune_segment`` tunes them like segment lengths.
"""
from __future__ import annotations

import json
import os
import tempfile

DEFAULT_CANDIDATES = (16384, 32768, 65536, 131072, 262144)
BOXDIT_GENERAL_TILES = (2048, 4096, 8192)  # starts per CTA of the general BoxDIT kernel


def key_of(algo: int, s_end: int, dtype: int, shapes, boxdit_lmax: int = 0, igrid_depth: int = 0,
           igrid_layers: int = 0) -> str:
    """Cache key: the grid, the input type and every range's (ndm, nt)."""
    sh = ",".join("%dx%d" % (int(a), int(b)) for a, b in shapes)
    return "a%d:s%d:k%d:d%d:p%d:t%d:%s" % (algo, s_end, boxdit_lmax, igrid_depth, igrid_layers, dtype, sh)


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict):
    """Atomic write (a temporary file renamed over the cache)."""
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_segment(key: str, set_segment, time_ms, candidates=DEFAULT_CANDIDATES, cache_path=None,
                 reps: int = 3, force: bool = False):
    """Returns ``(segment, timings)``.

    set_segment(seg) applies a candidate (it may raise for lengths the grid does
    not allow: those are skipped); time_ms() runs the search and returns its
    time in ms.  The minimum over ``reps`` runs is kept per candidate.  With a
    cache path, a cached choice for ``key`` is returned without timing (and the
    chosen length is applied) unless ``force``.
    """
    cache = load_cache(cache_path) if cache_path else {}
    if not force and key in cache:
        seg = int(cache[key]["segment"])
        set_segment(seg)
        return seg, cache[key].get("timings", {})
    timings = {}
    for seg in candidates:
        try:
            set_segment(int(seg))
        except Exception:
            continue
        timings[str(int(seg))] = min(float(time_ms()) for _ in range(max(1, reps)))
    if not timings:
        raise RuntimeError("no segment length could be applied")
    best = min(timings, key=lambda s: timings[s])
    set_segment(int(best))
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"segment": int(best), "timings": timings}
        save_cache(cache_path, cache)
    return int(best), timings


DEFAULT_CTAS = (0, 1, 2, 3)  # 0: as many as fit


def tune_launch(key: str, set_segment, set_ctas, time_ms, segments=DEFAULT_CANDIDATES, ctas=DEFAULT_CTAS,
                cache_path=None, reps: int = 3, force: bool = False):
    """Returns ``((segment, ctas_per_sm), timings)``: every pair of a segment
    length and a CTAs-per-SM setting is applied (set_segment / set_ctas; pairs
    either call rejects are skipped) and timed with time_ms() (minimum over
    ``reps``); the fastest is applied and, with a cache path, stored under
    ``key`` (a cached choice is applied without timing unless ``force``).
    Timings are keyed "segment/ctas"."""
    cache = load_cache(cache_path) if cache_path else {}
    if not force and key in cache and "ctas_per_sm" in cache[key]:
        seg, c = int(cache[key]["segment"]), int(cache[key]["ctas_per_sm"])
        set_segment(seg)
        set_ctas(c)
        return (seg, c), cache[key].get("timings", {})
    timings = {}
    for seg in segments:
        try:
            set_segment(int(seg))
        except Exception:
            continue
        for c in ctas:
            try:
                set_ctas(int(c))
            except Exception:
                continue
            timings["%d/%d" % (int(seg), int(c))] = min(float(time_ms()) for _ in range(max(1, reps)))
    if not timings:
        raise RuntimeError("no launch shape could be applied")
    best = min(timings, key=lambda k: timings[k])
    seg, c = (int(v) for v in best.split("/"))
    set_segment(seg)
    set_ctas(c)
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"segment": seg, "ctas_per_sm": c, "timings": timings}
        save_cache(cache_path, cache)
    return (seg, c), timings
