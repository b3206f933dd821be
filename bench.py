#!/usr/bin/env python3
"""Benchmark of the single-pulse-detection hot path on GB300.

One step = one pass of the whole path over one batch: boxcar search over the
plan's grid (ingest, per-width SNR, max/argmax, Y/W output) plus threshold /
peak-find candidates, i.e. one ``spd_search`` call through the C ABI.

Workload (default): SKA-MID-shaped lossy search, 4,096 DM trials x 1,048,576
samples at 64 us, N(0,1) noise with 500 rectangular pulses (widths log-uniform
1..4096, SNR U(6,20)), IGRID IG(1) with S_end = 8192, candidates above SNR 6.
The input (17.2 GB) is larger than L2, so no flush is needed between steps.

Metric: DM x time samples per second (whole job, all ranks); the JSON line also
carries x-real-time (the paper's SKA definition: samples/s x 64 us / 6000), the
mean SNR loss measured on the GPU on noise-free copies of the workload's pulses,
the roofline of the search kernel (CUDA events inside the timed region), the
end-to-end figure through the public API with host buffers, and the oracle's CPU
throughput on a bounded sample.

``--impl reference`` times the CPU oracle (the only reference this method has:
the paper's code is not available) on the same workload shape.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import spd_synth  # noqa: E402
from paper_1910_08324_gb300 import shard  # noqa: E402  (host-only helpers, no library load)

T_SAMP = 64e-6
SKA_DM = 6000
OUT_BYTES_PER_SAMPLE = 4 + 2  # f32 Y out, u16 W out (algorithmic, once each)
DTYPES = {"f32": (0, 4), "f16": (1, 2), "bf16": (2, 2), "u8": (3, 1)}  # spd_dtype, bytes per sample
METRIC = "DM x time samples/s"
# The arithmetic type of the path: every input type is converted exactly to f32 on
# load and every boxcar sum, SNR and maximum is an f32 operation (the proposal
# network multiplies bf16 operands into f32 sums); the stored input type is
# reported beside it as "input_dtype".
COMPUTE_DTYPE = "f32"
SM_MAX_HZ = 2070e6          # GB300 maximum SM clock
ALU_OPS_PER_CANDIDATE = 3    # add (the sum), scale, max: the least a boxcar candidate costs

ALGOS = {
    "ig1": dict(algo=2, igrid_depth=1, igrid_layers=4),
    "ig2": dict(algo=2, igrid_depth=2, igrid_layers=8),
    "ig3": dict(algo=2, igrid_depth=3, igrid_layers=16),
    "dit": dict(algo=2, igrid_depth=0, igrid_layers=1),
    "bd8": dict(algo=1, boxdit_lmax=8),
    "bd16": dict(algo=1, boxdit_lmax=16),
    "bd32": dict(algo=1, boxdit_lmax=32),
    "bd12": dict(algo=1, boxdit_lmax=12),  # any other even L^i_max: the general BoxDIT kernel
    "bd24": dict(algo=1, boxdit_lmax=24),
    "exh": dict(algo=0),
}
# the sources each search kernel family compiles from (a traffic record applies
# only while they are unchanged)
_CSRC = "paper_1910_08324_gb300/csrc/"
_COMMON = [_CSRC + "spd_common.cuh", _CSRC + "spd_internal.h"]
FAMILY_SOURCES = {
    "igrid": [_CSRC + "spd_igrid.cu", _CSRC + "spd_igrid.cuh", _CSRC + "spd_igrid_coded.cu"] + _COMMON,
    "boxdit": [_CSRC + "spd_boxdit.cu", _CSRC + "spd_boxdit_gen.cu"] + _COMMON,
    "exhaustive": [_CSRC + "spd_search.cu"] + _COMMON,
}
SEARCH_SOURCES = sorted({f for v in FAMILY_SOURCES.values() for f in v})


def algo_family(algo):
    return {0: "exhaustive", 1: "boxdit", 2: "igrid"}[ALGOS[algo]["algo"]]


def search_launches(algo, widths):
    """Kernel launches of one search: the general BoxDIT kernel (an L^i_max other
    than 8, 16 or 32) runs a plan above level 4 (more than the 5 k widths of levels
    0-4) as two launches, every other grid as one."""
    k = ALGOS[algo].get("boxdit_lmax")
    if ALGOS[algo]["algo"] == 1 and k not in (8, 16, 32) and len(widths) > 5 * k:
        return 2
    return 1


# uneven DM ranges of one batched search: (DM trials, time decimation) of a 2,097,152-sample base
BATCH_RANGES = [(1024, 1), (1024, 2), (768, 4), (512, 8), (256, 16)]
BATCH_BASE = 2097152
BATCH_S_END = 4096
TUNE_CACHE = os.path.join(ROOT, "paper_1910_08324_gb300", "_tune", "segments.json")
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ska_mid",
                    choices=["ska_mid", "exhaustive_small", "batched", "proposal", "noise_stats", "host_link"],
                    help="ska_mid: 4096 x 1M lossy search (default); exhaustive_small: 64 x 65536, widths 1..256")
    ap.add_argument("--algo", default="ig1", choices=sorted(ALGOS))
    ap.add_argument("--ndm", type=int, default=spd_synth.SKA_MID["ndm"])
    ap.add_argument("--nt", type=int, default=spd_synth.SKA_MID["nt"])
    ap.add_argument("--s-end", type=int, default=spd_synth.SKA_MID["s_end"])
    ap.add_argument("--threshold", type=float, default=6.0)
    ap.add_argument("--radius", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-chunks", type=int, default=4, help="row chunks of the end-to-end pipeline")
    ap.add_argument("--dtype", default="f32", choices=sorted(DTYPES),
                    help="storage type of the input samples")
    ap.add_argument("--cpu-rows", type=int, default=96)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="oracle time the cpu_baseline sample accumulates")
    ap.add_argument("--train-rows", type=int, default=3907,
                    help="proposal: rows of 1M samples to train on (3907 rows = 10^6 blocks of 4096 samples)")
    ap.add_argument("--train-steps", type=int, default=8000, help="proposal: Adam steps of 512 blocks")
    ap.add_argument("--logit-threshold", type=float, default=0.0, help="proposal: blocks above it are searched")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-loss", action="store_true")
    ap.add_argument("--no-components", action="store_true",
                    help="skip the noise-statistics pass timed beside the default step")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alu_peak_candidates(sm_count):
    """Candidates per second at the ALU roofline: every FP32 lane of every SM at
    the maximum clock, 3 lane operations per candidate."""
    return sm_count * 128 * SM_MAX_HZ / ALU_OPS_PER_CANDIDATE


def binding_roofline(cand_per_sample, bytes_per_sample, samples, kernel_ms, sm_count, hbm_peak_gbs):
    """Roofline of one search launch against the bound that binds it: the larger
    of its HBM time (algorithmic bytes at the measured copy rate) and its ALU time
    (candidates at the ALU peak).  ``frac`` is that bound's time over the measured
    time; both fractions are returned, with the balance point (candidates per
    sample at which the two times are equal)."""
    alu_peak = alu_peak_candidates(sm_count)
    t = kernel_ms / 1e3
    t_hbm = bytes_per_sample * samples / (hbm_peak_gbs * 1e9)
    t_alu = cand_per_sample * samples / alu_peak
    gbs = bytes_per_sample * samples / t / 1e9
    cps = cand_per_sample * samples / t
    r = {"frac_hbm": gbs / hbm_peak_gbs, "frac_alu": cps / alu_peak, "hbm_GBps": gbs, "candidates_per_s": cps,
         "balance_candidates_per_sample": alu_peak * bytes_per_sample / (hbm_peak_gbs * 1e9),
         "alu_peak_source": "%d SMs x 128 FP32 lanes x %.0f MHz / %d ops per candidate"
                            % (sm_count, SM_MAX_HZ / 1e6, ALU_OPS_PER_CANDIDATE)}
    if t_hbm >= t_alu:
        r.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak_gbs, "unit": "GB/s", "frac": gbs / hbm_peak_gbs})
    else:
        r.update({"bound": "alu", "achieved": cps, "peak": alu_peak, "unit": "candidates/s",
                  "frac": cps / alu_peak})
    return r


def source_hash(algo="ig1"):
    h = hashlib.sha256()
    for s in FAMILY_SOURCES[algo_family(algo)]:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(algo, ndm, nt):
    """Per-launch DRAM bytes of the search kernel from the committed ncu summary,
    if it was taken on the current kernel source and this algorithm (key: the
    algorithm, suffixed with the input type when it is not f32); else None."""
    p = os.path.join(ROOT, "profiles", "search_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(algo)
    if not e or e.get("source_hash") != source_hash(algo.split("_")[0]):
        return None
    return float(e["bytes_per_sample"]) * ndm * nt


MSD_SOURCES = ["paper_1910_08324_gb300/csrc/spd_msd.cu", "paper_1910_08324_gb300/csrc/spd_common.cuh",
               "paper_1910_08324_gb300/csrc/spd_internal.h"]


def recorded_msd_traffic(dtype, ndm, nt):
    """Per-launch DRAM bytes of the noise-statistics pass kernel from the committed
    ncu summary, if it was taken on the current sources and input type; else None."""
    p = os.path.join(ROOT, "profiles", "msd_pass_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        e = json.load(f).get("msd_pass_" + dtype)
    h = hashlib.sha256()
    for s in MSD_SOURCES:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    if not e or e.get("source_hash") != h.hexdigest()[:16]:
        return None
    return float(e["bytes_per_sample"]) * ndm * nt


class ClockSampler:
    """nvidia-smi clock/throttle sampling (every 20 ms) around the timed region.

    Each sample carries nvidia-smi's timestamp; ``begin()``/``end()`` mark the
    timed region on the host clock and the summary keeps the samples taken
    between the two marks (all samples when none fell inside, e.g. a region
    shorter than the sampling period)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=20):
        self.index = index
        self.period_ms = period_ms
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.t0 is not None and self.t1 is None:
            self.t1 = time.time()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _stamp(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((self._stamp(f[0]), float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if r[0] is not None and self.t0 is not None and self.t1 is not None
                  and self.t0 <= r[0] <= self.t1]
        use = inside or rows
        if not use:
            return None
        reasons = set()
        for r in use:
            for n, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted(reasons), "samples": len(use), "in_timed_region": bool(inside),
                "period_ms": self.period_ms}


def cpu_model() -> str:
    """Host CPU model name (lscpu), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_rate(x_rows, algo, s_end, mu=0.0, sigma=1.0, threads=0):
    """The oracle (definition form, FP64, OpenMP over rows) on a bounded sample."""
    import oracle
    kw = ALGOS[algo]
    if kw["algo"] == 2:
        g = oracle.grid_igrid(kw["igrid_depth"], kw["igrid_layers"], s_end)
    elif kw["algo"] == 1:
        g = oracle.grid_boxdit(kw["boxdit_lmax"], s_end)
    else:
        g = oracle.grid_exhaustive(s_end)
    xs = np.ascontiguousarray(x_rows, np.float64)
    t0 = time.perf_counter()
    oracle.search(xs, g, mu, sigma, threads=threads)
    dt = time.perf_counter() - t0
    return xs.size / dt, dt


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    ndm, nt = args.ndm, args.nt
    rows = min(args.cpu_rows, ndm)
    cores = os.cpu_count() or 1
    times = []
    for k in range(args.warmup + args.steps):
        x = spd_synth.gaussian_noise(rows, nt, spd_synth.SEED_BASE + 100 + k, dtype=np.float64)
        rate, dt = cpu_oracle_rate(x, args.algo, args.s_end)
        if k >= args.warmup:
            times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = rows * nt / (ms / 1e3)
    sample = "%d of %d rows x %d samples per step (oracle definition form, FP64)" % (rows, ndm, nt)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "ska_mid %dx%d" % (ndm, nt), "algo": args.algo, "s_end": args.s_end},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, torch, dist, spd, rank, world, local, dev):
    """Uneven DM ranges at their own decimations searched by one graph-captured
    persistent launch per step (plus each range's candidate step); the segment
    length comes from the autotuner."""
    from paper_1910_08324_gb300 import autotune
    algo = args.algo if args.algo.startswith("bd") else "bd16"
    kw = dict(ALGOS[algo])
    a = kw.pop("algo")
    dt_code, esize = DTYPES[args.dtype]
    shapes = [(n, BATCH_BASE // d) for n, d in BATCH_RANGES]
    b = spd.spd_batch_create(a, BATCH_S_END, [n for n, _ in shapes], [t for _, t in shapes], dtype=dt_code, **kw)
    xs, ys, wis, mus, sgs, tabs = [], [], [], [], [], []
    for r, (n, t) in enumerate(shapes):
        seed = spd_synth.SEED_BASE + 4 + 100 * r + 1000 * rank
        x = spd_synth.device_noise(n, t, seed, device=dev)
        tab = spd_synth.pulse_table(100, n, t, seed + 1, width_range=(1, BATCH_S_END), snr_range=(6.0, 20.0),
                                    min_gap=2 * 4600)
        spd_synth.device_inject(x, tab)
        xs.append(spd_synth.device_quantize(x, args.dtype))
        tabs.append(tab)
        ys.append(torch.empty((n, t), dtype=torch.float32, device=dev))
        wis.append(torch.empty((n, t), dtype=torch.int16, device=dev))
        if args.dtype == "u8":
            mus.append(torch.full((n,), spd_synth.U8_OFFSET, device=dev))
            sgs.append(torch.full((n,), spd_synth.U8_SCALE, device=dev))
        else:
            mus.append(torch.zeros(n, device=dev))
            sgs.append(torch.ones(n, device=dev))
    samples = sum(n * t for n, t in shapes)
    ws = torch.empty(b.workspace_size(), dtype=torch.uint8, device=dev)
    cap = 1 << 18
    outs = [torch.zeros(cap * 24, dtype=torch.uint8, device=dev) for _ in shapes]
    cnts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in shapes]
    stream = torch.cuda.Stream(dev)

    def search(st):
        spd.batch_execute(b, xs, ys, wis, mus, sgs, ws, stream=st)

    def step(st):
        search(st)
        for r in range(len(shapes)):
            spd.spd_batch_candidates(b, r, ys[r].data_ptr(), wis[r].data_ptr(), args.threshold, args.radius,
                                     outs[r].data_ptr(), cap, cnts[r].data_ptr(), ws.data_ptr(), ws.numel(),
                                     1, st.cuda_stream)

    def time_ms(fn, reps=1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn(stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        step(stream)  # first launches outside any capture
        key = autotune.key_of(a, BATCH_S_END, dt_code, shapes, boxdit_lmax=kw.get("boxdit_lmax", 0))
        (seg, ctas), timings = autotune.tune_launch(key, b.set_segment, b.set_ctas_per_sm, lambda: time_ms(search),
                                                    ctas=(0, 1, 2), cache_path=TUNE_CACHE, reps=2, force=True)
        step(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step(stream)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        clk.begin()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[2 * k].record(stream)
                graph.replay()
                ev[2 * k + 1].record(stream)
        torch.cuda.synchronize(dev)
        clk.end()
    total_ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps))
    if world > 1:
        total_ms = shard.max_over_ranks(total_ms, dist)
    ms_per_step = total_ms / args.steps
    value = samples * world / (ms_per_step / 1e3)
    search_ms = min(time_ms(search) for _ in range(3))
    widths, seps = spd.spd_plan_create(ndm=1, nt=shapes[0][1], s_end=BATCH_S_END, dtype=dt_code,
                                       algo=a, **kw).widths()
    cand_per_sample = float(np.sum(1.0 / seps))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    bps = esize + OUT_BYTES_PER_SAMPLE
    peak, peak_kind = measured_peaks()
    roofline = binding_roofline(cand_per_sample, bps, samples, search_ms, sm_count, peak)
    roofline.update({"traffic": None, "kernel": "batched search (%s)" % algo, "kernel_ms": search_ms,
                     "algorithmic_bytes_per_launch": bps * samples,
                     "hbm_peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                     if peak_kind == "measured" else "fallback 6800 GB/s"})
    n_cand = sum(int(c.item()) for c in cnts)
    # end to end: host inputs of every range (pinned).  The persistent search is
    # launched first and each range's units wait for its ready flag (a bounded
    # device wait); a copy stream copies the ranges in turn, each followed by a
    # 4-byte copy that sets its flag, so the search of a range overlaps the
    # copies of the later ones.  Then the candidate steps and the counts back.
    e2e = None
    if not args.no_e2e:
        hs = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in xs]
        for h, x in zip(hs, xs):
            h.copy_(x)
        ch = torch.zeros(len(shapes), dtype=torch.int64, pin_memory=True)
        flags = torch.zeros(len(shapes), dtype=torch.int32, device=dev)
        readys = [flags[r:r + 1] for r in range(len(shapes))]
        one = torch.ones(1, dtype=torch.int32, pin_memory=True)
        b.set_wait_ns(10 * 10 ** 9)
        cs = torch.cuda.Stream(dev)

        def e2e_step():
            with torch.cuda.stream(stream):
                flags.zero_()
                zeroed = torch.cuda.Event()
                zeroed.record(stream)
                spd.batch_execute(b, xs, ys, wis, mus, sgs, ws, readys=readys, stream=stream)
            cs.wait_event(zeroed)
            with torch.cuda.stream(cs):
                for r, (h, x) in enumerate(zip(hs, xs)):
                    x.copy_(h, non_blocking=True)
                    flags[r:r + 1].copy_(one, non_blocking=True)
            with torch.cuda.stream(stream):
                for r in range(len(shapes)):
                    spd.spd_batch_candidates(b, r, ys[r].data_ptr(), wis[r].data_ptr(), args.threshold,
                                             args.radius, outs[r].data_ptr(), cap, cnts[r].data_ptr(),
                                             ws.data_ptr(), ws.numel(), 1, stream.cuda_stream)
                for r, c in enumerate(cnts):
                    ch[r:r + 1].copy_(c, non_blocking=True)
            stream.synchronize()
            cs.synchronize()
            spd.spd_batch_status(b, ws.data_ptr(), stream.cuda_stream)  # raises if a wait ran out

        e2e_step()
        per_step = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            e2e_step()
            per_step.append(time.perf_counter() - t0)
        dt = statistics.mean(per_step)
        b.set_wait_ns(10 ** 9)
        e2e = {"value": samples / dt, "unit": "samples/s", "h2d_bytes_per_step": esize * samples,
               "d2h_bytes_per_step": 8 * len(shapes), "steps": args.e2e_steps, "ms_per_step": 1e3 * dt,
               "ms_median": 1e3 * statistics.median(per_step), "ms_steps": [round(1e3 * v, 2) for v in per_step],
               "api": "spd_batch_execute launched first with per-range ready flags; torch pinned H2D of each "
                      "range on a copy stream followed by its flag; spd_batch_candidates; D2H of counts"}
        del hs

    cpu = None
    if not args.no_cpu and rank == 0:
        done, spent = 0, 0.0
        while spent < args.cpu_seconds:
            for r, (n, t) in enumerate(shapes):
                xr = xs[r][: max(1, 24 >> r)].float().cpu().numpy()
                _, dtc = cpu_oracle_rate(xr, algo, BATCH_S_END, float(mus[r][0]), float(sgs[r][0]))
                done += xr.size
                spent += dtc
        cpu = {"value": done / spent, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": "%d samples: 24/12/6/3/1 rows of the five ranges per pass, %s grid, FP64, %.1f s"
                         % (done, algo, spent)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": COMPUTE_DTYPE, "input_dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "batched: 5 DM ranges %s at decimations 1/2/4/8/16 of %d samples, one "
                                   "graph-captured persistent launch" % ("/".join(str(n) for n, _ in BATCH_RANGES),
                                                                         BATCH_BASE),
                       "algo": algo, "input_dtype": args.dtype, "s_end": BATCH_S_END, "samples": samples,
                       "candidates_per_sample": cand_per_sample,
                       "tuned": {"segment": seg, "ctas_per_sm": ctas if ctas else "as many as fit",
                                 "threads_per_cta": 256, "starts_per_thread": 8,
                                 "fixed": "threads and starts per thread: the level layout of a 2048-sample chunk"},
                       "autotune_ms": timings, "candidates_found": n_cand,
                       "parallelism": "dp%d (ranges per GPU)" % world,
                       "l2": "inputs larger than L2 (%.1f GB per GPU); no flush" % (esize * samples / 1e9)},
            "e2e": e2e, "gpu_launches": 1 + 3 * len(shapes), "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    return 0


def run_host_link(args, torch, rank, dev):
    """The host link that bounds the end-to-end figures: plain torch copies of the
    workload's input bytes (ndm x nt f32) between pinned host memory and the device,
    each copy timed alone (synchronised wall time), with no library kernel in the
    process.  Prints the GB/s of every copy."""
    if rank != 0:
        return 0
    n = args.ndm * args.nt
    x = torch.empty(n, dtype=torch.float32, device=dev)
    h = torch.empty(n, dtype=torch.float32, pin_memory=True)
    h.fill_(1.0)
    q = n // 4

    def rates(dst, src, reps):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize(dev)
            out.append(round(src.numel() * src.element_size() / (time.perf_counter() - t0) / 1e9, 1))
        return out

    side = torch.cuda.Stream(dev)
    chunked = []
    for _ in range(6):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(side):
            for c in range(4):
                x[c * q:(c + 1) * q].copy_(h[c * q:(c + 1) * q], non_blocking=True)
        torch.cuda.synchronize(dev)
        chunked.append(round(4 * n / (time.perf_counter() - t0) / 1e9, 1))
    res = {"h2d_whole": rates(x, h, 6), "h2d_first_quarter": rates(x[:q], h[:q], 6),
           "h2d_last_quarter": rates(x[3 * q:], h[3 * q:], 6), "h2d_4_chunks_side_stream": chunked,
           "d2h_whole": rates(h, x, 3), "h2d_whole_after_d2h": rates(x, h, 6)}
    line = {"metric": "host link GB/s per copy", "unit": "GB/s", "bytes": 4 * n, "workload": "host_link",
            "higher_is_better": True, "copies": res, "host_cores": os.cpu_count() or 1, "cpu_model": cpu_model()}
    print(json.dumps(line), flush=True)
    return 0


def run_noise_stats(args, torch, dist, spd, rank, world, local, dev):
    """Noise statistics (Sec. 4.5) of the search's input: one step = one
    ``spd_noise_stats`` call of one pass (every decimation level of every row,
    then the per-width table) over the workload's rows (default 4096 x 1M samples
    of N(0,1) noise with the SKA-MID-shaped pulses).  Each rank computes the
    statistics of its own rows (weak scaling).  A 3-pass call with 2-sigma
    rejection is timed beside it."""
    import oracle  # the CPU leg only
    ndm, nt = args.ndm, args.nt
    dt_code, esize = DTYPES[args.dtype]
    kw = dict(ALGOS[args.algo])
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, s_end=args.s_end, dtype=dt_code, **kw)
    widths = plan.widths()[0]
    nw = len(widths)
    seed = spd_synth.SEED_BASE + 7 + 1000 * rank
    x = spd_synth.device_noise(ndm, nt, seed, device=dev)
    spd_synth.device_inject(x, spd_synth.ska_mid_pulses(seed=seed, ndm=ndm, nt=nt))
    xf = x
    x = spd_synth.device_quantize(xf, args.dtype)
    if x is not xf:
        del xf
    mu = torch.empty((ndm, nw), dtype=torch.float32, device=dev)
    sg = torch.empty((ndm, nw), dtype=torch.float32, device=dev)
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)

    def step(passes=1):
        spd.noise_stats(plan, x, mu, sg, ws, outlier_sigma=2.0, max_passes=passes, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        clk.begin()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                ev[2 * k].record(stream)
                step()
                ev[2 * k + 1].record(stream)
        torch.cuda.synchronize(dev)
        clk.end()
    total_ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps))
    if world > 1:
        total_ms = shard.max_over_ranks(total_ms, dist)
    ms_per_step = total_ms / args.steps
    samples = ndm * nt
    value = samples * world / (ms_per_step / 1e3)
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(3)
        e1.record(stream)
    e1.synchronize()
    ms_3 = e0.elapsed_time(e1)
    # roofline: the pass kernel reads every sample once; the per-step time also
    # holds the (small) reset and table kernels, so the achieved rate is a lower bound
    peak, peak_src = measured_peaks()
    alg_bytes = esize * samples
    achieved = alg_bytes / (ms_per_step / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_msd_traffic(args.dtype, ndm, nt), "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src
                if peak_src == "measured" else "fallback 6.8 TB/s",
                "kernel": "msd_pass_kernel (+ reset and table kernels in the timed call)",
                "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": ms_per_step}
    e2e = None
    if not args.no_e2e:
        hx = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        hx.copy_(x)
        hm = torch.empty((ndm, nw), dtype=torch.float32, pin_memory=True)
        hs = torch.empty((ndm, nw), dtype=torch.float32, pin_memory=True)

        def e2e_step():
            with torch.cuda.stream(stream):
                x.copy_(hx, non_blocking=True)
                step()
                hm.copy_(mu, non_blocking=True)
                hs.copy_(sg, non_blocking=True)
            stream.synchronize()

        e2e_step()
        per = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            e2e_step()
            per.append(time.perf_counter() - t0)
        dt = statistics.mean(per)
        e2e = {"value": samples / dt, "unit": "samples/s", "h2d_bytes_per_step": esize * samples,
               "d2h_bytes_per_step": 8 * ndm * nw, "steps": args.e2e_steps, "ms_per_step": 1e3 * dt,
               "ms_median": 1e3 * statistics.median(per), "ms_steps": [round(1e3 * v, 2) for v in per],
               "api": "pinned H2D of the rows, spd_noise_stats (one pass), D2H of the mu and sigma tables"}
        del hx
    cpu = None
    if not args.no_cpu and rank == 0:
        nlev = 1
        while nlev < 16 and (1 << (nlev - 1)) < int(widths[-1]):
            nlev += 1
        done, spent, rows = 0, 0.0, 0
        while spent < args.cpu_seconds and rows < ndm:
            r = min(16, ndm - rows)
            xr = x[rows:rows + r].float().cpu().numpy().astype(np.float64)
            t0 = time.perf_counter()
            m, sd, n = oracle.msd_levels(xr, nlev, thr=2.0, max_passes=1)
            oracle.msd_table(m, sd, n, widths)
            spent += time.perf_counter() - t0
            done += xr.size
            rows += r
        cpu = {"value": done / spent, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": "%d rows x %d samples, one pass, FP64 (oracle msd_levels + msd_table), %.1f s"
                         % (rows, nt, spent)}
    if rank == 0:
        line = {
            "metric": "noise-statistics samples/s (one pass)", "value": value, "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": COMPUTE_DTYPE, "input_dtype": args.dtype, "data": "synthetic",
            "config": {"workload": "noise statistics %d DM x %d samples" % (ndm, nt), "input_dtype": args.dtype,
                       "algo": args.algo, "s_end": args.s_end, "widths": nw, "ms_3_passes_2sigma": ms_3,
                       "parallelism": "dp%d (rows per GPU)" % world,
                       "l2": "input larger than L2 (%.1f GB per GPU); no flush" % (esize * samples / 1e9)},
            "e2e": e2e, "gpu_launches": 3 * args.steps, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


NET_FLOPS_PER_BLOCK = 2 * 256 * 16 * 9 * (1 + 16 + 16) + 2 * 16  # three k=9 convolutions, 16 channels, head
PROPOSAL_GRID = dict(algo=1, s_end=4096, boxdit_lmax=16, dtype=1)      # BD-16 on FP16 samples


def run_proposal(args, torch, dist, spd, rank, world, local, dev):
    """Learned block proposals on 4096 x 1M FP16 rows of white + 1/f noise with
    0.1% zero-DM spikes: the network is trained on the GPU first (untimed; labels
    from the plain search), then a step decimates and scores every block and
    searches the flagged ones with BD-16 at full resolution.  The plain BD-16
    search of every block is timed beside it, and recall and SNR loss of both
    are judged by the exhaustive search of windows around the injected pulses."""
    from paper_1910_08324_gb300 import proposal as P
    ndm, nt = args.ndm, args.nt
    grid = dict(PROPOSAL_GRID)
    gx = dict(algo=0, s_end=2048, dtype=1)
    t_setup = time.perf_counter()

    def series(rows, seed, pulses):
        x, _ = spd_synth.proposal_series(rows, nt, seed, device=dev)
        spd_synth.device_inject_many(x, pulses, amp=spd_synth.proposal_amplitudes(pulses, nt, device=dev))
        return x.half()

    def tables(g, x):
        plan = spd.spd_plan_create(ndm=x.shape[0], nt=nt, **g)
        nw = len(plan.widths()[0])
        mu = torch.empty((x.shape[0], nw), device=dev)
        sg = torch.empty((x.shape[0], nw), device=dev)
        ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device=dev)
        spd.noise_stats(plan, x, mu, sg, ws)
        return plan, mu, sg, ws

    # the labels' plain search of 10^6 training blocks of red noise with spikes
    # finds ~8e7 candidates above SNR 6: room for 1.3e8 records (3.2 GB)
    cap = 1 << 27
    out = torch.empty(cap * 24, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)

    def plain(plan, x, mu, sg, ws, Y, W):
        spd.search(plan, x, mu, sg, Y, W, args.threshold, args.radius, out, cnt, ws, noise_mode=1)
        k = int(cnt.item())
        if k > cap:
            raise RuntimeError("plain search: %d candidates exceed the cap" % k)
        return spd.records(out, k).copy()

    # ---- training (untimed): half the blocks hold one pulse; labels from the plain search
    seed = spd_synth.SEED_BASE + 50 + 1000 * rank
    ptr = spd_synth.block_pulses(args.train_rows, nt, P.BLOCK, seed, frac=0.5)
    xtr = series(args.train_rows, seed + 1, ptr)
    plan, mu, sg, ws = tables(grid, xtr)
    Ytr = torch.empty(xtr.shape, device=dev)
    Wtr = torch.empty(xtr.shape, dtype=torch.int16, device=dev)
    y = P.label_blocks(plain(plan, xtr, mu, sg, ws, Ytr, Wtr), ptr, args.train_rows, nt)
    X = P.decimated_blocks(xtr, mu[:, 0].contiguous(), sg[:, 0].contiguous(), dtype=grid["dtype"])
    del xtr, Ytr, Wtr, plan, ws
    params = torch.from_numpy(spd_synth.net_init_params(seed + 2)).to(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    losses, _, _ = P.train(params, X, torch.from_numpy(y).to(dev), steps=args.train_steps, batch=512, lr=3e-3,
                           seed=seed + 3)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    training = {"blocks": int(X.shape[0]), "positives": int(y.sum()), "steps": args.train_steps, "batch": 512,
                "seconds": train_s, "blocks_per_s": args.train_steps * 512 / train_s,
                "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-100:]))}
    del X

    # ---- evaluation series: 500 pulses, widths log-uniform 1..2048, SNR 5..20 (against the noise at their width)
    pev = spd_synth.pulse_table(500, ndm, nt, seed + 4, width_range=(1, 2048), snr_range=(5.0, 20.0),
                                min_gap=2 * 8192)
    x = series(ndm, seed + 5, pev)
    plan, mu, sg, ws = tables(grid, x)
    _, mux, sgx, _ = tables(gx, x)
    sj = P.pulse_snr(x, pev, mux, sgx, gx)
    del mux, sgx
    Y = torch.empty(x.shape, device=dev)
    W = torch.empty(x.shape, dtype=torch.int16, device=dev)
    setup_s = time.perf_counter() - t_setup

    def prop_step():
        return P.propose_and_search(params, x, mu, sg, grid, logit_threshold=args.logit_threshold,
                                    threshold=args.threshold, radius=args.radius)

    for _ in range(args.warmup):
        prop_step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    times = []
    with ClockSampler(local) as clk:
        clk.begin()
        for _ in range(args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rec, nflag = prop_step()
            torch.cuda.synchronize(dev)
            times.append(time.perf_counter() - t0)
        clk.end()
    total = sum(times)
    if world > 1:
        total = shard.max_over_ranks(total, dist)
    ms_per_step = 1e3 * total / args.steps
    value = ndm * nt * world / (ms_per_step / 1e3)
    s_prop = P.score(rec, pev, sj, ndm, nt)

    # the method without the network: plain BD-16 search of every block (same noise tables)
    pt = []
    for k in range(max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        rp = plain(plan, x, mu, sg, ws, Y, W)
        torch.cuda.synchronize(dev)
        if k:
            pt.append(time.perf_counter() - t0)
    s_plain = P.score(rp, pev, sj, ndm, nt)
    plain_ms = 1e3 * statistics.mean(pt)

    # per-kernel breakdown of one proposal step (CUDA events on the launching stream)
    st = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(st)
    d = P.decimated_blocks(x, mu[:, 0].contiguous(), sg[:, 0].contiguous(), dtype=grid["dtype"])
    ev[1].record(st)
    lg = torch.empty(d.shape[0], device=dev)
    spd.net_forward(params, d, lg)
    ev[2].record(st)
    ids = P.select_blocks(lg, args.logit_threshold)
    ev[3].record(st)
    torch.cuda.synchronize(dev)
    dec_ms, fwd_ms, sel_ms = (ev[i].elapsed_time(ev[i + 1]) for i in range(3))
    fw = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        spd.net_forward(params, d, lg)
        e1.record(st)
        e1.synchronize()
        fw.append(e0.elapsed_time(e1))
    fwd_ms = statistics.mean(fw)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    P.search_flagged(x, ids, mu, sg, grid, args.threshold, args.radius, noise_mode=1)
    torch.cuda.synchronize(dev)
    flagged_ms = 1e3 * (time.perf_counter() - t0)
    nblocks = d.shape[0]
    del d, lg

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = NET_FLOPS_PER_BLOCK * nblocks / (fwd_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "net_forward_kernel (BF16 mma.sync implicit GEMM)", "kernel_ms": fwd_ms,
                "algorithmic_flops_per_launch": NET_FLOPS_PER_BLOCK * nblocks,
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops (burst, of measured)" if peaks
                                else "fallback 1900 TFLOP/s"),
                "decimate_ms": dec_ms, "decimate_GBps": 2 * ndm * nt / (dec_ms / 1e3) / 1e9,
                "select_ms": sel_ms, "flagged_search_ms": flagged_ms}

    e2e = None
    if not args.no_e2e:
        # rows are independent: the copies of later row chunks overlap the proposal
        # search of the earlier ones (copy stream + events; records come back per chunk)
        xh = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        xh.copy_(x)
        nchunk = max(1, min(args.e2e_chunks, ndm))
        bounds = [(ndm * i // nchunk, ndm * (i + 1) // nchunk) for i in range(nchunk)]
        cs = torch.cuda.Stream(dev)
        comp = torch.cuda.current_stream(dev)

        def e2e_step():
            cs.wait_stream(comp)  # the previous step is done with x
            landed = []
            with torch.cuda.stream(cs):
                for r0, r1 in bounds:
                    x[r0:r1].copy_(xh[r0:r1], non_blocking=True)
                    e = torch.cuda.Event()
                    e.record(cs)
                    landed.append(e)
            parts = []
            for (r0, r1), e in zip(bounds, landed):
                comp.wait_event(e)
                r, _ = P.propose_and_search(params, x[r0:r1], mu[r0:r1], sg[r0:r1], grid,
                                            logit_threshold=args.logit_threshold, threshold=args.threshold,
                                            radius=args.radius, stream=comp)
                r = r.copy()
                r["row"] += r0
                parts.append(r)
            return np.concatenate(parts)

        same = bool(np.array_equal(e2e_step(), rec))  # chunked records = the whole-series step's
        torch.cuda.synchronize(dev)
        per, nrec = [], []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            nrec.append(len(e2e_step()))
            per.append(time.perf_counter() - t0)
        dt = statistics.mean(per)
        e2e = {"value": ndm * nt / dt, "unit": "samples/s", "h2d_bytes_per_step": 2 * ndm * nt,
               "d2h_bytes_per_step": int(24 * statistics.mean(nrec) + 16), "steps": args.e2e_steps,
               "ms_per_step": 1e3 * dt, "ms_median": 1e3 * statistics.median(per),
               "ms_steps": [round(1e3 * v, 2) for v in per], "chunks": nchunk,
               "records_equal_unchunked": same,
               "api": "torch pinned H2D per row chunk (copy stream) + one spd_propose_search C-ABI call per "
                      "chunk (proposal.propose_and_search, after its copy) + records to the host"}
        del xh

    cpu = None
    if not args.no_cpu and rank == 0:
        import oracle
        from oracle import net as onet
        g = oracle.grid_boxdit(16, 4096)
        lend, sep = P.plan_geometry(grid)
        done, spent, r = 0, 0.0, 0
        while done == 0 or spent < args.cpu_seconds:
            xr = x[r].float().cpu().numpy().astype(np.float64)
            m0, s0 = float(mu[r, 0]), float(sg[r, 0])
            t0 = time.perf_counter()
            dec = (xr.reshape(-1, 16).sum(axis=1) - 16 * m0) / (4 * s0)
            lgs = np.array([onet.forward(params.cpu().numpy().astype(np.float64), b)[0]
                            for b in dec.reshape(-1, 256)])
            flag = np.nonzero(lgs > args.logit_threshold)[0]
            if len(flag):
                rows = np.full((len(flag), sep + P.BLOCK + lend), -np.inf)
                for i, b in enumerate(flag):
                    a = b * P.BLOCK - sep
                    lo, hi = max(a, 0), min(a + rows.shape[1], nt)
                    rows[i, lo - a:hi - a] = xr[lo:hi]
                oracle.search(rows, g, np.repeat(mu[r:r + 1].cpu().numpy(), len(flag), 0),
                              np.repeat(sg[r:r + 1].cpu().numpy(), len(flag), 0), noise_mode=1)
            spent += time.perf_counter() - t0
            done += nt
            r += 1
        cpu = {"value": done / spent, "unit": "samples/s", "cores": 1, "kind": "oracle",
               "sample": "%d rows x %d samples: FP64 decimation, network forward per block (oracle.net) and "
                         "definition-form BD-16 search of the flagged blocks, %.1f s" % (r, nt, spent)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": COMPUTE_DTYPE, "input_dtype": "f16", "data": "synthetic",
            "config": {"workload": "proposal %d DM x %d FP16 samples, white + 1/f noise, 0.1%% zero-DM spikes, "
                                   "500 pulses (widths 1..2048, SNR 5..20)" % (ndm, nt),
                       "algo": "network proposals + bd16 (table noise)", "s_end": 4096,
                       "logit_threshold": args.logit_threshold, "threshold": args.threshold,
                       "peak_radius": args.radius, "blocks": nblocks, "blocks_searched": int(nflag),
                       "searched_fraction": nflag / nblocks,
                       "parallelism": "dp%d (rows per GPU)" % world,
                       "l2": "inputs larger than L2 (%.1f GB per GPU); no flush" % (2 * ndm * nt / 1e9),
                       "x_realtime_ska": value * T_SAMP / SKA_DM, "setup_s": setup_s},
            "proposal": s_prop, "plain": dict(s_plain, ms_per_step=plain_ms,
                                              value=ndm * nt / (plain_ms / 1e3)),
            "speedup_vs_plain": plain_ms / ms_per_step, "training": training,
            # per step: decimate, forward, select, gather, two row gathers, search, candidate count/scan/write
            "e2e": e2e, "gpu_launches": 10 * args.steps, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.workload == "exhaustive_small":
        args.ndm, args.nt, args.s_end, args.algo = 64, 65536, 256, "exh"
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import torch.distributed as dist

    import paper_1910_08324_gb300 as spd

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.workload == "batched":
        return run_batched(args, torch, dist, spd, rank, world, local, dev)
    if args.workload == "proposal":
        return run_proposal(args, torch, dist, spd, rank, world, local, dev)
    if args.workload == "noise_stats":
        return run_noise_stats(args, torch, dist, spd, rank, world, local, dev)
    if args.workload == "host_link":
        return run_host_link(args, torch, rank, dev)
    ndm, nt = args.ndm, args.nt
    kw = dict(ALGOS[args.algo])
    dt_code, esize = DTYPES[args.dtype]
    bytes_per_sample = esize + OUT_BYTES_PER_SAMPLE
    plan = spd.spd_plan_create(ndm=ndm, nt=nt, s_end=args.s_end, dtype=dt_code, **kw)
    widths, seps = plan.widths()
    cand_per_sample = float(np.sum(1.0 / seps))

    # inputs: every rank searches its own full-size block of DM trials (weak scaling)
    seed = spd_synth.SEED_BASE + 2 + 1000 * rank
    if args.workload == "exhaustive_small":
        xs, tab = spd_synth.exhaustive_small(seed=spd_synth.SEED_BASE + 1 + 1000 * rank)
        x = torch.from_numpy(xs).to(dev)
    else:
        tab = spd_synth.ska_mid_pulses(seed=seed, ndm=ndm, nt=nt)
        x = spd_synth.device_noise(ndm, nt, seed, device=dev)
        spd_synth.device_inject(x, tab)
    # stored samples of the requested type; noise statistics in stored units
    if args.dtype == "u8":
        mu = torch.full((ndm,), spd_synth.U8_OFFSET, device=dev)
        sg = torch.full((ndm,), spd_synth.U8_SCALE, device=dev)
    else:
        mu = torch.zeros(ndm, device=dev)
        sg = torch.ones(ndm, device=dev)
    xf = x                                     # float32 samples
    x = spd_synth.device_quantize(xf, args.dtype)  # the stored input (xf itself for f32)
    Y = torch.empty((ndm, nt), dtype=torch.float32, device=dev)
    W = torch.empty((ndm, nt), dtype=torch.int16, device=dev)
    ws = torch.empty(plan.workspace_size(), dtype=torch.uint8, device=dev)
    cap = 1 << 20
    out = torch.zeros(cap * 24, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def fused_step():
        spd.search(plan, x, mu, sg, Y, W, args.threshold, args.radius, out, cnt, ws, stream=sp)

    for _ in range(args.warmup):
        fused_step()
    torch.cuda.synchronize(dev)

    # timed region: K steps (search + candidates), each bracketed by events on the
    # launching stream.  When the working set (input + outputs) is smaller than
    # twice the L2, a 512 MiB buffer is written between steps (outside the events)
    # so that every step starts from a cold L2.
    flush = None
    if bytes_per_sample * ndm * nt < 2 * L2_BYTES:
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        clk.begin()
        for k in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev[3 * k].record(stream)
            spd.spd_execute(plan, x.data_ptr(), mu.data_ptr(), sg.data_ptr(), Y.data_ptr(),
                            W.data_ptr(), ws.data_ptr(), ws.numel(), sp)
            ev[3 * k + 1].record(stream)
            spd.spd_candidates(plan, Y.data_ptr(), W.data_ptr(), args.threshold, args.radius,
                               out.data_ptr(), cap, cnt.data_ptr(), ws.data_ptr(), ws.numel(), 1, sp)
            ev[3 * k + 2].record(stream)
        torch.cuda.synchronize(dev)
        clk.end()
    if world > 1:
        dist.barrier()
    search_ms = [ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(args.steps)]
    cand_ms = [ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(args.steps)]
    total_ms = sum(ev[3 * k].elapsed_time(ev[3 * k + 2]) for k in range(args.steps))
    if world > 1:
        total_ms = shard.max_over_ranks(total_ms, dist)
    ms_per_step = total_ms / args.steps
    samples_step = ndm * nt * world
    value = samples_step / (ms_per_step / 1e3)
    n_cand = int(cnt.item())

    # roofline of the dominant kernel (the search): algorithmic work / event time,
    # against the bound that binds the grid: its HBM time (input once, Y and W once)
    # or its ALU time (candidates x 3 lane operations), whichever is longer
    peak, peak_kind = measured_peaks()
    s_avg = statistics.mean(search_ms)
    traffic = recorded_traffic(args.algo if args.dtype == "f32" else "%s_%s" % (args.algo, args.dtype),
                               ndm, nt)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline = binding_roofline(cand_per_sample, bytes_per_sample, ndm * nt, s_avg, sm_count, peak)
    roofline.update({"traffic": traffic, "frac_of_nominal_7900": roofline["hbm_GBps"] / 7900.0,
                     "peak_source": ("%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                                     if peak_kind == "measured" else "fallback 6800 GB/s")
                     if roofline["bound"] == "hbm" else roofline["alu_peak_source"]})
    roofline.update({"kernel": "search (%s)" % args.algo, "kernel_ms": s_avg,
                     "candidates_ms": statistics.mean(cand_ms),
                     "algorithmic_bytes_per_launch": bytes_per_sample * ndm * nt})

    # mean SNR loss on noise-free copies of the workload's pulses (GPU search)
    loss = None
    if not args.no_loss and rank == 0:
        xf.zero_()
        spd_synth.device_inject(xf, tab)
        x.copy_(spd_synth.device_quantize(xf, args.dtype))
        fused_step()
        torch.cuda.synchronize(dev)
        lend = int(widths[-1])
        rs = []
        for p in tab:
            r, s, w = int(p["row"]), int(p["start"]), int(p["width"])
            a = max(0, s - lend)
            rs.append(float(Y[r, a:s + w].max().item()) / float(p["snr"]))  # SNR in units of sg
        loss = {"mean_snr_loss": float(1.0 - np.mean(rs)), "pulses": len(rs),
                "max_snr_loss": float(1.0 - np.min(rs)),
                "definition": "mean over the workload's pulses, noise-free, of 1 - RSNR/SNR"}
        if args.workload == "exhaustive_small":
            xf.copy_(torch.from_numpy(xs).to(dev))
        else:
            xf.copy_(spd_synth.device_noise(ndm, nt, seed, device=dev))
            spd_synth.device_inject(xf, tab)
        x.copy_(spd_synth.device_quantize(xf, args.dtype))

    # the noise-statistics pass (Sec. 4.5, the table-noise path's other hot kernel)
    # on the same resident rows, timed outside the step: 3 untimed passes, then 10
    # with CUDA events on the launching stream (the rows are larger than L2)
    components = None
    if not args.no_components and args.workload == "ska_mid":
        nw = len(widths)
        mut = torch.empty((ndm, nw), device=dev)
        sgt = torch.empty_like(mut)

        def ns_pass():
            spd.spd_noise_stats(plan, x.data_ptr(), 2.0, 1, mut.data_ptr(), sgt.data_ptr(), ws.data_ptr(),
                                ws.numel(), sp)

        for _ in range(3):
            ns_pass()
        torch.cuda.synchronize(dev)
        nev = [torch.cuda.Event(enable_timing=True) for _ in range(20)]
        for k in range(10):
            nev[2 * k].record(stream)
            ns_pass()
            nev[2 * k + 1].record(stream)
        torch.cuda.synchronize(dev)
        ns_ms = statistics.mean(nev[2 * k].elapsed_time(nev[2 * k + 1]) for k in range(10))
        ns_gbps = esize * ndm * nt / (ns_ms / 1e3) / 1e9
        components = {"noise_stats_pass": {
            "ms": ns_ms, "samples_per_s": ndm * nt / (ns_ms / 1e3), "achieved_GBps": ns_gbps, "peak": peak,
            "frac_hbm": ns_gbps / peak, "traffic": recorded_msd_traffic(args.dtype, ndm, nt),
            "algorithmic_bytes_per_launch": esize * ndm * nt,
            "kernel": "msd_pass (first pass of spd_noise_stats: level sums of every row, no rejection yet)",
            "timing": "outside the timed step, same resident rows, 10 passes after 3"}}
        del mut, sgt

    # end to end through the public API with host buffers (pinned), copies timed: the
    # rows go in chunks, each copied on a copy stream and searched on the compute
    # stream once its copy has landed, so copies overlap the searches of earlier chunks
    e2e = None
    if not args.no_e2e:
        xh = torch.empty((ndm, nt), dtype=x.dtype, pin_memory=True)
        xh.copy_(x)
        nck = max(1, min(args.e2e_chunks, ndm))
        bounds = [ndm * c // nck for c in range(nck + 1)]
        spans = list(zip(bounds, bounds[1:]))
        plans = [spd.spd_plan_create(ndm=b1 - b0, nt=nt, s_end=args.s_end, dtype=dt_code, **kw) for b0, b1 in spans]
        wse = torch.empty(max(pl.workspace_size() for pl in plans), dtype=torch.uint8, device=dev)
        outs = [torch.empty(cap * 24, dtype=torch.uint8, device=dev) for _ in spans]
        cnts = torch.zeros(nck, dtype=torch.int64, device=dev)
        cnt_h = torch.zeros(nck, dtype=torch.int64, pin_memory=True)
        out_h = torch.empty(nck * cap * 24, dtype=torch.uint8, pin_memory=True)
        cs = torch.cuda.Stream(dev)
        ks = torch.cuda.current_stream(dev)

        def e2e_step():
            for c, (b0, b1) in enumerate(spans):
                with torch.cuda.stream(cs):
                    x[b0:b1].copy_(xh[b0:b1], non_blocking=True)
                    landed = torch.cuda.Event()
                    landed.record(cs)
                ks.wait_event(landed)
                spd.search(plans[c], x[b0:b1], mu[b0:b1], sg[b0:b1], Y[b0:b1], W[b0:b1], args.threshold,
                           args.radius, outs[c], cnts[c:c + 1], wse, stream=ks)
            cnt_h.copy_(cnts, non_blocking=True)
            ks.synchronize()
            nbytes = 8 * nck
            for c in range(nck):
                k = min(int(cnt_h[c]), cap)
                out_h[c * cap * 24:c * cap * 24 + k * 24].copy_(outs[c][: k * 24])
                nbytes += 24 * k
            return nbytes

        e2e_step()  # first use of the chunk plans outside the timed region
        torch.cuda.synchronize(dev)
        d2h, per_step = [], []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            d2h.append(e2e_step())
            per_step.append(time.perf_counter() - t0)
        # every step counts: the mean step time (the median and each step are in the line too)
        dt = statistics.mean(per_step)
        if world > 1:
            dt = shard.max_over_ranks(dt, dist)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        x.copy_(xh, non_blocking=True)
        torch.cuda.synchronize(dev)
        h2d_gbps = esize * ndm * nt / (time.perf_counter() - t1) / 1e9
        e2e = {"value": samples_step / dt, "unit": "samples/s", "h2d_bytes_per_step": esize * ndm * nt,
               "d2h_bytes_per_step": int(statistics.mean(d2h)), "steps": args.e2e_steps,
               "ms_per_step": 1e3 * dt, "ms_median": 1e3 * statistics.median(per_step),
               "ms_steps": [round(1e3 * v, 2) for v in per_step], "chunks": nck,
               "h2d_GBps_one_copy": h2d_gbps,
               "api": "torch pinned H2D per row chunk (copy stream) + spd_search per chunk (C ABI, compute "
                      "stream, after its copy) + D2H of counts and records"}
        del xh, out_h, outs

    # oracle on the host cores, bounded sample (rank 0 only)
    cpu = None
    if not args.no_cpu and rank == 0:
        # batches of cpu_rows rows (cycling through the workload's rows) until
        # cpu_seconds of oracle time have accumulated
        rows = min(args.cpu_rows, ndm)
        done, spent, r0, batches = 0, 0.0, 0, 0
        while batches == 0 or spent < args.cpu_seconds:
            xs = x[r0:r0 + rows].float().cpu().numpy()
            _, dt = cpu_oracle_rate(xs, args.algo, args.s_end, float(mu[0]), float(sg[0]))
            done += xs.size
            spent += dt
            batches += 1
            r0 = (r0 + rows) % ndm
            if r0 + rows > ndm:
                r0 = 0
        x1 = x[:4].float().cpu().numpy()
        rate1, _ = cpu_oracle_rate(x1, args.algo, args.s_end, float(mu[0]), float(sg[0]), threads=1)
        cpu = {"value": done / spent, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "cpu_model": cpu_model(), "value_1thread": rate1,
               "sample": "%d batches of %d of %d rows x %d samples (%d row passes), %s grid, "
                         "definition form FP64, %.1f s of oracle time; 1-thread figure on 4 rows"
                         % (batches, rows, ndm, nt, batches * rows, args.algo, spent)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": COMPUTE_DTYPE, "input_dtype": args.dtype,
            "data": "synthetic",
            "config": {"workload": ("ska_mid %d DM x %d samples, 64 us, 500 pulses" % (ndm, nt))
                       if args.workload == "ska_mid" else
                       "exhaustive_small 64 DM x 65536 samples, 8 SNR-10 pulses, widths 1..256",
                       "algo": args.algo, "input_dtype": args.dtype, "s_end": args.s_end,
                       "l_end": int(widths[-1]),
                       "n_widths": int(len(widths)), "candidates_per_sample": cand_per_sample,
                       "threshold": args.threshold, "peak_radius": args.radius,
                       "candidates_found": n_cand, "parallelism": "dp%d (rows per GPU)" % world,
                       "l2": ("inputs larger than L2 (%.1f GB per GPU); no flush" % (esize * ndm * nt / 1e9))
                       if flush is None else "L2 flushed between steps (512 MiB write outside the timed events)",
                       "x_realtime_ska": value * T_SAMP / SKA_DM,
                       "x_realtime_batch": (nt * T_SAMP) / (ms_per_step / 1e3)},
            "snr_loss": loss,
            "components": components,
            "e2e": e2e,
            "gpu_launches": (search_launches(args.algo, widths) + 3) * args.steps,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
