"""Throughput benchmark of the PolariS hot path on GB300.

Workload (one "step" = one pass of the whole path over one batch): one 1-s
integration of the paper-shaped load - 4 IF streams (X0, X1, Y0, Y1), 2-bit
samples, 131072-point real FFT segments, 61 segments per IF (8 Msps), autos,
crosses and Stokes I, Q, U, V of both pairs - i.e. 4 x 61 x 131072 =
31,981,568 input samples per step.

  value  device-resident input (a 480 MB ring of distinct seconds, larger than
         L2, so every step reads its input from HBM), feed + integrate to device
         outputs through the C ABI, timed with CUDA events (forked from and joined
         back into the launching stream).  Consecutive steps are independent 1-s
         integrations; they alternate over --handles spectrometer handles on as many
         streams, as a streaming caller would run them, so that one integration's
         phase-2 tail and readout overlap the next one's phase 1.
  e2e    the same metric through the C ABI with pinned HOST buffers: host->device
         copy of the step's packed input and device->host copy of its autos,
         crosses and Stokes inside the timed region (--e2e-handles handles).

--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded sample of the same workload (the reference arm; there is no upstream code).

Multi-GPU (torchrun): the path does not need any exchange between GPUs, so each
rank runs an independent replica on its own GPU and data; value sums all ranks'
samples over the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import ctypes
import ctypes.util
import hashlib
import glob
import json
import math
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input Msample/s through unpack+FFT+correlate at 2^17 pt; fraction of roofline"
N_IF, BITS, N_FFT, SEGS = 4, 2, 131072, 61
SAMPLES_PER_IF = SEGS * N_FFT
SAMPLES_PER_STEP = N_IF * SAMPLES_PER_IF
WORDS_PER_IF = SAMPLES_PER_IF * BITS // 32
NBIN = N_FFT // 2 + 1
N_PAIR = 2
D2H_BYTES = NBIN * 4 * N_IF + NBIN * 8 * N_PAIR + NBIN * 16 * N_PAIR
H2D_BYTES = N_IF * WORDS_PER_IF * 4
CONFIG = {
    "workload": "4 IF x 2-bit x 131072-pt R2C FFT, 61 segments per IF = one 1-s integration at 8 Msps per step; "
                "4 autos + 2 complex crosses + Stokes I,Q,U,V (rectangular window)",
    "n_if": N_IF, "bits": BITS, "n_fft": N_FFT, "segments_per_integration": SEGS, "integrations_per_step": 1,
    "samples_per_step": SAMPLES_PER_STEP,
    "l2": "inputs larger than L2: 60 distinct seconds (480 MB ring) cycled, each step reads another second",
}
DEFAULT_HANDLES, DEFAULT_E2E_HANDLES = 3, 6
# With several integrations in flight, at most one phase-1 CTA per SM leaves every SM room for
# another integration's phase 2 (shared-memory-bound work beside FP32-bound work): 594k against
# 578k-583k Msample/s with three handles (one handle alone is 6% slower with the cap).
DEFAULT_CAPS = "1,0"


# ------------------------------------------------------------------------------------------
# algorithmic work (flops) per step, split by kernel
# ------------------------------------------------------------------------------------------
def algorithmic_flops():
    """Nominal flop counts: FFT 5 N log2 N / 2 per real segment (split between the two
    kernels by their radix stages: log2 N1 = 8 rows, log2 N2 = 9 columns), correlate
    32 flop per bin per segment-time for the four autos and two crosses, window 1 flop
    per sample."""
    segs = N_IF * SEGS
    fft_stage = segs * 5.0 * N_FFT / 2.0  # one radix-2 stage of all real segments
    n1_log, n2_log = 8, 9
    corr = SEGS * NBIN * 32.0
    window = float(SAMPLES_PER_STEP)
    return {
        "phase1_decode_rowdft": fft_stage * n1_log + window,
        "phase2_coldft_correlate": fft_stage * n2_log + corr,
        "readout_stokes": 0.0,
        "path": fft_stage * math.log2(N_FFT) + corr + window,
    }


def fp32_peak_tflops(num_sms: int, sm_mhz: float) -> float:
    """CUDA-core FP32 peak: SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return num_sms * 128 * 2 * sm_mhz * 1e6 / 1e12


KERNEL_SOURCES = {
    # files whose contents define each timed kernel (a traffic record is valid for these only)
    "phase1_decode_rowdft": ("polaris_device.cuh", "polaris_kernels.cuh", "polaris_n17.cu"),
    "phase2_coldft_correlate": ("polaris_device.cuh", "polaris_kernels.cuh", "polaris_n17.cu"),
    "readout_stokes": ("polaris_abi.cu",),
}


def source_digest(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_1412_1256_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        parts = line.split()
        if len(parts) == 2 and not line.startswith("#"):
            vals[parts[0]] = parts[1]
    if vals.get("source_digest") != source_digest(kernel):
        return None
    try:
        return float(vals["dram_bytes_per_segment_pair"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------------------------------
# clocks: read-only NVML queries in a sampling thread
# ------------------------------------------------------------------------------------------
class ClockSampler:
    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
               0x10: "sync_boost", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown", 0x100: "display_clock_setting"}

    def __init__(self, cuda_index: int, period_s: float = 0.0005):
        self.samples, self.reasons, self.max_mhz = [], 0, None
        self.period, self._stop = period_s, threading.Event()
        self.ok = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            # map the CUDA ordinal to the NVML one when CUDA_VISIBLE_DEVICES renumbers devices
            index = cuda_index
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis:
                ids = [v.strip() for v in vis.split(",") if v.strip()]
                if cuda_index < len(ids) and ids[cuda_index].isdigit():
                    index = int(ids[cuda_index])
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                return
            self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            self.lib, self.h = lib, h
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = mx.value
            self.ok = True
        except OSError:
            pass

    def _run(self):
        c = ctypes.c_uint()
        r = ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0:
                self.samples.append(c.value)
            if self.reason_fn is not None and self.reason_fn(self.h, ctypes.byref(r)) == 0:
                self.reasons |= r.value
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self.t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "samples": 0}
        names = [n for b, n in self.REASONS.items() if self.reasons & b and n != "gpu_idle"]
        return {"sm_mhz": float(statistics.median(self.samples)), "sm_max_mhz": self.max_mhz, "reasons": names,
                "samples": len(self.samples)}


class _GpmInfo(ctypes.Structure):
    _fields_ = [("shortName", ctypes.c_char_p), ("longName", ctypes.c_char_p), ("unit", ctypes.c_char_p)]


class _GpmMetric(ctypes.Structure):
    _fields_ = [("metricId", ctypes.c_uint), ("nvmlReturn", ctypes.c_int), ("value", ctypes.c_double),
                ("metricInfo", _GpmInfo)]


class _GpmMetricsGet(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint), ("numMetrics", ctypes.c_uint), ("sample1", ctypes.c_void_p),
                ("sample2", ctypes.c_void_p), ("metrics", _GpmMetric * 210)]


class LiveCounters:
    """Read-only NVML GPU performance-monitoring (GPM) counters over a stretch of live work:
    two counter samples around a region that runs unprofiled and unserialised, so the
    figures describe the schedule the timed region runs (kernels of several streams side by
    side), which a kernel profiler replaying launches one at a time does not see.  NVML
    reports DRAM bandwidth as a percentage of a theoretical maximum; bytes come from
    calibrating that percentage with a device copy of known size measured the same way."""
    METRICS = {"dram_bw_util_pct": 10, "sm_util_pct": 2, "sm_occupancy_pct": 3, "fp32_util_pct": 12}

    def __init__(self, cuda_index: int):
        self.ok, self.why = False, ""
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                self.why = "nvmlInit failed"
                return
            index = cuda_index
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis:
                ids = [v.strip() for v in vis.split(",") if v.strip()]
                if cuda_index < len(ids) and ids[cuda_index].isdigit():
                    index = int(ids[cuda_index])
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                self.why = "no NVML handle"
                return
            sup = (ctypes.c_uint * 2)(1, 0)  # {version, isSupportedDevice}
            if lib.nvmlGpmQueryDeviceSupport(h, sup) != 0 or not sup[1]:
                self.why = "GPM not supported on this device"
                return
            self.samples = [ctypes.c_void_p(), ctypes.c_void_p()]
            for smp in self.samples:
                if lib.nvmlGpmSampleAlloc(ctypes.byref(smp)) != 0:
                    self.why = "nvmlGpmSampleAlloc failed"
                    return
            self.lib, self.h, self.ok = lib, h, True
        except (OSError, AttributeError) as e:
            self.why = f"NVML GPM unavailable: {e}"

    def measure(self, torch, dev, run, prefill: int, min_s: float = 1.0):
        """Counters over a stretch of steady work: `prefill` calls of `run()` are queued before
        the first sample and more are queued until min_s seconds have passed on the host, so
        the device is busy with the same work at both samples (the counters' own sampling
        instants then do not matter); NVML wants more than 100 ms between samples."""
        torch.cuda.synchronize(dev)
        for _ in range(prefill):
            run()
        if self.lib.nvmlGpmSampleGet(self.h, self.samples[0]) != 0:
            return None
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < min_s:
            run()
        if self.lib.nvmlGpmSampleGet(self.h, self.samples[1]) != 0:
            return None
        torch.cuda.synchronize(dev)
        mg = _GpmMetricsGet()
        mg.version, mg.numMetrics = 1, len(self.METRICS)
        mg.sample1, mg.sample2 = self.samples[0].value, self.samples[1].value
        for k, mid in enumerate(self.METRICS.values()):
            mg.metrics[k].metricId = mid
        if self.lib.nvmlGpmMetricsGet(ctypes.byref(mg)) != 0:
            return None
        return {name: (float(mg.metrics[k].value) if mg.metrics[k].nvmlReturn == 0 else None)
                for k, name in enumerate(self.METRICS)}

    def close(self):
        if self.ok:
            for smp in self.samples:
                self.lib.nvmlGpmSampleFree(smp)


def _event_ms(torch, dev, run, calls: int) -> float:
    """Device milliseconds per call of `run()` (events on the current stream, after warm-up)."""
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        run()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(calls):
        run()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / calls


def live_dram(torch, dev, cuda_index, run, ms_per_call, units_per_call, unit_name):
    """DRAM bytes per unit of live work from NVML's DRAM-bandwidth percentage, taken in a
    steady state.  The percentage is turned into bytes per second with streams of known
    traffic on 1 GiB buffers (a copy: 2 GiB per call; a fill: 1 GiB written; a sum: 1 GiB
    read), each timed with events and sampled the same way; their agreement shows how
    linear the percentage is in bytes.  ms_per_call is the work's own measured time."""
    lc = LiveCounters(cuda_index)
    if not lc.ok:
        return {"unavailable": lc.why}
    try:
        gib = 1 << 30
        src = torch.empty(gib // 4, dtype=torch.float32, device=dev).fill_(1.0)
        dst = torch.empty_like(src)
        acc = torch.empty((), dtype=torch.float32, device=dev)
        streams = {"copy": (lambda: dst.copy_(src), 2 * gib), "write": (lambda: dst.fill_(2.0), gib),
                   "read": (lambda: torch.sum(src, 0, out=acc), gib)}
        cal = {}
        for name, (fn, nbytes) in streams.items():
            ms = _event_ms(torch, dev, fn, 20)
            m = lc.measure(torch, dev, fn, prefill=int(60 / ms) + 1)
            if not m or not m["dram_bw_util_pct"]:
                return {"unavailable": f"GPM metrics not returned ({name})"}
            gbs = nbytes / (ms * 1e-3) / 1e9
            cal[name] = {"gbs": gbs, "dram_bw_util_pct": m["dram_bw_util_pct"],
                         "gbs_per_pct": gbs / m["dram_bw_util_pct"]}
        del src, dst
        work = lc.measure(torch, dev, run, prefill=int(60 / ms_per_call) + 1)
        if not work or work["dram_bw_util_pct"] is None:
            return {"unavailable": "GPM metrics not returned (work)"}
        gbs_per_pct = cal["copy"]["gbs_per_pct"]
        gbs = gbs_per_pct * work["dram_bw_util_pct"]
        per_unit = gbs * 1e9 * (ms_per_call * 1e-3) / units_per_call
        spread = [c["gbs_per_pct"] for c in cal.values()]
        return {f"dram_bytes_per_{unit_name}": per_unit, "dram_gbs": gbs,
                f"dram_bytes_per_{unit_name}_range": [per_unit * min(spread) / gbs_per_pct,
                                                     per_unit * max(spread) / gbs_per_pct],
                "dram_bw_util_pct": work["dram_bw_util_pct"],
                "sm_util_pct": work["sm_util_pct"], "sm_occupancy_pct": work["sm_occupancy_pct"],
                "fp32_util_pct": work["fp32_util_pct"], "calibration": cal,
                "note": "NVML GPM counters (read-only), sampled twice while the device runs the timed "
                        "region's schedule unprofiled; the DRAM percentage is converted to bytes with "
                        "the copy's GB/s per percent (the range uses the fill's and the sum's)"}
    finally:
        lc.close()


# ------------------------------------------------------------------------------------------
# inputs
# ------------------------------------------------------------------------------------------
def slowest(dist, seconds: float) -> float:
    """The largest of every rank's time (gloo all-reduce MAX; one rank: itself)."""
    if dist is None:
        return float(seconds)
    import torch

    tt = torch.tensor([float(seconds)], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world: int, steps: int, samples_per_step: int, seconds: float) -> float:
    """Msample/s of all ranks together: every rank processes its own samples_per_step per
    step (weak scaling), over the slowest rank's time."""
    return world * steps * samples_per_step / seconds / 1e6


def make_unique_seconds(n_unique: int):
    from paper_1412_1256_gb300 import synth

    out = []
    for i in range(n_unique):
        packed, meta = synth.config_paper(seed=1256 + i, n_segments=SEGS, n_fft=N_FFT, n_if=N_IF, bits=BITS)
        out.append(np.stack(packed).view(np.int32))  # [N_IF, WORDS_PER_IF]
    return out


# ------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on a bounded sample
# ------------------------------------------------------------------------------------------
def time_oracle(unique, segs: int, repeats: int = 1):
    """Time the FP64 oracle on `segs` segments of one integration (4 IF), `repeats` times."""
    import oracle

    oracle.build()
    u = unique[0].view(np.uint32)
    n = segs * N_FFT
    packed = [np.ascontiguousarray(u[i, : n * BITS // 32]) for i in range(N_IF)]
    t0 = time.perf_counter()
    for _ in range(repeats):
        oracle.spectrometer(packed, BITS, N_FFT, n)
    dt = time.perf_counter() - t0
    return repeats * N_IF * n / dt / 1e6, dt


_ORACLE_INPUT = None


def _oracle_init(words):
    global _ORACLE_INPUT
    _ORACLE_INPUT = words


def _oracle_chunk(seg_range):
    """One worker's share: the oracle's whole path on segments [s0, s1) of one integration."""
    import oracle

    s0, s1 = seg_range
    wps = N_FFT * BITS // 32
    packed = [np.ascontiguousarray(_ORACLE_INPUT[i, s0 * wps:s1 * wps]) for i in range(N_IF)]
    oracle.spectrometer(packed, BITS, N_FFT, (s1 - s0) * N_FFT)
    return s1 - s0


class OraclePool:
    """The unchanged FP64 oracle on every host core: a spawn-started process pool (safe after
    CUDA is initialised), each worker given the integration's packed words once; a timed
    call splits `segs` segments into one contiguous chunk per worker."""

    def __init__(self, unique, workers: int | None = None):
        import multiprocessing as mp

        import oracle

        oracle.build()
        self.workers = max(1, workers or os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_init,
                                                 initargs=(unique[0].view(np.uint32),))
        # workers up and warm (bounded: a worker that cannot start must not hang the bench)
        self.pool.map_async(_oracle_chunk, [(0, 1)] * self.workers).get(timeout=600)

    def run(self, segs: int, repeats: int = 1):
        """(Msample/s, seconds) for `repeats` passes over `segs` segments of 4 IFs."""
        chunks = []
        for _ in range(repeats):
            bounds = [segs * w // self.workers for w in range(self.workers + 1)]
            chunks += [(bounds[w], bounds[w + 1]) for w in range(self.workers) if bounds[w + 1] > bounds[w]]
        t0 = time.perf_counter()
        done = sum(self.pool.map_async(_oracle_chunk, chunks).get(timeout=3600))
        dt = time.perf_counter() - t0
        return N_IF * done * N_FFT / dt / 1e6, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, rank):
    if rank != 0:
        return
    unique = make_unique_seconds(1)
    pool = OraclePool(unique)
    # size the per-step sample so that warmup + steps take about args.ref_seconds
    _, t1 = pool.run(pool.workers)
    budget = args.ref_seconds / max(1, args.steps + args.warmup)
    segs = int(max(pool.workers, min(SEGS, budget * pool.workers / max(t1, 1e-3))))
    for _ in range(args.warmup):
        pool.run(segs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pool.run(segs)
    dt = time.perf_counter() - t0
    pool.close()
    value = args.steps * N_IF * segs * N_FFT / dt / 1e6
    sample = (f"{segs} of the 61 segments of one integration per step (4 IF x {segs} x 131072 samples), "
              f"FP64 oracle on {pool.workers} processes")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Msample/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": CONFIG,
        "cpu_baseline": {"value": value, "unit": "Msample/s", "cores": pool.workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Msample/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def assign_streams(work, n_lanes):
    """Greedy longest-first schedule of independent jobs [(samples, n_fft)] onto n_lanes
    streams: each job (heaviest first) goes to the lane with the least work so far.  A job's
    work is its samples times a cost factor for transforms above 2^17 points, whose phase 1
    costs more per point (measured: about 1.4x, 1.75x, 2.1x at 2^18, 2^19, 2^20)."""
    def cost(n, n_fft):
        return n * {1 << 18: 1.4, 1 << 19: 1.75, 1 << 20: 2.1}.get(n_fft, 1.0)

    order = sorted(range(len(work)), key=lambda i: -cost(*work[i]))
    load = [0.0] * n_lanes
    lanes = [[] for _ in range(n_lanes)]
    for i in order:
        k = min(range(n_lanes), key=lambda j: load[j])
        lanes[k].append(i)
        load[k] += cost(*work[i])
    return lanes


def batch_graph_variant(torch, polaris, dev, local_rank, world, n_streams=64, seed=2024, caps=None, n_side=8):
    """Many independent 2-IF spectrometers at once (a mixed multi-stream workload): N
    log-uniform in 2^12..2^20, 2- or 8-bit, 0.1..2 s of 16-Msps data each (whole segments),
    every handle's feed + integrate captured into one CUDA graph and replayed; reports the
    aggregate input rate, and the same work issued eagerly for comparison."""
    rng = np.random.default_rng(seed)
    stream = torch.cuda.Stream(dev)
    items = []
    total = 0
    for _ in range(n_streams):
        logn = int(rng.integers(12, 21))
        bits = int(rng.choice([2, 8]))
        dur = float(np.exp(rng.uniform(np.log(0.1), np.log(2.0))))
        n_fft = 1 << logn
        nseg = max(1, int(round(dur * 16e6 / n_fft)))
        n = nseg * n_fft
        words = n * bits // 32
        dev_in = [torch.randint(-2**31, 2**31 - 1, (words,), dtype=torch.int32, device=dev) for _ in range(2)]
        nb = n_fft // 2 + 1
        outs = (torch.empty((2, nb), device=dev), torch.empty((1, nb, 2), device=dev),
                torch.empty((1, 4, nb), device=dev))
        sp = polaris.Spectrometer(2, bits, n_fft, device=local_rank, max_batch_segments=nseg)
        if caps:
            sp.set_launch_caps(*caps)
        items.append((sp, dev_in, n, outs))
        total += 2 * n

    # the handles spread over side streams so that small transforms run side by side: longest
    # first, each onto the side stream with the least work so far (work = samples, weighted by
    # the per-sample cost of large transforms); forked from and joined back into the issuing
    # stream
    side = [torch.cuda.Stream(dev) for _ in range(n_side)]
    lanes = assign_streams([(items[i][2], items[i][0].n_fft) for i in range(len(items))], len(side))

    def issue_all(cs):
        fork = torch.cuda.Event()
        fork.record(cs)
        joins = []
        for k, ss in enumerate(side):
            ss.wait_event(fork)
            for i in lanes[k]:
                sp, dev_in, n, outs = items[i]
                sp.feed(dev_in, n, on_device=True, stream=ss)
                sp.integrate_device(*outs, stream=ss)
            ev = torch.cuda.Event()
            ev.record(ss)
            joins.append(ev)
        for ev in joins:
            cs.wait_event(ev)

    with torch.cuda.stream(stream):
        issue_all(stream)  # per-kernel set-up outside the capture
    stream.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(reps):
            issue_all(stream)
        ev1.record(stream)
    stream.synchronize()
    eager_ms = ev0.elapsed_time(ev1) / reps
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        issue_all(torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(reps):
            g.replay()
        ev1.record(stream)
    stream.synchronize()
    graph_ms = ev0.elapsed_time(ev1) / reps
    # one more replay inside an NVTX range, for profilers (ncu --graph-profiling graph
    # --nvtx --nvtx-include "batchreplay/")
    torch.cuda.nvtx.range_push("batchreplay")
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = sum(sp.kernel_launches() for sp, *_ in items)
    for sp, *_ in items:
        sp.close()
    return {"streams": n_streams, "samples_per_pass": total, "graph_ms_per_pass": graph_ms,
            "ctas_per_sm_caps": list(caps) if caps else "library default",
            "eager_ms_per_pass": eager_ms, "value": world * total / (graph_ms * 1e-3) / 1e6,
            "eager_value": world * total / (eager_ms * 1e-3) / 1e6, "unit": "Msample/s",
            "note": "N log-uniform 2^12..2^20, 2/8-bit, 0.1..2 s at 16 Msps (whole segments), seed 2024"}


def adjoint_variant(torch, polaris, dev, local_rank, world, n_ring=20, seed=1256):
    """Differentiable leakage calibration: 2 circular-feed IFs (R, L), int8, 16384-point
    segments, 256 segments per pass; forward model + loss + adjoint (window, gain and
    leakage gradients) per pass.  A CUDA graph holds n_ring passes over n_ring distinct
    inputs (n_ring x 8.4 MB, larger than L2), so no pass finds its input in L2 and no
    host overhead is timed; the forward-only pass (model + loss) is timed the same way."""
    from paper_1412_1256_gb300 import synth

    packed, cfg = synth.config_circular(seed=seed)
    n_fft, n, bits = cfg["n_fft"], cfg["n_samples"], cfg["bits"]
    nseg = n // n_fft
    nb = n_fft // 2 + 1
    # one seeded input copied into n_ring distinct device buffers (distinct addresses: L2 cold)
    host = [torch.from_numpy(p.view(np.int32)) for p in packed]
    ring = [[h.to(dev) for h in host] for _ in range(n_ring)]
    rng = np.random.default_rng(seed)
    w = torch.from_numpy((0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n_fft) / n_fft)).astype(np.float32)).to(dev)
    mag, ph = rng.uniform(0.8, 1.2, 2), rng.uniform(-np.pi, np.pi, 2)
    gains = torch.tensor([mag[0] * np.cos(ph[0]), mag[0] * np.sin(ph[0]), mag[1] * np.cos(ph[1]),
                          mag[1] * np.sin(ph[1])], dtype=torch.float32, device=dev)
    leak = torch.from_numpy(rng.uniform(-0.035, 0.035, (2, nb, 2)).astype(np.float32)).to(dev)
    stream = torch.cuda.Stream(dev)
    out = {}
    with polaris.Adjoint(n_fft, bits, device=local_rank) as adj:
        with torch.cuda.stream(stream):
            target = (adj.run(ring[0], n, w, gains, leak, stream=stream)["stokes"] * 0.9).contiguous()
        stream.synchronize()
        for name, grads in (("forward_loss", False), ("forward_adjoint", True)):
            def issue(cs):
                return [adj.run(ring[i], n, w, gains, leak, target, grads=grads, stream=cs) for i in range(n_ring)]

            with torch.cuda.stream(stream):
                issue(stream)
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                keep = issue(torch.cuda.current_stream())
            for _ in range(3):
                graph.replay()
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            with torch.cuda.stream(stream):
                ev0.record(stream)
                for _ in range(reps):
                    graph.replay()
                ev1.record(stream)
            stream.synchronize()
            ms = ev0.elapsed_time(ev1) / (reps * n_ring)
            transforms = 3 if grads else 1  # the adjoint transforms every segment forward and back again
            flops = transforms * 5.0 * n_fft * math.log2(n_fft) * nseg
            out[name] = {"ms_per_pass": ms, "value": world * 2 * n / (ms * 1e-3) / 1e6, "unit": "Msample/s",
                         "transforms_per_segment": transforms, "gflop_per_pass": flops / 1e9,
                         "tflops": flops / (ms * 1e-3) / 1e12}
            assert all(torch.isfinite(k["loss"]).all() for k in keep)
            del graph, keep
    out["note"] = ("2 circular-feed IFs (R, L) int8, N = 16384, 256 segments, a line with q, u, v = 0.3, -0.2, "
                   "0.1 over unpolarised noise; |g| 0.8..1.2, |D| <= 0.05, Hann window; CUDA graph of 20 passes "
                   "over 20 distinct input buffers (168 MB > L2); flops = 5 N log2 N per complex transform of "
                   "a segment pair")
    return out


def tc_precision_variant(torch, polaris, dev, local_rank, world, n_unique=16, reps=3, seed=1256):
    """The precision workload: 2 IFs (X, Y), int8, 262144-point segments, 10 s at 16 Msps
    (610 segments), Hann window, a line 40 dB above the continuum with a 1e-3 derivative V
    profile.  The FP32 CUDA-core path and the tensor-core DFT path (fp16 x3, bf16 x3, bf16)
    integrate the same device-resident 10 s (n_unique distinct segments tiled over 320 MB,
    larger than L2); each is timed with CUDA events (feed + integrate).  Each tensor-core
    precision's spectra of the n_unique distinct segments are compared per bin with the FP32
    path's (the errors against the FP64 oracle come from tests/tc_precision_report.py)."""
    from paper_1412_1256_gb300 import synth

    packed, cfg = synth.config_precision(seed=seed, n_segments=n_unique)
    n_fft = cfg["n_fft"]
    nseg_total = 610
    n_total = nseg_total * n_fft
    words_u = n_unique * n_fft // 4
    ring = []
    for p in packed:
        u = torch.from_numpy(p.view(np.int32)).to(dev)
        big = torch.empty(n_total // 4, dtype=torch.int32, device=dev)
        for s0 in range(0, nseg_total, n_unique):
            c = min(n_unique, nseg_total - s0)
            big[s0 * n_fft // 4:(s0 + c) * n_fft // 4] = u[:c * n_fft // 4]
        ring.append(big)
    unique = [r[:words_u] for r in ring]
    n_u = n_unique * n_fft
    stream = torch.cuda.Stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nb = n_fft // 2 + 1

    def diffs(got, ref):
        # autos per bin relative; Stokes relative to I (floored at 5% of the channel mean)
        ra = np.abs(ref["autos"])
        da = np.abs(got["autos"] - ref["autos"]) / np.maximum(ra, 0.05 * ra.mean())
        I = np.abs(ref["stokes"][0])
        ds = np.abs(got["stokes"] - ref["stokes"]) / np.maximum(I, 0.05 * I.mean())[None, :]
        return {"max_autos_vs_fp32": float(da.max()), "median_autos_vs_fp32": float(np.median(da)),
                "max_stokes_vs_fp32": float(ds.max())}

    out = {}
    # FP32 CUDA-core path (the spectrometer), same window and data
    with polaris.Spectrometer(2, 8, n_fft, window="hann", device=local_rank) as sp:
        autos = torch.empty((2, nb), device=dev)
        cross = torch.empty((1, nb, 2), device=dev)
        stokes = torch.empty((1, 4, nb), device=dev)
        with torch.cuda.stream(stream):
            sp.feed(unique, n_u, on_device=True, stream=stream)
            sp.integrate_device(autos, cross, stokes, stream=stream)
            stream.synchronize()
            ref32 = {"autos": autos.cpu().numpy().astype(np.float64), "stokes": stokes.cpu().numpy()[0].astype(np.float64)}
            sp.feed(ring, n_total, on_device=True, stream=stream)
            sp.integrate_device(autos, cross, stokes, stream=stream)
            stream.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                sp.feed(ring, n_total, on_device=True, stream=stream)
                sp.integrate_device(autos, cross, stokes, stream=stream)
            ev1.record(stream)
            stream.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
    out["fp32"] = dict(ms_per_10s=ms, value=world * 2 * n_total / (ms * 1e-3) / 1e6)
    for prec in ("fp16x3", "bf16x3", "bf16"):
        with polaris.TensorCoreSpectrometer(8, n_fft, prec, "hann", device=local_rank) as tc:
            with torch.cuda.stream(stream):
                tc.feed(unique, n_u, stream=stream)
                g = tc.integrate(stream=stream)
                e = diffs({"autos": g["autos"], "stokes": g["stokes"]}, ref32)
                tc.feed(ring, n_total, stream=stream)
                tc.integrate(stream=stream)
                ev0.record(stream)
                for _ in range(reps):
                    tc.feed(ring, n_total, stream=stream)
                    tc.integrate(stream=stream)
                ev1.record(stream)
                stream.synchronize()
            ms = ev0.elapsed_time(ev1) / reps
        out[prec] = dict(e, ms_per_10s=ms, value=world * 2 * n_total / (ms * 1e-3) / 1e6,
                         speedup_vs_fp32=out["fp32"]["ms_per_10s"] / ms)
    out["unit"] = "Msample/s"
    out["note"] = ("2 IF int8, N = 2^18, 610 segments (10 s at 16 Msps), Hann, 40 dB line + 1e-3 dI/dnu V; "
                   "per-bin differences from the FP32 path over 16 distinct segments (autos per bin, Stokes by "
                   "I; denominators floored at 5% of the channel mean); time = feed + integrate of the 10 s "
                   "(320 MB device ring)")
    return out


def run_ours(args, rank, world, local_rank, dist):
    import torch

    from paper_1412_1256_gb300 import polaris

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    polaris.load()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    unique = make_unique_seconds(args.unique)
    ring_n = args.ring
    ring = torch.empty((ring_n, N_IF, WORDS_PER_IF), dtype=torch.int32, device=dev)
    for i in range(ring_n):
        ring[i].copy_(torch.from_numpy(unique[i % len(unique)]))
    autos = torch.empty((N_IF, NBIN), dtype=torch.float32, device=dev)
    cross = torch.empty((N_PAIR, NBIN, 2), dtype=torch.float32, device=dev)
    stokes = torch.empty((N_PAIR, 4, NBIN), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = polaris.Spectrometer(N_IF, BITS, N_FFT, device=local_rank, max_batch_segments=args.batch_segments)
    # the timed steps alternate over H handles, each with its own stream and outputs
    # (independent integrations); handle 0 also serves the per-kernel profiling pass
    H = max(1, args.handles)
    handles = [(sp, stream, (autos, cross, stokes))]
    for _ in range(H - 1):
        handles.append((polaris.Spectrometer(N_IF, BITS, N_FFT, device=local_rank,
                                             max_batch_segments=args.batch_segments),
                        torch.cuda.Stream(dev),
                        (torch.empty_like(autos), torch.empty_like(cross), torch.empty_like(stokes))))

    def step(i, h=None):
        sph, sth, outs = handles[i % H if h is None else h]
        sec = ring[i % ring_n]
        sph.feed([sec[j] for j in range(N_IF)], SAMPLES_PER_IF, on_device=True, stream=sth)
        return sph.integrate_device(*outs, stream=sth)

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.caps:
        c1, c2 = (int(x) for x in args.caps.split(","))
        for hd in handles:
            hd[0].set_launch_caps(c1, c2)
    for i in range(max(args.warmup, H)):
        assert step(i) == SEGS
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    next_step = [args.warmup]

    def timed_block():
        """One timed region of exactly args.steps steps, bracketed by a barrier and a device
        synchronisation on both sides; returns the slowest rank's milliseconds."""
        barrier()
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push("timed_region")  # (a profiler can replay one region whole)
        e0.record(stream)
        for _, sth, _ in handles[1:]:
            sth.wait_event(e0)  # fork
        for i in range(args.steps):
            step(next_step[0] + i)
        next_step[0] += args.steps
        for _, sth, _ in handles[1:]:
            ev = torch.cuda.Event()
            ev.record(sth)
            stream.wait_event(ev)  # join
        e1.record(stream)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        barrier()
        return slowest(dist, e0.elapsed_time(e1))

    # The K-step timed region is repeated R times (R >= --repeats, and enough for about
    # --min-timed-ms of timed work in total); value is taken at the median region, and
    # the spread of all R is reported beside it.
    l0 = sum(h[0].kernel_launches() for h in handles)
    with ClockSampler(local_rank) as clk:
        blocks = [timed_block()]
        reps = max(args.repeats, int(math.ceil(args.min_timed_ms / max(blocks[0], 1e-3))))
        reps = min(reps, max(args.repeats, 2000))
        while len(blocks) < reps:
            blocks.append(timed_block())
    launches = (sum(h[0].kernel_launches() for h in handles) - l0) / len(blocks)

    # live DRAM traffic and SM counters over the timed region's schedule (outside the timed
    # regions): the same steps on the same handles and streams, forked and joined as above
    live = None
    if not args.no_live_counters:
        def region():
            e0.record(stream)
            for _, sth, _ in handles[1:]:
                sth.wait_event(e0)
            for i in range(args.steps):
                step(next_step[0] + i)
            next_step[0] += args.steps
            for _, sth, _ in handles[1:]:
                ev = torch.cuda.Event()
                ev.record(sth)
                stream.wait_event(ev)
        live = live_dram(torch, dev, local_rank, region, float(statistics.median(blocks)), args.steps,
                         "integration")
        if "dram_bytes_per_integration" in live:
            # one pass over the packed input and one write of the spectra
            alg = 4 * N_IF * WORDS_PER_IF + 4 * (autos.numel() + cross.numel() + stokes.numel())
            live["algorithmic_bytes_per_integration"] = alg
            live["traffic_over_algorithmic"] = live["dram_bytes_per_integration"] / alg
    for hd in handles[1:]:
        hd[0].close()
    t_max = float(statistics.median(blocks))
    t_ms = t_max
    value = whole_job_rate(world, args.steps, SAMPLES_PER_STEP, t_max * 1e-3)
    qs = np.percentile(np.array(blocks) / args.steps, [0, 10, 25, 50, 75, 90, 100])
    spread = {"repeats": len(blocks), "min_ms_per_step": qs[0], "p10_ms_per_step": qs[1], "p25_ms_per_step": qs[2],
              "median_ms_per_step": qs[3], "p75_ms_per_step": qs[4], "p90_ms_per_step": qs[5],
              "max_ms_per_step": qs[6], "rel_iqr": (qs[4] - qs[2]) / qs[3],
              "timed_ms_total": float(sum(blocks)),
              "note": f"{len(blocks)} timed regions of {args.steps} steps each; value and ms_per_step are "
                      f"the median region's"}

    # per-kernel device time: a second timed pass with every launch bracketed by events, one
    # handle on one stream, each kernel alone at its default occupancy (the CTA caps are a
    # policy for integrations in flight side by side)
    if args.caps:
        sp.set_launch_caps(0, 0)
    sp.set_profiling(True)
    prof_steps = max(3, min(args.steps, 50))
    for i in range(prof_steps):
        step(i, 0)
    torch.cuda.synchronize(dev)
    kt = sp.kernel_times()
    sp.set_profiling(False)
    if args.caps:
        sp.set_launch_caps(*(int(x) for x in args.caps.split(",")))

    # e2e through the C ABI with pinned host buffers: every step copies its input from
    # pinned host memory (feed with host pointers, asynchronous mode: the copy is queued and
    # the call returns; the pinned buffers stay unchanged) and reads its spectra back into
    # pinned host memory (integrate_async: readout and copies queued in one call).  L
    # spectrometer handles on L streams take steps in turn, so that copies and kernels of
    # consecutive integrations overlap (a streaming caller's pattern); the host waits for
    # step i's outputs after queueing step i + L - 1.
    e2e_value, e2e_spread = None, None
    if not args.no_e2e:
        n_host = min(len(unique), 4)
        pinned = [torch.from_numpy(unique[i]).pin_memory() for i in range(n_host)]
        host = [p.numpy().view(np.uint32) for p in pinned]
        lanes = []
        L = max(2, args.e2e_handles)
        for k in range(L):
            spk = sp if k == 0 else polaris.Spectrometer(N_IF, BITS, N_FFT, device=local_rank,
                                                         max_batch_segments=args.batch_segments)
            if args.caps:
                spk.set_launch_caps(*(int(x) for x in args.caps.split(",")))
            stk = torch.cuda.Stream(dev)
            dev_out = (torch.empty((N_IF, NBIN), dtype=torch.float32, device=dev),
                       torch.empty((N_PAIR, NBIN, 2), dtype=torch.float32, device=dev),
                       torch.empty((N_PAIR, 4, NBIN), dtype=torch.float32, device=dev))
            host_out = tuple(torch.empty(t.shape, dtype=torch.float32, pin_memory=True) for t in dev_out)
            lanes.append((spk, stk, dev_out, host_out, torch.cuda.Event()))

        def e2e_issue(i):
            spk, stk, dev_out, host_out, done = lanes[i % L]
            spk.feed([host[i % n_host][j] for j in range(N_IF)], SAMPLES_PER_IF, on_device=False, stream=stk,
                     host_async=True)
            nseg = spk.integrate_async(dict(zip(("autos", "cross", "stokes"), host_out)), stream=stk)
            done.record(stk)
            return nseg

        def e2e_wait(i):
            lanes[i % L][4].synchronize()

        for i in range(2 * L):
            assert e2e_issue(i) == SEGS
            e2e_wait(i)
        e2e_steps = max(3, min(args.steps, args.e2e_steps))

        def e2e_block(base):
            """One end-to-end timed region of e2e_steps steps (host clock, synchronised on both
            sides); returns the slowest rank's seconds."""
            torch.cuda.synchronize(dev)
            barrier()
            t0 = time.perf_counter()
            for i in range(min(L - 1, e2e_steps)):
                assert e2e_issue(base + i) == SEGS
            for i in range(e2e_steps):
                if i + L - 1 < e2e_steps:
                    assert e2e_issue(base + i + L - 1) == SEGS
                e2e_wait(base + i)  # step i's spectra are in host memory
            torch.cuda.synchronize(dev)
            return slowest(dist, time.perf_counter() - t0)

        # repeated like the device-resident region; the median region gives the value
        e2e_blocks = [e2e_block(0)]
        e2e_reps = max(args.repeats, int(math.ceil(args.min_timed_ms * 1e-3 / max(e2e_blocks[0], 1e-6))))
        e2e_reps = min(e2e_reps, max(args.repeats, 2000))
        while len(e2e_blocks) < e2e_reps:
            e2e_blocks.append(e2e_block(len(e2e_blocks) * e2e_steps))
        dt = float(statistics.median(e2e_blocks))
        e2e_value = whole_job_rate(world, e2e_steps, SAMPLES_PER_STEP, dt)
        e2e_spread = {"repeats": len(e2e_blocks), "steps_per_region": e2e_steps,
                      "min_ms_per_step": min(e2e_blocks) * 1e3 / e2e_steps,
                      "max_ms_per_step": max(e2e_blocks) * 1e3 / e2e_steps}
        for ln in lanes[1:]:
            ln[0].close()

    # variants of the same workload (NEXT-4): 50% overlap (hop = N/2, Sec. 3.1) and the
    # code-histogram statistics (Sec. 2 bit distribution), each through the same API
    variants = None
    if not args.no_variants:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(make, nsteps):
            """nsteps steps alternating over H handles made by make(), as in the main timing;
            returns (ms per step, segments of the last step, the handles, warm-up steps)."""
            hs = [(make(), stream if k == 0 else torch.cuda.Stream(dev),
                   (autos, cross, stokes) if k == 0 else
                   (torch.empty_like(autos), torch.empty_like(cross), torch.empty_like(stokes))) for k in range(H)]
            if args.caps:
                for hd in hs:
                    hd[0].set_launch_caps(*(int(x) for x in args.caps.split(",")))

            def stepv(i):
                spv, st, outs = hs[i % H]
                sec = ring[i % ring_n]
                spv.feed([sec[j] for j in range(N_IF)], SAMPLES_PER_IF, on_device=True, stream=st)
                return spv.integrate_device(*outs, stream=st)

            warm = max(3, H)
            for i in range(warm):
                stepv(i)
            torch.cuda.synchronize(dev)
            segs = 0
            ev0.record(stream)
            for _, st, _ in hs[1:]:
                st.wait_event(ev0)
            for i in range(nsteps):
                segs = stepv(warm + i)
            for _, st, _ in hs[1:]:
                evj = torch.cuda.Event()
                evj.record(st)
                stream.wait_event(evj)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            return ev0.elapsed_time(ev1) / nsteps, segs, hs, warm

        nv = max(10, min(args.steps, 100))
        variants = {}
        ms, segs, hs, _ = timed(lambda: polaris.Spectrometer(N_IF, BITS, N_FFT, hop=N_FFT // 2, device=local_rank), nv)
        for hd in hs:
            hd[0].close()
        variants["overlap_50"] = {"hop": N_FFT // 2, "segments_per_step": segs, "ms_per_step": ms,
                                  "value": world * SAMPLES_PER_STEP / (ms * 1e-3) / 1e6, "unit": "Msample/s",
                                  "steps": nv, "handles": H}
        ms, segs, hs, warm = timed(lambda: polaris.Spectrometer(N_IF, BITS, N_FFT, device=local_rank, code_stats=True),
                                   nv)
        sps = hs[0][0]
        sps.set_profiling(True)
        for i in range(10):
            sps.feed([ring[i % ring_n][j] for j in range(N_IF)], SAMPLES_PER_IF, on_device=True, stream=stream)
            sps.integrate_device(autos, cross, stokes, stream=stream)
        torch.cuda.synchronize(dev)
        kh = sps.kernel_times()["code_histogram"]
        sps.set_profiling(False)
        counted = sum(int(hd[0].code_histogram().sum()) for hd in hs)
        assert counted == N_IF * N_FFT * SEGS * (warm + nv + 10)
        for hd in hs:
            hd[0].close()
        variants["code_stats"] = {"ms_per_step": ms, "value": world * SAMPLES_PER_STEP / (ms * 1e-3) / 1e6,
                                  "unit": "Msample/s", "steps": nv, "handles": H,
                                  "histogram_kernel_ms": kh[0] / kh[1] if kh[1] else None}
        caps = tuple(int(x) for x in args.caps.split(",")) if args.caps else None
        variants["batch_graph"] = batch_graph_variant(torch, polaris, dev, local_rank, world, caps=caps)
        variants["adjoint"] = adjoint_variant(torch, polaris, dev, local_rank, world)
        variants["tc_precision"] = tc_precision_variant(torch, polaris, dev, local_rank, world)

    sp.close()
    if rank != 0:
        return

    flops = algorithmic_flops()
    clocks = clk.summary()
    peak_mhz = float(clocks["sm_max_mhz"] or 2070.0)
    peak = fp32_peak_tflops(num_sms, peak_mhz)
    kernels = {}
    total_kt = sum(v[0] for v in kt.values()) or 1.0
    for k, (ms, n) in kt.items():
        if n and k in flops:
            per_step = flops[k]  # flops per step for this kernel
            launches_per_step = n / prof_steps
            kernels[k] = {"avg_ms": ms / n, "launches": n, "share": ms / total_kt,
                          "tflops": (per_step * prof_steps / (ms * 1e-3) / 1e12) if ms > 0 and per_step else 0.0,
                          "launches_per_step": launches_per_step}
    dom = max(kernels, key=lambda k: kernels[k]["avg_ms"] * kernels[k]["launches"])
    ach = kernels[dom]["tflops"]
    traffic = recorded_traffic(dom)
    if traffic is not None:
        # bytes per launch: per-segment-pair figure x pair-segments per launch
        traffic = traffic * (N_PAIR * SEGS) / kernels[dom]["launches_per_step"]
    path_tflops = flops["path"] * args.steps / (t_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Msample/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: seeded 4-IF 2-bit streams, Gaussian noise + three Gaussian lines (FWHM 20 ch, 5x "
                "continuum; unpolarised, linear, circular)",
        "config": CONFIG,
        "roofline": {
            "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic, "kernel": dom,
            "peak_source": f"derived: {num_sms} SMs x 128 FP32 lanes x 2 flop x {peak_mhz:.0f} MHz (max SM clock)",
            "peak_at_measured_clock": fp32_peak_tflops(num_sms, float(clocks["sm_mhz"] or peak_mhz)),
            "measured_sm_mhz": clocks["sm_mhz"],
        },
        "path_roofline": {
            "achieved": path_tflops, "peak": peak, "unit": "TFLOP/s", "frac": path_tflops / peak,
            "roofline_msample_s": peak * 1e12 / (flops["path"] / SAMPLES_PER_STEP) / 1e6,
            "note": "whole step (all kernels, launch gaps included) against the FP32 roofline",
        },
        "kernels": kernels,
        "e2e": {"value": e2e_value, "unit": "Msample/s", "h2d_bytes_per_step": H2D_BYTES,
                "d2h_bytes_per_step": D2H_BYTES, "spread": e2e_spread},
        "gpu_launches": int(round(launches)),
        "gpu_launches_note": "kernels of ours launched per timed region of `steps` steps (the mean over the repeats)",
        "repeats": spread["repeats"],
        "spread": spread,
        "clocks": clocks,
        "live_counters": live,
        "pipeline": {"handles": H, "e2e_handles": None if args.no_e2e else max(2, args.e2e_handles),
                     "ctas_per_sm_caps": args.caps or "library default",
                     "note": "consecutive steps (independent 1-s integrations) alternate over this many "
                             "spectrometer handles, each on its own stream, with the CTA-per-SM caps above; "
                             "per-kernel times come from a separate pass of one handle on one stream, each "
                             "kernel alone at its default occupancy"},
    }
    if variants is not None:
        for v in ("forward_loss", "forward_adjoint"):
            variants["adjoint"][v]["frac_of_fp32_peak"] = variants["adjoint"][v]["tflops"] / peak
        line["variants"] = variants
    if world == 1 and not args.no_cpu_baseline:
        # the oracle on every host core (about 10-30 s of CPU work), and on one core beside it
        pool = OraclePool(unique)
        v, dt = pool.run(args.cpu_segs, args.cpu_repeats)
        pool.close()
        v1, dt1 = time_oracle(unique, args.cpu_segs, 1)
        line["cpu_baseline"] = {"value": v, "unit": "Msample/s", "cores": pool.workers, "kind": "oracle",
                                "sample": f"{args.cpu_repeats} x {args.cpu_segs} segments of one "
                                          f"integration (4 IF x 131072-sample segments), FP64 oracle on "
                                          f"{pool.workers} processes, {dt:.1f} s wall; one core: {v1:.1f} Msample/s "
                                          f"({dt1:.1f} s for {args.cpu_segs} segments)",
                                "value_one_core": v1}
    print(json.dumps(line), flush=True)


def run_variant(name, local_rank, caps=""):
    """One variant alone (not the benchmark line): its JSON on one line."""
    import torch

    from paper_1412_1256_gb300 import polaris

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    polaris.load()
    fn = {"batch_graph": batch_graph_variant, "tc_precision": tc_precision_variant, "adjoint": adjoint_variant}[name]
    kw = {"caps": tuple(int(x) for x in caps.split(","))} if (name == "batch_graph" and caps) else {}
    print(json.dumps({"variant": name, **fn(torch, polaris, dev, local_rank, 1, **kw)}), flush=True)


def run_sweep(args, local_rank):
    """Throughput against N (--sweep LOGN,...): 4 IFs of --sweep-bits-bit samples, rectangular
    window, about 8 M samples per IF per step (whole segments), one handle on one stream,
    the library's default batch, input cycling over 8 device buffers (which fit in L2);
    prints one JSON line {"sweep": {log2 N: Msample/s}, ...}.  Not the benchmark line."""
    import torch

    from paper_1412_1256_gb300 import polaris

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    polaris.load()
    bits, n_if, reps = args.sweep_bits, 4, args.sweep_reps
    out = {}
    gen = torch.Generator(device=dev)
    gen.manual_seed(1256)
    for logn in [int(x) for x in args.sweep.split(",") if x]:
        n_fft = 1 << logn
        n = max(1, (8 << 20) // n_fft) * n_fft
        ring = [[torch.randint(-2**31, 2**31 - 1, (n * bits // 32,), dtype=torch.int32, device=dev, generator=gen)
                 for _ in range(n_if)] for _ in range(8)]
        nb = n_fft // 2 + 1
        outs = (torch.empty((n_if, nb), device=dev), torch.empty((n_if // 2, nb, 2), device=dev),
                torch.empty((n_if // 2, 4, nb), device=dev))
        st = torch.cuda.Stream(dev)
        with polaris.Spectrometer(n_if, bits, n_fft, device=local_rank) as sp:
            for i in range(3):
                sp.feed(ring[i % 8], n, on_device=True, stream=st)
                sp.integrate_device(*outs, stream=st)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for i in range(reps):
                sp.feed(ring[i % 8], n, on_device=True, stream=st)
                sp.integrate_device(*outs, stream=st)
            e1.record(st)
            st.synchronize()
        out[logn] = n_if * n * reps / (e0.elapsed_time(e1) * 1e-3) / 1e6
        del ring
    print(json.dumps({"sweep": out, "unit": "Msample/s", "bits": bits, "n_if": n_if, "reps": reps}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ring", type=int, default=60, help="distinct seconds of input kept on the device")
    ap.add_argument("--unique", type=int, default=2, help="distinct generated seconds (tiled over the ring)")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--handles", type=int, default=DEFAULT_HANDLES,
                    help="spectrometer handles (and streams) the timed steps alternate over")
    ap.add_argument("--e2e-handles", type=int, default=DEFAULT_E2E_HANDLES,
                    help="handles (and streams) of the end-to-end loop")
    ap.add_argument("--repeats", type=int, default=25,
                    help="timed regions of --steps steps each (at least; see --min-timed-ms); the median is reported")
    ap.add_argument("--min-timed-ms", type=float, default=60.0,
                    help="repeat the timed region until about this much timed work in total")
    ap.add_argument("--cpu-segs", type=int, default=61)
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="reference arm: about this many seconds of oracle work over warmup + steps")
    ap.add_argument("--cpu-repeats", type=int, default=8,
                    help="CPU baseline: passes over --cpu-segs segments, split over the host cores")
    ap.add_argument("--caps", default=DEFAULT_CAPS,
                    help="P1,P2: CTAs per SM of the two FFT kernels at most, for every handle of the timed and "
                         "end-to-end loops (0: as many as fit; empty: the library's choice)")
    ap.add_argument("--batch-segments", type=int, default=0,
                    help="segments per kernel pass (0: the library's default, at least 64 segments per pass)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-live-counters", action="store_true",
                    help="skip the NVML GPM pass (live DRAM bytes per integration, SM counters)")
    ap.add_argument("--no-variants", action="store_true", help="skip the overlap / code-statistics variants")
    ap.add_argument("--sweep", default="", help="comma-separated log2 N: print the throughput against N instead")
    ap.add_argument("--only", choices=["batch_graph", "tc_precision", "adjoint"], default=None,
                    help="run one variant of the workload alone and print its JSON (for profiling)")
    ap.add_argument("--sweep-bits", type=int, default=2)
    ap.add_argument("--sweep-reps", type=int, default=20)
    args = ap.parse_args()
    if args.sweep:
        run_sweep(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.only:
        run_variant(args.only, int(os.environ.get("LOCAL_RANK", "0")), args.caps)
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist_mod.init_process_group("gloo", rank=rank, world_size=world)
        dist = dist_mod
    try:
        if args.impl == "reference":
            run_reference(args, rank)
        else:
            run_ours(args, rank, world, local_rank, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
