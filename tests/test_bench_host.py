"""Host-side logic of bench.py that needs no GPU: the stream assignment of the mixed batch,
the nominal flop split behind the roofline fractions, the FP32 peak, the traffic records'
source digests, and the live-counter pass degrading to an `unavailable` record where
NVML's performance counters cannot be read."""
import itertools

import pytest

import bench


def test_assign_streams_covers_every_job_once_and_balances():
    work = [(n, 1 << k) for n, k in zip([5, 40, 7, 13, 21, 3, 8, 34, 2, 1], [12, 20, 14, 17, 18, 13, 19, 16, 15, 12])]
    for lanes in (1, 2, 3, 8):
        out = bench.assign_streams(work, lanes)
        assert len(out) == lanes
        flat = sorted(itertools.chain.from_iterable(out))
        assert flat == list(range(len(work)))  # every job exactly once

        def cost(i):
            n, n_fft = work[i]
            return n * {1 << 18: 1.4, 1 << 19: 1.75, 1 << 20: 2.1}.get(n_fft, 1.0)

        loads = [sum(cost(i) for i in lane) for lane in out]
        # greedy longest-first: no lane exceeds the least loaded one by more than the largest job
        assert max(loads) - min(loads) <= max(cost(i) for i in range(len(work))) + 1e-9


def test_flop_split_and_peak():
    f = bench.algorithmic_flops()
    segs = bench.N_IF * bench.SEGS
    stage = segs * 5.0 * bench.N_FFT / 2.0
    # phase 1 holds 8 of the 17 radix-2 stages plus the window, phase 2 the other 9 plus the
    # correlation of every bin of every segment-time (32 flop)
    assert f["phase1_decode_rowdft"] == pytest.approx(8 * stage + bench.SAMPLES_PER_STEP)
    assert f["phase2_coldft_correlate"] == pytest.approx(9 * stage + bench.SEGS * bench.NBIN * 32.0)
    assert f["path"] == pytest.approx(f["phase1_decode_rowdft"] + f["phase2_coldft_correlate"] + f.get("readout_stokes", 0.0))
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784)


def test_traffic_records_match_the_kernel_sources():
    # the committed records were taken on the committed kernels: bench.py reports them
    for kernel in ("phase1_decode_rowdft", "phase2_coldft_correlate"):
        t = bench.recorded_traffic(kernel)
        assert t is not None and 1e5 < t < 2e6, kernel  # bytes per pair-segment


def test_live_counters_unavailable_without_gpm(monkeypatch):
    import ctypes

    def no_nvml(*a, **k):
        raise OSError("libnvidia-ml.so.1: not present")

    monkeypatch.setattr(ctypes, "CDLL", no_nvml)
    lc = bench.LiveCounters(0)
    assert not lc.ok and "unavailable" in lc.why
    out = bench.live_dram(None, None, 0, lambda: None, 1.0, 1, "integration")
    assert set(out) == {"unavailable"}
