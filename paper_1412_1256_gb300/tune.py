"""Offline launch tuner for the spectrometer's FFT kernels.

For each transform size and sample width it times feed + integrate of 4 IF streams (about
8 M samples per IF per step, rectangular window, one handle on one stream, device-resident
input) over candidate launch choices:

  * segments per kernel pass (max_batch_segments): the built-in rule and 64 .. 4096;
  * CTAs per SM of phase 1 and of phase 2 at most: as many as fit (0) or one.

The tile width of phase 1 and the points per lane are compile-time choices of the kernels
(one instantiation per size and width) and are not tuned here.  The fastest choice per
(log2 N, bits) becomes an entry of ``csrc/polaris_tuning.h`` only when it beats the built-in
choice by more than ``--min-gain`` (timing noise otherwise decides); every measurement is
written to ``tuning.json`` beside this file.  Run on the GPU the table is for, then rebuild:

    python -m paper_1412_1256_gb300.tune [--sizes 10,...,20] [--bits 2,8] [--reps 10]
"""
from __future__ import annotations

import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "csrc", "polaris_tuning.h")
RECORD = os.path.join(HERE, "tuning.json")

HEADER_TOP = """// Launch choices per transform size and sample width, written by paper_1412_1256_gb300/tune.py
// from timings on a GB300 (feed + integrate of 4 IF streams, one handle on one stream).  An
// entry replaces the built-in choice when a spectrometer is created with max_batch_segments = 0:
// max_batch = segments per kernel pass (0: the built-in rule), cap1 / cap2 = CTAs per SM of
// phase 1 / phase 2 at most (0: as many as fit).  Sizes and widths without an entry keep the
// built-in choices.
#pragma once

namespace polaris {
struct TuneEntry {
  int logn, bits, max_batch, cap1, cap2;
};
static const TuneEntry kTuned[] = {
"""
HEADER_END = """};
}  // namespace polaris
"""


def render_header(entries) -> str:
    """The table as C++: entries = [(logn, bits, max_batch, cap1, cap2)]."""
    lines = [f"    {{{l}, {b}, {m}, {c1}, {c2}}}," for (l, b, m, c1, c2) in sorted(entries)]
    if not lines:
        lines = ["    {0, 0, 0, 0, 0},  // (no entry: the built-in choices won everywhere)"]
    return HEADER_TOP + "\n".join(lines) + "\n" + HEADER_END


def parse_header(text: str):
    """Entries of a table written by render_header (the placeholder row is skipped)."""
    import re

    out = []
    for m in re.finditer(r"\{\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+),\s*(\d+)\s*\}", text):
        e = tuple(int(x) for x in m.groups())
        if e[0] > 0:
            out.append(e)
    return out


def candidates(nseg_step: int):
    """(max_batch_segments, cap1, cap2); max_batch 0 = the built-in rule."""
    batches = [0] + [b for b in (64, 256, 1024, 4096) if b < nseg_step]
    out = []
    for b in batches:
        for c1 in (0, 1):
            for c2 in (0, 1):
                out.append((b, c1, c2))
    return out


def time_choice(torch, polaris, ring, bits, n_fft, n, choice, reps):
    b, c1, c2 = choice
    dev = ring[0][0].device
    nb = n_fft // 2 + 1
    outs = (torch.empty((4, nb), device=dev), torch.empty((2, nb, 2), device=dev),
            torch.empty((2, 4, nb), device=dev))
    st = torch.cuda.current_stream(dev)
    with polaris.Spectrometer(4, bits, n_fft, max_batch_segments=b) as sp:
        sp.set_launch_caps(c1, c2)
        for i in range(2):
            sp.feed(ring[i % len(ring)], n, on_device=True, stream=st)
            sp.integrate_device(*outs, stream=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(reps):
            sp.feed(ring[i % len(ring)], n, on_device=True, stream=st)
            sp.integrate_device(*outs, stream=st)
        e1.record(st)
        torch.cuda.synchronize(dev)
    return 4 * n * reps / (e0.elapsed_time(e1) * 1e-3) / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="10,11,12,13,14,15,16,17,18,19,20")
    ap.add_argument("--bits", default="2,8")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--min-gain", type=float, default=0.03, help="relative gain needed to leave the built-in choice")
    ap.add_argument("--dry-run", action="store_true", help="measure and print; write nothing")
    args = ap.parse_args()

    import torch

    from paper_1412_1256_gb300 import polaris

    polaris.load()
    dev = torch.device("cuda", 0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1256)
    record = {"gpu": torch.cuda.get_device_name(dev), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
              "workload": "4 IF streams, rect window, ~8 M samples per IF per step, one handle on one stream",
              "unit": "Msample/s", "min_gain": args.min_gain, "results": {}}
    entries = []
    for bits in [int(x) for x in args.bits.split(",")]:
        for logn in [int(x) for x in args.sizes.split(",")]:
            n_fft = 1 << logn
            nseg = max(1, (8 << 20) // n_fft)
            n = nseg * n_fft
            ring = [[torch.randint(-2**31, 2**31 - 1, (n * bits // 32,), dtype=torch.int32, device=dev,
                                   generator=gen) for _ in range(4)] for _ in range(4)]
            rates = {}
            for ch in candidates(nseg):
                rates[ch] = time_choice(torch, polaris, ring, bits, n_fft, n, ch, args.reps)
            base = rates[(0, 0, 0)]
            best = max(rates, key=rates.get)
            chosen = best if rates[best] > base * (1 + args.min_gain) else (0, 0, 0)
            if chosen != (0, 0, 0):
                entries.append((logn, bits) + chosen)
            record["results"][f"{logn},{bits}"] = {
                "segments_per_step": nseg, "builtin": base, "best": list(best), "best_rate": rates[best],
                "chosen": list(chosen), "all": {f"{b},{c1},{c2}": r for (b, c1, c2), r in rates.items()}}
            print(f"2^{logn} {bits}-bit: built-in {base:.0f}, best {best} {rates[best]:.0f}, chosen {chosen}",
                  flush=True)
            del ring
    if not args.dry_run:
        with open(HEADER, "w") as f:
            f.write(render_header(entries))
        with open(RECORD, "w") as f:
            json.dump(record, f, indent=1)
        print(f"wrote {HEADER} ({len(entries)} entries) and {RECORD}; rebuild the library to use them")


if __name__ == "__main__":
    main()
