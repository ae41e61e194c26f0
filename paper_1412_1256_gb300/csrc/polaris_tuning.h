// Launch choices per transform size and sample width, written by paper_1412_1256_gb300/tune.py
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
    {0, 0, 0, 0, 0},  // (no entry: the built-in choices won everywhere)
};
}  // namespace polaris
