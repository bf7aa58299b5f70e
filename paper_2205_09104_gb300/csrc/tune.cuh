// Launch autotuner: for a kernel family and a problem shape (the key), time every candidate
// launch configuration once on the caller's stream with CUDA events and keep the fastest.
// Decisions live in a process-wide table keyed by the shape and the GPU model (compute
// capability and SM count), so devices of different models never share one; a decision read
// from the cache file without a model suffix applies to every device.  If the environment
// variable COARSE_AUTOTUNE_CACHE
// names a file, decisions are read from it at first use and every new decision is appended to
// it, so later processes skip the timing.  A stream that is being captured into a CUDA graph
// cannot be timed: there the first candidate (the static default) is used and nothing is recorded.
#pragma once

#include <functional>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace coarse {

struct TuneChoice {
  int a = 0, b = 0, c = 0;  // meaning defined by the kernel family
};

// Picks the configuration for `key` among `cands` (cands[0] = default).  `run(choice)` must
// launch the kernel once with that configuration on `s` and return COARSE_OK; the launches
// must be idempotent (same output however often they run).  Synchronises `s` when it times.
int tune_pick(const std::string& key, const std::vector<TuneChoice>& cands,
              const std::function<int(const TuneChoice&)>& run, cudaStream_t s, TuneChoice* out);

// Bucket of a size for tuning keys: floor(log2(v)).
int tune_bucket(long long v);

// Decisions of the hot launch paths, per device ordinal, for lock-free reads on every launch:
// family (0 = single-RHS stencil, 1 = odd-even half apply), block precision, n / 16 - 1, size
// bucket -> candidate, or -1 while undecided.  tune_pick remains the source of the decisions;
// coarse_autotune_set clears these entries so that the next launch looks its key up again.
int tune_fast_get(int family, int prec, int ni, int vb);
void tune_fast_put(int family, int prec, int ni, int vb, int choice);

}  // namespace coarse
