// Launch-configuration autotuner (tune.cpp).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>

namespace rte {

// Times the candidates 0 .. ncand-1 of one kernel on stream s (run(i)
// launches candidate i; one warm-up launch each, then three rounds of reps
// launches between CUDA events, the best round counting) and stores the
// fastest in *best, keeping the default candidate def unless another is at
// least 3 % faster.  The choice is cached per key for the process, so later
// handles with the same shapes reuse it without timing.  run's return code is
// checked; a failing candidate is skipped.
int autotune(cudaStream_t s, const std::string& key, int ncand,
             const std::function<int(int)>& run, int* best, int def, int reps = 5);

// "key=choice (ms per candidate ...);" for every tuned key, for reports.
std::string autotune_report();

}  // namespace rte
