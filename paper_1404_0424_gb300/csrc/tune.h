// The autotuner's schedule cache (tune.cu), host side.
#pragma once

#include <cstdint>
#include <string>

namespace cgm {

// A plan schedule as the autotuner records it (the fields of cg_schedule).
struct TuneEntry {
  int32_t precision;   // CG_PREC_*
  int32_t order;       // 0: work units in descriptor order, 1: longest first
  int32_t concurrent;  // 1: bins side by side on forked streams, 0: one after another
  int32_t grid_pct;    // grid of each bin, percent of its resident CTAs
  float ms;            // one run of the plan when it was timed
};

// Entry of `key` (device name and plan shape class); false if none.
bool tune_lookup(const std::string& key, TuneEntry* out);
// Records an entry (and rewrites the file named by CGMIMO_TUNE_CACHE, if any).
void tune_store(const std::string& key, const TuneEntry& e);

}  // namespace cgm
