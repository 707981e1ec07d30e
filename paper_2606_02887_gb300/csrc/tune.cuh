// Launch configuration of the A*X product kernels chosen by the autotuner (tune.cu), and
// its JSON cache keyed by device.
#pragma once

#include <string>

namespace snmf {

// Zero fields keep the built-in heuristic of the kernel's launcher.
struct ProdTune {
  int splits = 0;   // split-K slices
  int stages = 0;   // tcgen05 product: shared-memory ring stages
  int per_sm = 0;   // tcgen05 product: CTAs planned per SM (sets the default split count)
  int bn = 0;       // tcgen05 product: output columns per CTA tile (multiple of 16, <= 256)
  int row_bm = 0;   // row kernels of a step (FP32): rows per CTA
  int row_tc = 0;   // 1: the step's row products on the tensor cores (rowtc.cu, r = 64)
};

struct TuneEntry {
  ProdTune cfg;
  double ms = 0.0;  // measured mean time of one product (CUDA events)
};

// "<device name>/<SM count>" of the current device ("" when it cannot be queried).
std::string tune_device_key();
// Cache lookup / store in the JSON file at `path` (NULL or empty: an in-process cache
// only).  The file maps device keys to shape keys ("dense/<dtype>/n<n>/N<N>") to entries.
bool tune_lookup(const char* path, const std::string& dev, const std::string& key, TuneEntry* out);
bool tune_store(const char* path, const std::string& dev, const std::string& key, const TuneEntry& e);

}  // namespace snmf
