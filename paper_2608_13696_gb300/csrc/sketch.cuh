// Sample sketch of a group-by input: parameters shared between the kernel
// (sketch.cu) and the C-ABI layer (api.cu).
#pragma once

#include "rel_internal.cuh"

namespace rel {

constexpr int SKETCH_SAMPLE = 4096;
constexpr int SKETCH_TOP = REL_SKETCH_TOP;

struct SketchParams {
  int64_t n_rows;
  const uint8_t* col[REL_MAX_COLS];
  int32_t ctype[REL_MAX_COLS];
  int32_t n_keys, n_preds;
  int32_t key_col[REL_MAX_KEYS];
  int32_t key_shift[REL_MAX_KEYS];
  uint64_t key_mask[REL_MAX_KEYS];
  int32_t pred_col[REL_MAX_PREDS];
  int64_t pred_lo[REL_MAX_PREDS], pred_hi[REL_MAX_PREDS];
};

// What the kernel writes (device memory, read back by the host).
struct DevSketch {
  int32_t sample_rows, kept, ndv, singletons, runs, pad;
  int64_t key_min, key_max;
  int64_t top_key[SKETCH_TOP];
  int32_t top_count[SKETCH_TOP];
  uint8_t hll[256];
};

rel_status sketch_launch(const SketchParams& p, DevSketch* out, cudaStream_t st);
// ps and outs: n entries in device memory.
rel_status sketch_many_launch(const SketchParams* ps, DevSketch* outs, int n, cudaStream_t st);

}  // namespace rel
