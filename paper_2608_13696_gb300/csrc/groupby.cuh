// Group-by launch parameters shared between the kernels (groupby.cu) and the
// C-ABI layer (api.cu).
#pragma once

#include "rel_internal.cuh"

namespace rel {

constexpr int GB_BLOCK = 256;
constexpr int GB_STAGES = 3;
constexpr int TINY_SLOTS = 8;
constexpr int SHARED_PROBES = 16;

enum GbMode : int { MODE_GLOBAL = 0, MODE_TINY = 1, MODE_SHARED = 2, MODE_KEYSET = 3 };
enum GbShape : int { SHAPE_GENERIC = 0, SHAPE_Q1 = 1, SHAPE_KV64 = 2, SHAPE_KV32 = 3 };

struct GbParams {
  int64_t n_rows;
  int32_t n_cols, n_keys, n_preds, n_aggs;
  const uint8_t* col[REL_MAX_COLS];
  int32_t ctype[REL_MAX_COLS];
  int32_t csize[REL_MAX_COLS];
  uint32_t stage_off[REL_MAX_COLS];  // byte offset of column c inside one stage
  uint32_t stage_bytes;              // bytes of one stage (all columns)
  int32_t tile_rows;                 // rows per tile, a multiple of 16
  int32_t key_col[REL_MAX_KEYS];
  int32_t key_shift[REL_MAX_KEYS];
  uint64_t key_mask[REL_MAX_KEYS];
  int32_t pred_col[REL_MAX_PREDS];
  int64_t pred_lo[REL_MAX_PREDS], pred_hi[REL_MAX_PREDS];
  int32_t aop[REL_MAX_AGGS], abase[REL_MAX_AGGS], anf[REL_MAX_AGGS];
  int32_t afcol[REL_MAX_AGGS][2];
  int64_t ac[REL_MAX_AGGS][2], as[REL_MAX_AGGS][2];
  uint32_t umax_mask;  // bit a: aggregate a keeps an unsigned max (MIN / MAX)
  // roles of the specialised shapes
  int32_t r_k0, r_k1, r_pred, r_a, r_b, r_d, r_t;  // Q1: keys, filter, sum cols, factor cols
  // global table (or key set in MODE_KEYSET)
  uint64_t* tkeys;
  unsigned long long* taggs;  // slots x n_aggs words
  int32_t log2_slots;
  uint32_t max_probe;
  uint32_t smem_slots;  // MODE_SHARED / MODE_KEYSET per-CTA table slots (power of two)
  WsHeader* hdr;
};

struct GbOut {
  int64_t* keys;
  int64_t* aggs[REL_MAX_AGGS];
  int64_t capacity;
};

// Host-side launchers (groupby.cu).
rel_status gb_launch_main(const GbParams& p, int shape, int mode, bool use_tma,
                          cudaStream_t st);
rel_status gb_launch_compact(const GbParams& p, const GbOut& o, cudaStream_t st);
// Aggregate-array width the kernel for a shape is compiled with.
int gb_shape_width(int shape);
// Shared-memory bytes of a backend's per-CTA table (before the staging ring).
uint64_t gb_backend_smem_bytes(int mode, int shape, uint32_t smem_slots);

}  // namespace rel
