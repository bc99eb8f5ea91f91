// Batched execution of many small group-by and join instances in two
// persistent launches (batch.cu).
#pragma once

#include "join.cuh"
#include "rel_internal.cuh"

namespace rel {

constexpr int BATCH_MAX_AGGS = 4;
constexpr int BATCH_MAX_SMEM_SLOTS = 4096;
// Rows of one group-by work item: up to this many tiles of blockDim x ITEMS
// rows, so the per-item costs (the work counter, the instance search, the
// descriptor copy, clearing and flushing a shared-memory table) are paid once
// per ~64K rows rather than once per tile.
constexpr int BATCH_GB_SPAN = 32;

// One group-by instance as the kernels see it.
struct alignas(16) BatchGb {
  const void* keys;
  const int64_t* vals;
  int64_t n_rows;
  uint64_t* tkeys;             // slots stored keys (key ^ KEY_FLIP), 0 = empty
  unsigned long long* taggs;   // slots x n_aggs words, slot-major
  int64_t* out_keys;
  int64_t* out_aggs[BATCH_MAX_AGGS];
  int64_t out_capacity;
  int32_t key_type;  // REL_I32 or REL_I64
  int32_t n_aggs;
  int32_t ops[BATCH_MAX_AGGS];
  int32_t log2_slots;
  int32_t smem_slots;  // 0: every row updates the global table
  uint32_t max_probe;
  int32_t span;        // tiles of blockDim x ITEMS rows per work item
};

// One join partition: its build side, its probe side, its table and outputs.
struct alignas(16) BatchJoin {
  const int64_t* bkeys;
  const int64_t* bpay;
  int64_t n_build;
  const int64_t* pkeys;
  int64_t n_probe;
  uint64_t* tkeys;
  JoinVal* tvals;
  JoinVal* side;  // build rows whose key is INT64_MIN
  int32_t* o_pi;
  int32_t* o_bi;
  int64_t* o_pay;
  int64_t capacity;
  int32_t log2_slots;
  uint32_t max_probe;
};

// Per-instance results, zeroed before every run.
struct alignas(64) BatchStatus {
  unsigned long long n_out;   // groups, or pairs
  unsigned long long n_side;  // rows (group-by) or build rows (join) with key INT64_MIN
  unsigned int overflow;      // a bounded probe gave up
  unsigned int pad;
  unsigned long long side_aggs[BATCH_MAX_AGGS];
};

struct BatchArgs {
  const BatchGb* gb;
  const BatchJoin* jn;
  const long long* gb_tiles;  // [n_g + 1] exclusive prefix of each instance's row tiles
  const long long* jb_tiles;  // [n_j + 1] build tiles
  const long long* jp_tiles;  // [n_j + 1] probe tiles
  const long long* gc_tiles;  // [n_g + 1] compaction tiles (table slots)
  BatchStatus* gst;
  BatchStatus* jst;
  unsigned long long* ctr;  // [2] work counters of the two launches
  int32_t n_g, n_j;
};

// Launch the two persistent kernels (items rows per thread per tile, probe
// width threads per table probe); grid sizes and dynamic shared memory from
// the caller.
rel_status batch_launch(const BatchArgs& a, int block, int items, int width, int smem_bytes,
                        int grid_a, int grid_b, cudaStream_t st);
rel_status batch_occupancy(int block, int items, int width, int smem_bytes, int* per_sm_a,
                           int* per_sm_b);

}  // namespace rel
