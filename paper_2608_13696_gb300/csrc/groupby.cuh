// Group-by launch parameters shared between the kernels (groupby.cu) and the
// C-ABI layer (api.cu).
#pragma once

#include "rel_internal.cuh"

namespace rel {

constexpr int GB_BLOCK = 256;                // consumer threads per CTA
constexpr int GB_THREADS = GB_BLOCK + 32;    // + one TMA producer warp
constexpr int GB_MAX_STAGES = 8;
constexpr int GB_SMEM_HEAD = 256;  // full[8] and empty[8] mbarriers, abort flag
constexpr int TINY_MAX_SLOTS = 32;
constexpr int SHARED_MAX_SLOTS = 4096;

enum GbMode : int {
  MODE_LAYERED = 0,
  MODE_KEYSET = 1,
  MODE_TINY = 2,
  MODE_PHIST = 3,     // partitioned: count rows per (partition, CTA)
  MODE_PSCATTER = 4   // partitioned: write rows into their partitions
};

// What a pass does with rows whose key is INT64_MIN (they bypass tables).
enum SideMode : int { SIDE_AGG = 0, SIDE_COUNT = 1, SIDE_SKIP = 2 };

// Partitioned group-by record: the stored key and the row's raw value.
struct alignas(16) PartRec {
  unsigned long long ek;
  long long val;
};
constexpr int PART_MAX_BITS = 14;  // at most 16384 partitions
constexpr int PART_CHUNKS = 16;    // CTAs that may share one oversized partition
// Streaming scatter in two levels: the first writes records into at most
// 2^PART_L1_BITS bins (the top bits of the partition index), the second
// splits every bin into its partitions.  Both sort a tile of PART_TILE
// records by destination in shared memory and write each destination's run
// contiguously.
constexpr int PART_L1_BITS = 8;
constexpr int PART_TILE = 4096;

// Row shapes.  The specialised ones fix column types and aggregate kinds at
// compile time; KV4 / KV2 hold their aggregates in the internal order
// (sum, count, min, max) / (sum, count) and the host permutes the outputs.
enum GbShape : int {
  SHAPE_GENERIC = 0,
  SHAPE_Q1 = 1,
  SHAPE_KVRT64 = 2,  // runtime aggregate ops, int64 key
  SHAPE_KVRT32 = 3,  // runtime aggregate ops, int32 key
  SHAPE_KV4_64 = 4,  // sum, count, min, max of one int64 value; int64 key
  SHAPE_KV4_32 = 5,
  SHAPE_KV2_64 = 6,  // sum, count
  SHAPE_KV2_32 = 7,
  SHAPE_COUNT = 8
};

// Partition of a stored key: top bits of a multiplicative hash independent
// of the table hashes.  The histogram and scatter passes must agree on it.
__device__ __forceinline__ uint32_t part_of(uint64_t ek, uint32_t bits) {
  return (uint32_t)((ek * 0xD6E8FEB86659FD93ull) >> (64 - bits));
}

struct GbParams {
  int64_t n_rows;
  int32_t n_cols, n_keys, n_preds, n_aggs;
  const uint8_t* col[REL_MAX_COLS];
  int32_t ctype[REL_MAX_COLS];
  int32_t csize[REL_MAX_COLS];
  uint32_t stage_off[REL_MAX_COLS];  // byte offset of column c inside one stage
  uint32_t stage_bytes;              // bytes of one stage (all columns)
  int32_t tile_rows;                 // rows per tile, a multiple of 16
  int32_t n_stages;                  // 2..GB_MAX_STAGES
  int32_t key_col[REL_MAX_KEYS];
  int32_t key_shift[REL_MAX_KEYS];
  uint64_t key_mask[REL_MAX_KEYS];
  int32_t pred_col[REL_MAX_PREDS];
  int64_t pred_lo[REL_MAX_PREDS], pred_hi[REL_MAX_PREDS];
  int32_t aop[REL_MAX_AGGS], abase[REL_MAX_AGGS], anf[REL_MAX_AGGS];
  int32_t afcol[REL_MAX_AGGS][2];
  int64_t ac[REL_MAX_AGGS][2], as[REL_MAX_AGGS][2];
  uint32_t umax_mask;  // bit a: aggregate word a keeps an unsigned max (MIN / MAX)
  // roles of the specialised shapes
  int32_t r_k0, r_k1, r_pred, r_a, r_b, r_d, r_t;
  // per-CTA layers
  uint32_t tiny_slots;     // 0 or 8 / 16 / 32 thread-private slots
  uint32_t tiny_probes;    // probes in the thread-private table before moving on
  uint32_t smem_slots;     // 0 or a power of two <= SHARED_MAX_SLOTS (CTA-shared table)
  uint32_t shared_probes;  // probes in the CTA-shared table before moving on
  uint32_t tiny_mult;      // multiplier of the thread-private slot hash
  uint32_t tiny_frozen;    // 1: slots preloaded from tiny_init, no other key admitted
  uint64_t tiny_init[TINY_MAX_SLOTS];  // stored keys per slot (0 = empty)
  uint64_t tiny_dense;     // register mode: 4-bit dense id of each of <= 16 slots
  uint32_t tiny_ns;        // register mode: dense slots compiled in (4 or 8)
  int32_t req_tile, req_stages;  // staging chosen by the plan (0: automatic)
  // partitioned variant
  uint32_t part_bits;       // log2 of the partition count
  uint32_t fixed_grid;      // CTAs of the histogram and scatter passes (equal)
  uint32_t* hist;           // [P][fixed_grid] counts, then exclusive offsets
  unsigned long long* part_start;  // [P + 1] first record of each partition
  PartRec* recs;            // records of every non-pinned row, by partition
  PartRec* recs1;           // streaming, part_bits > PART_L1_BITS: records by level-1 bin
  unsigned int* cursor;     // [P] next free record of each partition
  unsigned int* cursor1;    // [2^PART_L1_BITS] next free record of each level-1 bin
  unsigned int* l2_tiles;   // [bins + 1] exclusive prefix of the level-2 tiles per bin
  // global table (or key set in MODE_KEYSET)
  uint64_t* tkeys;
  unsigned long long* taggs;  // slots x n_aggs words
  int32_t log2_slots;
  uint32_t max_probe;
  WsHeader* hdr;
  uint64_t wait_ns;     // limit of every bounded device wait (WAIT_LIMIT_NS)
  uint32_t test_stall;  // test hook: consumers never hand a stage back
};

struct GbOut {
  int64_t* keys;
  int64_t* aggs[REL_MAX_AGGS];  // in the kernel's aggregate order
  int64_t capacity;
};

// Host-side launchers (groupby.cu).
rel_status gb_launch_main(const GbParams& p, int shape, int mode, bool use_tma,
                          cudaStream_t st);
rel_status gb_launch_compact(const GbParams& p, const GbOut& o, cudaStream_t st);
// Partitioned variant: partition starts (and, with cta_offsets, every CTA's
// offset inside each partition) from the histogram, then per-partition tables.
rel_status gb_launch_part_scan(const GbParams& p, bool cta_offsets, cudaStream_t st);
rel_status gb_launch_part_agg(const GbParams& p, int shape, const GbOut& o, cudaStream_t st);
// Streaming kernel for key/value shapes (stream.cu): pinned keys and/or a
// small shared table in front of the global table, no staging ring.
bool gb_stream_eligible(const GbParams& p, int shape, int n_hot);
rel_status gb_launch_stream(const GbParams& p, int shape, cudaStream_t st);
// Histogram (scatter = false) or scatter pass of the partitioned variant for
// key/value shapes, streaming; grid = p.fixed_grid CTAs in both passes.
bool gb_ppass_stream_eligible(const GbParams& p, int shape, int n_hot);
// Grid of the streaming histogram pass: the CTAs resident at once on all
// SMs, at most cap (0 when the pass cannot launch).
uint32_t gb_ppass_stream_grid(const GbParams& p, int shape, uint32_t cap);
rel_status gb_launch_ppass_stream(const GbParams& p, int shape, bool scatter, cudaStream_t st);
// Level 2 of the streaming scatter (part_bits > PART_L1_BITS): recs1 -> recs.
rel_status gb_launch_part_l2(const GbParams& p, cudaStream_t st);
// Aggregate-array width the kernel for a shape is compiled with.
int gb_shape_width(int shape);
// Shared-memory bytes of the per-CTA tables (before the staging ring).
uint64_t gb_backend_smem_bytes(int mode, int shape, uint32_t tiny_slots, uint32_t smem_slots);
// Occupancy of a configured launch (CTAs per SM), or 0 when it cannot launch.
int gb_ctas_per_sm(const GbParams& p, int shape, int mode, bool use_tma);

}  // namespace rel
