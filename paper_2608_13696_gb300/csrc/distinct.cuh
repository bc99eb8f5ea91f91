// Exact distinct count of one int32 / int64 key column (the plain form's
// sizing pre-pass): parameters shared between the kernel (distinct.cu) and
// the C-ABI layer (api.cu).
#pragma once

#include "rel_internal.cuh"

namespace rel {

// The key set is an array of buckets of DS_BUCKET_SLOTS stored keys (one
// 32-byte sector each, read with one 256-bit load).  A key's probe sequence
// starts at its home bucket and walks the following buckets; DS_MAX_PROBE
// buckets without a free slot or the key mean the set is too full (overflow).
constexpr int DS_BUCKET_SLOTS = 4;
constexpr int DS_MAX_PROBE = 64;

struct DistinctParams {
  const void* keys;       // int32 or int64 column (device)
  int64_t n_rows;
  uint64_t* set;          // n_buckets x DS_BUCKET_SLOTS stored keys, zeroed
  uint64_t n_buckets;     // any count >= 1
  uint32_t n_pass, pass;  // hash split: this launch counts keys of pass `pass`
  uint32_t filter_slots;  // per-CTA filter of recently sent keys: 0 or a power of two
  WsHeader* hdr;          // aux += distinct keys of this pass; n_side += INT64_MIN rows
                          // (pass 0); overflow set when a probe gives up
};

// Bytes of shared memory the kernel needs for a filter of `filter_slots`.
inline size_t distinct_smem_bytes(uint32_t filter_slots) { return 8ull * filter_slots; }

rel_status distinct_launch(const DistinctParams& p, int key_type, cudaStream_t st);

// HyperLogLog over every key of one int32 / int64 column (p = 12: 4096
// registers, caller-zeroed device uint32[4096]; register = top 12 bits of
// fmix64(key ^ 2^63), value = leading zeros of the remaining 52 bits + 1,
// 53 when they are all zero).  One streaming pass.
constexpr int HLL_P = 12;
constexpr int HLL_REGS = 1 << HLL_P;
rel_status hll_launch(const void* keys, int key_type, int64_t n, uint32_t* regs, cudaStream_t st);
// Cardinality estimate of HLL_REGS registers (Flajolet, Fusy, Gandouet and
// Meunier 2007, with the small-range correction).
double hll_estimate(const uint32_t* regs);

}  // namespace rel
