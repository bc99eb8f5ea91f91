// Join launch parameters shared between the kernels (join.cu) and the C-ABI
// layer (api.cu).
#pragma once

#include "rel_internal.cuh"

namespace rel {

// Table entry payload: the build row's payload and index (16 bytes).
struct alignas(16) JoinVal {
  long long payload;
  int32_t bidx;
  int32_t pad;
};

// One slot of the single-call join table: the stored key (key ^ KEY_FLIP,
// 0 = empty) and the build row index -- 16 bytes, read with one 128-bit
// load.  The payload is gathered by that index from the table's own copy of
// the payload column, so the L2-resident part of a 10^6-row table is 32 MB of
// slots + 8 MB of payloads.
struct alignas(16) JoinSlot {
  unsigned long long ek;
  int32_t bidx;
  int32_t pad;
};
static_assert(sizeof(JoinSlot) == 16, "two slots per sector");

// Workspace layout: [WsHeader 256 B][slots x 16 B][payload n_build x 8 B]
//                   [side n_build x 16 B]
struct JoinParams {
  JoinSlot* slots;
  long long* pay;    // payload of build row j at pay[j]
  JoinVal* side;     // build rows whose key is INT64_MIN
  WsHeader* hdr;
  int32_t log2_slots;
};

struct JoinOut {
  int32_t* probe_idx;
  int32_t* build_idx;
  int64_t* payload;
  int64_t capacity;
};

rel_status join_launch_build(const JoinParams& p, const int64_t* keys, const int64_t* payload,
                             int64_t n, cudaStream_t st);
// emit = false counts the pairs into hdr->aux (the exact output size).
rel_status join_launch_probe(const JoinParams& p, const JoinOut& o, const int64_t* probe,
                             int64_t n, bool emit, cudaStream_t st);

}  // namespace rel
