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

// Workspace layout: [WsHeader 256 B][tkeys slots x 8 B][tvals slots x 16 B]
//                   [side n_build x 16 B]
struct JoinParams {
  uint64_t* tkeys;   // stored keys (key ^ KEY_FLIP), 0 = empty
  JoinVal* tvals;
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
