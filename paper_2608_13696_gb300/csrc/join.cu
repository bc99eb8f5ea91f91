// Hash equi-join kernels for sm_103a: build, count and probe.
//
// The paper's join runs three kernels over a hash table that is read
// randomly: insert (build), count (size the output) and retrieve (emit the
// matches), with the payload brought in by a separate gather (Sec. 7,
// Table 9).  Here the table is an open-addressing array at load <= 1/2 --
// 2^21 slots x 24 bytes for a 10^6-row build side, so it stays resident in
// the 129 MB L2 while the probe side streams from HBM -- and the probe writes
// (probe_idx, build_idx, payload) directly: each warp compacts its lanes'
// matches with a ballot / popc and reserves output space with one atomic.
#include "join.cuh"

namespace rel {

namespace {

constexpr int J_BLOCK = 256;

__global__ void __launch_bounds__(J_BLOCK) join_build_k(const __grid_constant__ JoinParams p,
                                                        const int64_t* __restrict__ keys,
                                                        const int64_t* __restrict__ payload,
                                                        int64_t n) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  for (int64_t j = (int64_t)blockIdx.x * J_BLOCK + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * J_BLOCK) {
    const uint64_t ek = (uint64_t)__ldg((const long long*)keys + j) ^ KEY_FLIP;
    const JoinVal v{__ldg((const long long*)payload + j), (int32_t)j, 0};
    if (ek == 0) {  // INT64_MIN: side list
      const unsigned long long pos = atomicAdd(&p.hdr->n_side, 1ull);
      p.side[pos] = v;
      continue;
    }
    uint64_t s = slot_of(ek, p.log2_slots);
    bool placed = false;
    for (uint64_t i = 0; i <= mask; ++i) {
      if (ld_relaxed(p.tkeys + s) == 0 &&
          atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek) == 0) {
        p.tvals[s] = v;
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    if (!placed) atomicOr(&p.hdr->overflow, 1u);
  }
}

// Next match of a lane's probe sequence.  State: slot s (table) or index s
// into the side list (key INT64_MIN).  Returns false when the sequence ends.
__device__ __forceinline__ bool next_match(const JoinParams& p, uint64_t ek, bool side,
                                           uint64_t n_side, uint64_t& s, JoinVal& out) {
  if (side) {
    if (s >= n_side) return false;
    out = p.side[s++];
    return true;
  }
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  for (uint64_t i = 0; i <= mask; ++i) {
    const uint64_t k = p.tkeys[s];
    if (k == 0) return false;
    const uint64_t cur = s;
    s = (s + 1) & mask;
    if (k == ek) {
      out = p.tvals[cur];
      return true;
    }
  }
  return false;
}

template <bool EMIT>
__global__ void __launch_bounds__(J_BLOCK) join_probe_k(const __grid_constant__ JoinParams p,
                                                        const __grid_constant__ JoinOut o,
                                                        const int64_t* __restrict__ probe,
                                                        int64_t n) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t n_side = p.hdr->n_side;
  unsigned long long counted = 0;
  for (int64_t base = (int64_t)blockIdx.x * J_BLOCK; base < n;
       base += (int64_t)gridDim.x * J_BLOCK) {
    const int64_t i = base + threadIdx.x;
    bool active = i < n;
    const uint64_t ek = active ? ((uint64_t)__ldg((const long long*)probe + i) ^ KEY_FLIP) : 0;
    const bool side = ek == 0;
    uint64_t s = side ? 0 : slot_of(ek, p.log2_slots);
    while (__any_sync(0xffffffffu, active)) {
      JoinVal v;
      bool hit = false;
      if (active) {
        hit = next_match(p, ek, side, n_side, s, v);
        active = hit;
      }
      if (!EMIT) {
        counted += hit;
        continue;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (!m) continue;
      unsigned long long wb = 0;
      if (lane == 0) wb = atomicAdd(&p.hdr->n_out, (unsigned long long)__popc(m));
      wb = __shfl_sync(0xffffffffu, wb, 0);
      if (hit) {
        const uint64_t pos = wb + __popc(m & lt);
        if (pos < (uint64_t)o.capacity) {
          o.probe_idx[pos] = (int32_t)i;
          o.build_idx[pos] = v.bidx;
          o.payload[pos] = v.payload;
        }
      }
    }
  }
  if (!EMIT) {
#pragma unroll
    for (int off = 16; off; off >>= 1) counted += __shfl_xor_sync(0xffffffffu, counted, off);
    if (lane == 0 && counted) atomicAdd(&p.hdr->aux, counted);
  }
}

int grid_for(int64_t n, int per_sm_hint) {
  int64_t g = (n + J_BLOCK - 1) / J_BLOCK;
  const int64_t cap = (int64_t)relhost::device_sms() * per_sm_hint;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

rel_status join_launch_build(const JoinParams& p, const int64_t* keys, const int64_t* payload,
                             int64_t n, cudaStream_t st) {
  if (n == 0) return REL_OK;
  relhost::launch_begin(relhost::K_JOIN_BUILD, st);
  join_build_k<<<grid_for(n, 8), J_BLOCK, 0, st>>>(p, keys, payload, n);
  relhost::launch_end(relhost::K_JOIN_BUILD, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(join build)");
}

rel_status join_launch_probe(const JoinParams& p, const JoinOut& o, const int64_t* probe,
                             int64_t n, bool emit, cudaStream_t st) {
  if (n == 0) return REL_OK;
  const int id = emit ? relhost::K_JOIN_PROBE : relhost::K_JOIN_COUNT;
  relhost::launch_begin(id, st);
  if (emit)
    join_probe_k<true><<<grid_for(n, 8), J_BLOCK, 0, st>>>(p, o, probe, n);
  else
    join_probe_k<false><<<grid_for(n, 8), J_BLOCK, 0, st>>>(p, o, probe, n);
  relhost::launch_end(id, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(join probe)");
}

}  // namespace rel
