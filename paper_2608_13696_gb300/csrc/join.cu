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
  bool dup = false;
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
      uint64_t cur = ld_relaxed(p.tkeys + s);
      if (cur == 0) {
        cur = atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek);
        if (cur == 0) {
          p.tvals[s] = v;
          placed = true;
          break;
        }
      }
      // Two inserts of one key start at the same slot and claim slots in
      // probe order, so the later one always passes the earlier one's slot:
      // duplicates are always noticed.
      if (cur == ek) dup = true;
      s = (s + 1) & mask;
    }
    if (!placed) atomicOr(&p.hdr->overflow, 1u);
  }
  if (dup) atomicOr(&p.hdr->dups, 1u);
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

// Probe with J_IT rows per thread in flight.  Every row's first slot and, for
// a hit, its payload are loaded for all J_IT rows before any is used, so a
// warp keeps J_IT independent L2 round trips outstanding instead of one.
// With unique build keys (no duplicate seen while building) a row stops at
// its first match; otherwise -- and for the INT64_MIN side list -- it walks
// its whole probe sequence.  Matches are written in row-slot order: one
// atomic per warp reserves the tile's output, each row-slot's matches are
// compacted with a ballot, so consecutive lanes write consecutive entries.
constexpr int J_IT = 4;

template <bool EMIT>
__global__ void __launch_bounds__(J_BLOCK) join_probe_fast_k(const __grid_constant__ JoinParams p,
                                                             const __grid_constant__ JoinOut o,
                                                             const int64_t* __restrict__ probe,
                                                             int64_t n) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  const bool unique = ld_relaxed_u32(&p.hdr->dups) == 0;
  const uint64_t n_side = p.hdr->n_side;
  unsigned long long counted = 0;
  const int64_t tile = (int64_t)J_BLOCK * J_IT;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
    uint64_t ek[J_IT], s[J_IT], k[J_IT];
    bool hit[J_IT], slow[J_IT];
#pragma unroll
    for (int j = 0; j < J_IT; ++j) {
      const int64_t i = base + (int64_t)j * J_BLOCK + threadIdx.x;
      ek[j] = i < n ? ((uint64_t)__ldcs((const long long*)probe + i) ^ KEY_FLIP) : 0;
      s[j] = slot_of(ek[j], p.log2_slots);
    }
#pragma unroll
    for (int j = 0; j < J_IT; ++j) k[j] = p.tkeys[s[j]];
#pragma unroll
    for (int j = 0; j < J_IT; ++j) {
      const int64_t i = base + (int64_t)j * J_BLOCK + threadIdx.x;
      const bool valid = i < n;
      slow[j] = valid && (ek[j] == 0 || !unique);
      hit[j] = false;
      if (valid && !slow[j]) {
        for (uint64_t step = 0; step <= mask && k[j] != 0 && k[j] != ek[j]; ++step) {
          s[j] = (s[j] + 1) & mask;
          k[j] = p.tkeys[s[j]];
        }
        hit[j] = k[j] == ek[j];
      }
    }
    JoinVal v[J_IT];
    if (EMIT) {
#pragma unroll
      for (int j = 0; j < J_IT; ++j)
        if (hit[j]) v[j] = p.tvals[s[j]];
    }
    unsigned m[J_IT];
    unsigned total = 0;
#pragma unroll
    for (int j = 0; j < J_IT; ++j) {
      m[j] = __ballot_sync(0xffffffffu, hit[j]);
      total += __popc(m[j]);
    }
    if (!EMIT) {
      counted += lane == 0 ? total : 0;
    } else if (total) {
      unsigned long long wb = 0;
      if (lane == 0) wb = atomicAdd(&p.hdr->n_out, (unsigned long long)total);
      wb = __shfl_sync(0xffffffffu, wb, 0);
#pragma unroll
      for (int j = 0; j < J_IT; ++j) {
        if (hit[j]) {
          const uint64_t pos = wb + __popc(m[j] & lt);
          if (pos < (uint64_t)o.capacity) {
            o.probe_idx[pos] = (int32_t)(base + (int64_t)j * J_BLOCK + threadIdx.x);
            o.build_idx[pos] = v[j].bidx;
            o.payload[pos] = v[j].payload;
          }
        }
        wb += __popc(m[j]);
      }
    }
    // rows that may match more than once (or the INT64_MIN side list): walk
    // the whole sequence, one match per round, compacted per round
#pragma unroll
    for (int j = 0; j < J_IT; ++j) {
      if (!__any_sync(0xffffffffu, slow[j])) continue;
      const int64_t i = base + (int64_t)j * J_BLOCK + threadIdx.x;
      const bool side = ek[j] == 0;
      uint64_t q = side ? 0 : slot_of(ek[j], p.log2_slots);
      bool active = slow[j];
      while (__any_sync(0xffffffffu, active)) {
        JoinVal w;
        bool h = false;
        if (active) {
          h = next_match(p, ek[j], side, n_side, q, w);
          active = h;
        }
        if (!EMIT) {
          counted += h;
          continue;
        }
        const unsigned mm = __ballot_sync(0xffffffffu, h);
        if (!mm) continue;
        unsigned long long wb = 0;
        if (lane == 0) wb = atomicAdd(&p.hdr->n_out, (unsigned long long)__popc(mm));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (h) {
          const uint64_t pos = wb + __popc(mm & lt);
          if (pos < (uint64_t)o.capacity) {
            o.probe_idx[pos] = (int32_t)i;
            o.build_idx[pos] = w.bidx;
            o.payload[pos] = w.payload;
          }
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
  // one wave of resident CTAs, each walking the tiles: a second, partial
  // wave would leave most SMs idle at the end
  static int occ[2] = {0, 0};
  int& o_ = occ[emit ? 1 : 0];
  if (o_ == 0) {
    const cudaError_t e0 =
        emit ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_, join_probe_fast_k<true>, J_BLOCK, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o_, join_probe_fast_k<false>, J_BLOCK, 0);
    if (e0 != cudaSuccess || o_ < 1) o_ = 4;
  }
  const int64_t tiles = (n + (int64_t)J_BLOCK * J_IT - 1) / ((int64_t)J_BLOCK * J_IT);
  int64_t g = (int64_t)relhost::device_sms() * o_;
  if (g > tiles) g = tiles;
  relhost::launch_begin(id, st);
  if (emit)
    join_probe_fast_k<true><<<(int)g, J_BLOCK, 0, st>>>(p, o, probe, n);
  else
    join_probe_fast_k<false><<<(int)g, J_BLOCK, 0, st>>>(p, o, probe, n);
  relhost::launch_end(id, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(join probe)");
}

}  // namespace rel
