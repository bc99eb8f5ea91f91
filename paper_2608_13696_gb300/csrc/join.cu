// Hash equi-join kernels for sm_103a: build, count and probe.
//
// The paper's join runs three kernels over a hash table that is read
// randomly: insert (build), count (size the output) and retrieve (emit the
// matches), with the payload brought in by a separate gather (Sec. 7,
// Table 9), and finds count and retrieve bound by instruction issue and
// memory latency on GH200.  Here the table is an open-addressing array at
// load <= 1/2 of 16-byte slots (key, build row index) plus the table's own
// copy of the payload column -- 32 MB + 8 MB for a 10^6-row build side, small
// enough to stay in the GB300's L2 (whose random-access sweet spot is below
// ~64 MB) while the probe keys stream from HBM with evict-first loads and the
// outputs leave with streaming stores.  The payload gather is fused into the
// probe.  Every probe row's first slot is loaded before any is resolved,
// probe keys arrive in 16-byte vector loads, and each warp compacts its
// lanes' matches with a ballot / popc and reserves output space with one
// atomic.
#include "join.cuh"

namespace rel {

namespace {

constexpr int J_BLOCK = 256;

// One slot (key, build row index), marked evict-last in L2 so that the table
// outlives the streamed probe keys (evict-first) and the streamed outputs.
__device__ __forceinline__ void ld_slot(const JoinSlot* p, uint64_t& ek, int32_t& bidx) {
  unsigned long long a, b;
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
      "ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], pol;\n\t}"
      : "=l"(a), "=l"(b)
      : "l"(p));
  ek = a;
  bidx = (int32_t)(uint32_t)b;
}

__global__ void __launch_bounds__(J_BLOCK) join_build_k(const __grid_constant__ JoinParams p,
                                                        const int64_t* __restrict__ keys,
                                                        const int64_t* __restrict__ payload,
                                                        int64_t n) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  bool dup = false;
  for (int64_t j = (int64_t)blockIdx.x * J_BLOCK + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * J_BLOCK) {
    const uint64_t ek = (uint64_t)__ldg((const long long*)keys + j) ^ KEY_FLIP;
    const long long pay = __ldg((const long long*)payload + j);
    p.pay[j] = pay;  // the table's copy of the payload column
    if (ek == 0) {  // INT64_MIN: side list
      const unsigned long long pos = atomicAdd(&p.hdr->n_side, 1ull);
      p.side[pos] = JoinVal{pay, (int32_t)j, 0};
      continue;
    }
    uint64_t s = slot_of(ek, p.log2_slots);
    bool placed = false;
    for (uint64_t i = 0; i <= mask; ++i) {
      uint64_t cur = ld_relaxed((const uint64_t*)&p.slots[s].ek);
      if (cur == 0) {
        cur = atomicCAS(&p.slots[s].ek, 0ull, (unsigned long long)ek);
        if (cur == 0) {
          p.slots[s].bidx = (int32_t)j;
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
                                           uint64_t n_side, uint64_t& s, int64_t& pay,
                                           int32_t& bidx) {
  if (side) {
    if (s >= n_side) return false;
    const JoinVal v = p.side[s++];
    pay = v.payload;
    bidx = v.bidx;
    return true;
  }
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  for (uint64_t i = 0; i <= mask; ++i) {
    uint64_t k;
    ld_slot(p.slots + s, k, bidx);
    if (k == 0) return false;
    s = (s + 1) & mask;
    if (k == ek) {
      pay = p.pay[bidx];
      return true;
    }
  }
  return false;
}

// Probe with J_IT rows per thread in flight, in groups of J_G: every row of
// a group has its first slot (key, payload, build index) loaded before any is
// resolved, so a warp keeps J_G independent L2 round trips outstanding per
// lane.  With unique build keys (no duplicate seen while building) a row
// stops at its first match; otherwise -- and for the INT64_MIN side list --
// it walks its whole probe sequence.  Matches are written in row-slot order:
// one atomic per warp and group reserves the output, each row-slot's matches
// are compacted with a ballot, so consecutive lanes write consecutive
// entries.  Rows: base + v * 2 * J_BLOCK + 2 * tid + {0, 1}, probe keys read
// two at a time with 16-byte loads.
constexpr int J_IT = 8;
constexpr int J_G = 4;

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
  const bool vec = (uintptr_t)probe % 16 == 0;
  unsigned long long counted = 0;
  const int64_t tile = (int64_t)J_BLOCK * J_IT;
  for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
    uint64_t ek[J_IT];
    int64_t row[J_IT];
#pragma unroll
    for (int v = 0; v < J_IT / 2; ++v) {
      const int64_t r = base + (int64_t)v * 2 * J_BLOCK + 2 * threadIdx.x;
      row[2 * v] = r;
      row[2 * v + 1] = r + 1;
      if (vec && r + 1 < n) {
        const longlong2 kk = __ldcs((const longlong2*)(probe + r));
        ek[2 * v] = (uint64_t)kk.x ^ KEY_FLIP;
        ek[2 * v + 1] = (uint64_t)kk.y ^ KEY_FLIP;
      } else {
        ek[2 * v] = r < n ? (uint64_t)__ldcs((const long long*)probe + r) ^ KEY_FLIP : 0;
        ek[2 * v + 1] = r + 1 < n ? (uint64_t)__ldcs((const long long*)probe + r + 1) ^ KEY_FLIP : 0;
      }
    }
#pragma unroll
    for (int g = 0; g < J_IT; g += J_G) {
      uint64_t s[J_G], k[J_G];
      int64_t pay[J_G];
      int32_t bidx[J_G];
      bool hit[J_G], slow[J_G];
#pragma unroll
      for (int q = 0; q < J_G; ++q) {
        const bool valid = row[g + q] < n;
        slow[q] = valid && (ek[g + q] == 0 || !unique);
        s[q] = slot_of(ek[g + q], p.log2_slots);
        k[q] = 0;
        if (valid && !slow[q]) ld_slot(p.slots + s[q], k[q], bidx[q]);
      }
#pragma unroll
      for (int q = 0; q < J_G; ++q) {
        hit[q] = false;
        if (row[g + q] < n && !slow[q]) {
          for (uint64_t step = 0; step <= mask && k[q] != 0 && k[q] != ek[g + q]; ++step) {
            s[q] = (s[q] + 1) & mask;
            ld_slot(p.slots + s[q], k[q], bidx[q]);
          }
          hit[q] = k[q] == ek[g + q];
        }
      }
      // the payload gather of every hit of the group
#pragma unroll
      for (int q = 0; q < J_G; ++q)
        if (EMIT && hit[q]) pay[q] = __ldg(p.pay + bidx[q]);
      unsigned m[J_G];
      unsigned total = 0;
#pragma unroll
      for (int q = 0; q < J_G; ++q) {
        m[q] = __ballot_sync(0xffffffffu, hit[q]);
        total += __popc(m[q]);
      }
      if (!EMIT) {
        counted += lane == 0 ? total : 0;
      } else if (total) {
        unsigned long long wb = 0;
        if (lane == 0) wb = atomicAdd(&p.hdr->n_out, (unsigned long long)total);
        wb = __shfl_sync(0xffffffffu, wb, 0);
#pragma unroll
        for (int q = 0; q < J_G; ++q) {
          if (hit[q]) {
            const uint64_t pos = wb + __popc(m[q] & lt);
            if (pos < (uint64_t)o.capacity) {  // streaming stores: keep the table in L2
              __stcs(o.probe_idx + pos, (int32_t)row[g + q]);
              __stcs(o.build_idx + pos, bidx[q]);
              __stcs((long long*)o.payload + pos, (long long)pay[q]);
            }
          }
          wb += __popc(m[q]);
        }
      }
      // rows that may match more than once (or the INT64_MIN side list): walk
      // the whole sequence, one match per round, compacted per round
#pragma unroll
      for (int q = 0; q < J_G; ++q) {
        if (!__any_sync(0xffffffffu, slow[q])) continue;
        const bool side = ek[g + q] == 0;
        uint64_t qs = side ? 0 : slot_of(ek[g + q], p.log2_slots);
        bool active = slow[q];
        while (__any_sync(0xffffffffu, active)) {
          int64_t wp = 0;
          int32_t wi = 0;
          bool h = false;
          if (active) {
            h = next_match(p, ek[g + q], side, n_side, qs, wp, wi);
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
              o.probe_idx[pos] = (int32_t)row[g + q];
              o.build_idx[pos] = wi;
              o.payload[pos] = wp;
            }
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
