// Batched group-by and join: thousands of uneven instances in two persistent
// launches instead of several launches (and host round trips) per instance.
//
// Most of the paper's kernel time at small scale factors sits in launches
// too small to fill the GPU (Sec. 5.3).  Here every instance is cut into
// tiles of blockDim x ITEMS rows; each CTA of a persistent grid (sized to the
// resident capacity) takes the next tile from one atomic work counter, finds
// its instance by binary search over the tiles' prefix sums, and processes
// it.  Launch A: join builds and group-by aggregation (independent).  Launch
// B: join probes (after every build) and group-by compaction (after every
// aggregation).  The caller zeroes the counters and tables before A, so one
// batch is one memset plus two launches, which a CUDA graph replays.
//
// Tables follow the single-instance kernels: open addressing on stored keys
// key ^ 2^63 (0 = empty, INT64_MIN on a side path), zero-identity aggregate
// words, bounded probing with an overflow flag per instance.  Probing is done
// by W cooperating threads (W = 1, 2, 4, 8) that each read one slot of a
// W-slot window.  Group-by instances with few groups can pre-aggregate each
// tile in a shared-memory table and merge it into the global table.
#include <cooperative_groups.h>

#include <type_traits>

#include "batch.cuh"

namespace cg = cooperative_groups;

namespace rel {

namespace {

constexpr uint32_t BATCH_SMEM_MULT = 0x9E3779B1u;
constexpr int BATCH_SMEM_PROBES = 32;

__device__ __forceinline__ int find_instance(const long long* start, int n, long long item) {
  int lo = 0, hi = n;  // start[lo] <= item < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= item)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t encode_word(int op, int64_t v) {
  return op == REL_COUNT ? 1ull
         : op == REL_MIN ? (uint64_t)v ^ MIN_FLIP
         : op == REL_MAX ? (uint64_t)v ^ MAX_FLIP
                         : (uint64_t)v;
}

__device__ __forceinline__ void red_global(unsigned long long* w, int op, uint64_t x) {
  if (op == REL_MIN || op == REL_MAX)
    atomicMax(w, (unsigned long long)x);
  else
    atomicAdd(w, (unsigned long long)x);
}

__device__ __forceinline__ void red_shared(unsigned long long* w, int op, uint64_t x) {
  if (op == REL_MIN || op == REL_MAX) {
    if (x > *(volatile unsigned long long*)w) atomicMax(w, (unsigned long long)x);
  } else {
    sadd64(w, x);
  }
}

// The encoded words of one row (or of a pre-aggregated slot) for aggregate a.
struct Words {
  uint64_t w[BATCH_MAX_AGGS];
};

__device__ __forceinline__ Words row_words(const BatchGb& g, int64_t v) {
  Words x;
#pragma unroll
  for (int a = 0; a < BATCH_MAX_AGGS; ++a) x.w[a] = a < g.n_aggs ? encode_word(g.ops[a], v) : 0;
  return x;
}

__device__ __forceinline__ void red_words(const BatchGb& g, unsigned long long* t, const Words& x) {
#pragma unroll
  for (int a = 0; a < BATCH_MAX_AGGS; ++a)
    if (a < g.n_aggs) red_global(t + a, g.ops[a], x.w[a]);
}

__device__ __forceinline__ void side_update(const BatchGb& g, BatchStatus* st, const Words& x) {
  atomicAdd(&st->n_side, 1ull);
  red_words(g, st->side_aggs, x);
}

// One thread: insert-or-accumulate encoded words into the global table,
// starting from slot s whose content cur was already loaded.
__device__ __forceinline__ void global_resolve(const BatchGb& g, BatchStatus* st, uint64_t ek,
                                               uint64_t s, uint64_t cur, const Words& x) {
  const uint64_t mask = (1ull << g.log2_slots) - 1;
  for (uint32_t i = 0; i < g.max_probe; ++i) {
    if (i) cur = ld_relaxed(g.tkeys + s);
    if (cur == 0) {
      cur = atomicCAS((unsigned long long*)(g.tkeys + s), 0ull, (unsigned long long)ek);
      if (cur == 0) cur = ek;
    }
    if (cur == ek) {
      red_words(g, g.taggs + s * (uint64_t)g.n_aggs, x);
      return;
    }
    s = (s + 1) & mask;
    if ((i & 31) == 31 && ld_relaxed_u32(&st->overflow)) return;  // already overflowed
  }
  atomicOr(&st->overflow, 1u);
}

__device__ __forceinline__ void global_update(const BatchGb& g, BatchStatus* st, uint64_t ek,
                                              const Words& x) {
  const uint64_t s = slot_of(ek, g.log2_slots);
  global_resolve(g, st, ek, s, ld_relaxed(g.tkeys + s), x);
}

// W threads probe together: each reads one slot of a W-slot window; a key
// found anywhere in the window is updated, else the lowest empty slot is
// claimed.  Slots are never freed, so every inserter of a key meets the same
// first window with room and finds the key there.  (ek, v, valid) is the
// calling thread's row; the group serves its W rows one after another.
template <int W>
__device__ __noinline__ void global_update_coop(const BatchGb& g, BatchStatus* st, uint64_t ek,
                                                int64_t v, bool valid) {
  const auto tile = cg::tiled_partition<W>(cg::this_thread_block());
  const uint64_t mask = (1ull << g.log2_slots) - 1;
  const int rank = (int)tile.thread_rank();
  for (int r = 0; r < W; ++r) {
    const uint64_t k = tile.shfl(ek, r);
    const int64_t vr = tile.shfl(v, r);
    if (!tile.shfl((int)valid, r)) continue;
    const Words x = row_words(g, vr);
    if (k == 0) {
      if (rank == 0) side_update(g, st, x);
      continue;
    }
    const uint64_t base = slot_of(k, g.log2_slots);
    bool done = false;
    for (uint32_t i = 0; i < g.max_probe && !done; i += W) {
      if ((i & 31) == 32 - W && tile.any(ld_relaxed_u32(&st->overflow) != 0)) {
        done = true;  // already overflowed: the result is discarded
        break;
      }
      const uint64_t s = (base + i + rank) & mask;
      const uint64_t cur = ld_relaxed(g.tkeys + s);
      const unsigned hit = tile.ballot(cur == k);
      if (hit) {
        if (rank == __ffs(hit) - 1) red_words(g, g.taggs + s * (uint64_t)g.n_aggs, x);
        done = true;
        break;
      }
      unsigned emp = tile.ballot(cur == 0);
      while (emp) {
        const int leader = __ffs(emp) - 1;
        unsigned long long res = 0;
        if (rank == leader) {
          res = atomicCAS((unsigned long long*)(g.tkeys + s), 0ull, (unsigned long long)k);
          if (res == 0 || res == k) red_words(g, g.taggs + s * (uint64_t)g.n_aggs, x);
        }
        res = tile.shfl(res, leader);
        if (res == 0 || res == k) {
          done = true;
          break;
        }
        emp &= ~(1u << leader);
      }
    }
    if (!done && rank == 0) atomicOr(&st->overflow, 1u);
  }
}

// One tile of B x ITEMS rows starting at row r0: each row goes to the
// shared-memory table (when the instance has one) or the global table.
template <int ITEMS, int W>
__device__ __forceinline__ void gb_rows(const BatchGb& g, BatchStatus* st, long long r0,
                                        uint64_t* smk, unsigned long long* sma) {
  const int B = blockDim.x;
  uint64_t ek[ITEMS];
  int64_t vv[ITEMS];
  bool ok[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const long long r = r0 + (long long)j * B + threadIdx.x;
    ok[j] = r < g.n_rows;
    int64_t k = 0, v = 0;
    if (ok[j]) {
      k = g.key_type == REL_I32 ? (int64_t)__ldcs((const int*)g.keys + r)
                                : (int64_t)__ldcs((const long long*)g.keys + r);
      if (g.vals) v = (int64_t)__ldcs((const long long*)g.vals + r);
    }
    ek[j] = (uint64_t)k ^ KEY_FLIP;
    vv[j] = v;
  }
  if (g.smem_slots) {
    const uint32_t S = (uint32_t)g.smem_slots, A = (uint32_t)g.n_aggs;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (!ok[j]) continue;
      const Words x = row_words(g, vv[j]);
      if (ek[j] == 0) {
        side_update(g, st, x);
        continue;
      }
      uint32_t s = small_slot_of(ek[j], S - 1, BATCH_SMEM_MULT);
      bool placed = false;
      for (int i = 0; i < BATCH_SMEM_PROBES; ++i) {
        uint64_t cur = *(volatile uint64_t*)(smk + s);
        if (cur == 0) {
          cur = atomicCAS((unsigned long long*)(smk + s), 0ull, (unsigned long long)ek[j]);
          if (cur == 0) cur = ek[j];
        }
        if (cur == ek[j]) {
#pragma unroll
          for (int a = 0; a < BATCH_MAX_AGGS; ++a)
            if (a < (int)A) red_shared(sma + (size_t)s * A + a, g.ops[a], x.w[a]);
          placed = true;
          break;
        }
        s = (s + 1) & (S - 1);
      }
      if (!placed) global_update(g, st, ek[j], x);
    }
    return;
  }
  if (W == 1) {
    // every row's first slot is read before any row is resolved: ITEMS
    // independent L2 round trips in flight per thread instead of one
    uint64_t gs[ITEMS], gk[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      gs[j] = slot_of(ek[j], g.log2_slots);
      gk[j] = (ok[j] && ek[j] != 0) ? ld_relaxed(g.tkeys + gs[j]) : 0;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (!ok[j]) continue;
      const Words x = row_words(g, vv[j]);
      if (ek[j] == 0)
        side_update(g, st, x);
      else
        global_resolve(g, st, ek[j], gs[j], gk[j], x);
    }
  } else {
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) global_update_coop<W>(g, st, ek[j], vv[j], ok[j]);
  }
}

// Work item t of a group-by: g.span consecutive tiles.  With a shared-memory
// table the item pre-aggregates all its rows there (cleared once, flushed to
// the global table once, one update per distinct key).
template <int ITEMS, int W>
__device__ __forceinline__ void gb_tile(const BatchGb& g, BatchStatus* st, long long t,
                                        uint64_t* smk, unsigned long long* sma) {
  const int B = blockDim.x;
  const long long T = (long long)B * ITEMS;
  const long long first = t * (long long)g.span;
  const long long last = (g.n_rows + T - 1) / T < first + g.span ? (g.n_rows + T - 1) / T
                                                                 : first + g.span;
  const uint32_t S = (uint32_t)g.smem_slots, A = (uint32_t)g.n_aggs;
  if (S) {
    for (uint32_t i = threadIdx.x; i < S * (1 + A); i += B) smk[i] = 0;
    __syncthreads();
  }
  for (long long k = first; k < last; ++k) gb_rows<ITEMS, W>(g, st, k * T, smk, sma);
  if (S) {
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < S; s += B) {
      const uint64_t k = smk[s];
      if (k == 0) continue;
      Words x;
#pragma unroll
      for (int a = 0; a < BATCH_MAX_AGGS; ++a) x.w[a] = a < (int)A ? sma[(size_t)s * A + a] : 0;
      global_update(g, st, k, x);
    }
    __syncthreads();
  }
}

template <int ITEMS>
__device__ __forceinline__ void build_tile(const BatchJoin& J, BatchStatus* st, long long t) {
  const int B = blockDim.x;
  const long long r0 = t * (long long)B * ITEMS;
  const uint64_t mask = (1ull << J.log2_slots) - 1;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const long long r = r0 + (long long)j * B + threadIdx.x;
    if (r >= J.n_build) continue;
    const uint64_t ek = (uint64_t)__ldg((const long long*)J.bkeys + r) ^ KEY_FLIP;
    const JoinVal v{__ldg((const long long*)J.bpay + r), (int32_t)r, 0};
    if (ek == 0) {
      const unsigned long long pos = atomicAdd(&st->n_side, 1ull);
      J.side[pos] = v;
      continue;
    }
    uint64_t s = slot_of(ek, J.log2_slots);
    bool placed = false;
    for (uint32_t i = 0; i < J.max_probe; ++i) {
      if (ld_relaxed(J.tkeys + s) == 0 &&
          atomicCAS((unsigned long long*)(J.tkeys + s), 0ull, (unsigned long long)ek) == 0) {
        J.tvals[s] = v;
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    if (!placed) atomicOr(&st->overflow, 1u);
  }
}

// Persistent launch A: join builds, then group-by tiles, from one counter.
template <int ITEMS, int W>
__global__ void __launch_bounds__(512) batch_a(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) uint8_t bsm[];
  __shared__ long long s_item;
  __shared__ int s_inst;
  __shared__ union {
    BatchGb g;
    BatchJoin j;
  } s_desc;
  uint64_t* smk = (uint64_t*)bsm;
  const long long n_build = a.n_j ? a.jb_tiles[a.n_j] : 0;
  const long long total = n_build + (a.n_g ? a.gb_tiles[a.n_g] : 0);
  for (;;) {
    // one thread takes the next tile and finds its instance; the CTA copies
    // that instance's descriptor into shared memory
    if (threadIdx.x == 0) {
      const long long item = (long long)atomicAdd(a.ctr, 1ull);
      s_item = item;
      s_inst = item >= total  ? -1
               : item < n_build ? find_instance(a.jb_tiles, a.n_j, item)
                                : find_instance(a.gb_tiles, a.n_g, item - n_build);
    }
    __syncthreads();
    const long long item = s_item;
    const int i = s_inst;
    if (i < 0) break;
    const bool is_build = item < n_build;
    {
      const uint4* src = is_build ? (const uint4*)(a.jn + i) : (const uint4*)(a.gb + i);
      const int words = (is_build ? sizeof(BatchJoin) : sizeof(BatchGb)) / sizeof(uint4);
      if ((int)threadIdx.x < words) ((uint4*)&s_desc)[threadIdx.x] = src[threadIdx.x];
    }
    __syncthreads();
    if (is_build) {
      build_tile<ITEMS>(s_desc.j, a.jst + i, item - a.jb_tiles[i]);
    } else {
      const BatchGb& g = s_desc.g;
      unsigned long long* sma = (unsigned long long*)(smk + g.smem_slots);
      gb_tile<ITEMS, W>(g, a.gst + i, item - n_build - a.gb_tiles[i], smk, sma);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int64_t decode_word(int op, uint64_t w) {
  return op == REL_MIN ? (int64_t)(w ^ MIN_FLIP) : op == REL_MAX ? (int64_t)(w ^ MAX_FLIP) : (int64_t)w;
}

template <int ITEMS>
__device__ __forceinline__ void compact_tile(const BatchGb& g, BatchStatus* st, long long t) {
  const int B = blockDim.x;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const long long slots = 1ll << g.log2_slots;
  const long long s0 = t * (long long)B * ITEMS;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const long long s = s0 + (long long)j * B + threadIdx.x;
    const uint64_t k = s < slots ? g.tkeys[s] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, k != 0);
    if (!m) continue;
    unsigned long long wb = 0;
    if (lane == 0) wb = atomicAdd(&st->n_out, (unsigned long long)__popc(m));
    wb = __shfl_sync(0xffffffffu, wb, 0);
    if (k != 0) {
      const unsigned long long pos = wb + __popc(m & lt);
      if (pos < (unsigned long long)g.out_capacity) {
        g.out_keys[pos] = (int64_t)(k ^ KEY_FLIP);
        const unsigned long long* w = g.taggs + (uint64_t)s * g.n_aggs;
#pragma unroll
        for (int a = 0; a < BATCH_MAX_AGGS; ++a)
          if (a < g.n_aggs) g.out_aggs[a][pos] = decode_word(g.ops[a], w[a]);
      }
    }
  }
  if (t == 0 && threadIdx.x == 0 && st->n_side > 0) {
    const unsigned long long pos = atomicAdd(&st->n_out, 1ull);
    if (pos < (unsigned long long)g.out_capacity) {
      g.out_keys[pos] = INT64_MIN;
#pragma unroll
      for (int a = 0; a < BATCH_MAX_AGGS; ++a)
        if (a < g.n_aggs) g.out_aggs[a][pos] = decode_word(g.ops[a], st->side_aggs[a]);
    }
  }
}

template <int ITEMS>
__device__ __forceinline__ void probe_tile(const BatchJoin& J, BatchStatus* st, long long t) {
  const int B = blockDim.x;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t mask = (1ull << J.log2_slots) - 1;
  const unsigned long long n_side = st->n_side;
  const long long r0 = t * (long long)B * ITEMS;
  for (int j = 0; j < ITEMS; ++j) {
    const long long r = r0 + (long long)j * B + threadIdx.x;
    const bool valid = r < J.n_probe;
    const uint64_t ek = valid ? (uint64_t)__ldg((const long long*)J.pkeys + r) ^ KEY_FLIP : 0;
    const bool side = valid && ek == 0;
    uint64_t s = side ? 0 : slot_of(ek, J.log2_slots);
    uint32_t steps = 0;
    bool active = valid;
    while (__any_sync(0xffffffffu, active)) {
      bool hit = false;
      JoinVal v{0, 0, 0};
      if (active) {
        // next match of this row's probe sequence
        if (side) {
          if (s < n_side) {
            v = J.side[s++];
            hit = true;
          }
        } else {
          while (steps < J.max_probe) {
            const uint64_t k = J.tkeys[s];
            if (k == 0) break;
            const uint64_t cur = s;
            s = (s + 1) & mask;
            ++steps;
            if (k == ek) {
              v = J.tvals[cur];
              hit = true;
              break;
            }
          }
        }
        active = hit;
      }
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      if (!m) continue;
      unsigned long long wb = 0;
      if (lane == 0) wb = atomicAdd(&st->n_out, (unsigned long long)__popc(m));
      wb = __shfl_sync(0xffffffffu, wb, 0);
      if (hit) {
        const unsigned long long pos = wb + __popc(m & lt);
        if (pos < (unsigned long long)J.capacity) {
          J.o_pi[pos] = (int32_t)r;
          J.o_bi[pos] = v.bidx;
          J.o_pay[pos] = v.payload;
        }
      }
    }
  }
}

// Persistent launch B: join probes, then group-by compaction.
template <int ITEMS>
__global__ void __launch_bounds__(512) batch_b(const __grid_constant__ BatchArgs a) {
  __shared__ long long s_item;
  __shared__ int s_inst;
  __shared__ union {
    BatchGb g;
    BatchJoin j;
  } s_desc;
  const long long n_probe = a.n_j ? a.jp_tiles[a.n_j] : 0;
  const long long total = n_probe + (a.n_g ? a.gc_tiles[a.n_g] : 0);
  for (;;) {
    if (threadIdx.x == 0) {
      const long long item = (long long)atomicAdd(a.ctr + 1, 1ull);
      s_item = item;
      s_inst = item >= total  ? -1
               : item < n_probe ? find_instance(a.jp_tiles, a.n_j, item)
                                : find_instance(a.gc_tiles, a.n_g, item - n_probe);
    }
    __syncthreads();
    const long long item = s_item;
    const int i = s_inst;
    if (i < 0) break;
    const bool is_probe = item < n_probe;
    {
      const uint4* src = is_probe ? (const uint4*)(a.jn + i) : (const uint4*)(a.gb + i);
      const int words = (is_probe ? sizeof(BatchJoin) : sizeof(BatchGb)) / sizeof(uint4);
      if ((int)threadIdx.x < words) ((uint4*)&s_desc)[threadIdx.x] = src[threadIdx.x];
    }
    __syncthreads();
    if (is_probe)
      probe_tile<ITEMS>(s_desc.j, a.jst + i, item - a.jp_tiles[i]);
    else
      compact_tile<ITEMS>(s_desc.g, a.gst + i, item - n_probe - a.gc_tiles[i]);
    __syncthreads();
  }
}

template <int ITEMS, int W>
rel_status launch_pair(const BatchArgs& a, int block, int smem, int grid_a, int grid_b,
                       cudaStream_t st) {
  relhost::launch_begin(relhost::K_BATCH_A, st);
  batch_a<ITEMS, W><<<grid_a, block, smem, st>>>(a);
  relhost::launch_end(relhost::K_BATCH_A, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return relhost::cuda_fail(e, "launch(batch A)");
  relhost::launch_begin(relhost::K_BATCH_B, st);
  batch_b<ITEMS><<<grid_b, block, 0, st>>>(a);
  relhost::launch_end(relhost::K_BATCH_B, st);
  e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(batch B)");
}

template <int ITEMS, int W>
rel_status occ_pair(int block, int smem, int* pa, int* pb) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(pa, batch_a<ITEMS, W>, block, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(pb, batch_b<ITEMS>, block, 0);
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "occupancy(batch)");
}

template <int ITEMS, class F>
rel_status with_width(int width, F&& f) {
  switch (width) {
    case 1: return f(std::integral_constant<int, ITEMS>{}, std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, ITEMS>{}, std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, ITEMS>{}, std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, ITEMS>{}, std::integral_constant<int, 8>{});
  }
  relhost::set_error("batch: probe width must be 1, 2, 4 or 8");
  return REL_E_INVALID;
}

template <class F>
rel_status with_config(int items, int width, F&& f) {
  switch (items) {
    case 4: return with_width<4>(width, f);
    case 8: return with_width<8>(width, f);
    case 16: return with_width<16>(width, f);
  }
  relhost::set_error("batch: items per thread must be 4, 8 or 16");
  return REL_E_INVALID;
}

}  // namespace

rel_status batch_launch(const BatchArgs& a, int block, int items, int width, int smem_bytes,
                        int grid_a, int grid_b, cudaStream_t st) {
  return with_config(items, width, [&](auto I, auto W) {
    return launch_pair<decltype(I)::value, decltype(W)::value>(a, block, smem_bytes, grid_a,
                                                               grid_b, st);
  });
}

rel_status batch_occupancy(int block, int items, int width, int smem_bytes, int* per_sm_a,
                           int* per_sm_b) {
  return with_config(items, width, [&](auto I, auto W) {
    return occ_pair<decltype(I)::value, decltype(W)::value>(block, smem_bytes, per_sm_a, per_sm_b);
  });
}

}  // namespace rel
