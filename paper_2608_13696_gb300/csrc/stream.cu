// Streaming group-by for key/value rows: one int32 or int64 key column, one
// int64 value column, aggregates (sum, count[, min, max]) -- the shapes KV4 /
// KV2 of the fused kernel, without its staging ring.
//
// The paper's group-by kernels are issue-bound (Sec. 5, 7): instructions per
// DRAM sector, not bandwidth, limit them.  This kernel keeps the per-row path
// short.  Rows come straight from HBM in 16-byte vector loads (two rows per
// load and column, ST_U rows per thread per chunk, evict-first), so a thread
// has 2 x ST_U / 2 loads in flight and no shared-memory staging or barrier
// sits on the path.  Each row then goes to the first layer that takes it:
//  * pinned hot keys (from the sample sketch): a one-probe perfect-hash test
//    against the pinned key, then thread-private accumulators in shared
//    memory (one column per thread: no atomics, no bank conflicts);
//  * optionally a CTA-shared table with shared-memory atomics;
//  * the global table: every row still unplaced issues its first slot read
//    before any is resolved (ST_U independent L2 round trips per thread),
//    then claims or accumulates with CAS / RED atomics, bounded probing.
// At the end each CTA folds its thread-private words (warp shuffles, then
// shared atomics) and its shared table into the global table, which the
// compaction kernel turns into the output.
#include "groupby.cuh"

namespace rel {

namespace {

constexpr int ST_BLOCK = 128;
constexpr int ST_U = 8;          // rows per thread per chunk (a multiple of 2)
// pinned keys with thread-private accumulators: 32 KB of them per CTA
template <int NA>
constexpr int pin_max() {
  return NA == 4 ? 8 : 16;
}
constexpr int ST_PIN_LIMIT = 16;
constexpr uint32_t ST_SMEM_MULT = 0x85EBCA77u;

template <int NA>
__device__ __forceinline__ void words_of(uint64_t v, uint64_t (&w)[NA]) {
  w[0] = v;
  w[1] = 1;
  if constexpr (NA == 4) {
    w[2] = v ^ MIN_FLIP;
    w[3] = v ^ MAX_FLIP;
  }
}

// word a keeps an unsigned max (MIN / MAX) rather than a sum
template <int NA>
__device__ __forceinline__ constexpr bool umax_word(int a) {
  return NA == 4 && a >= 2;
}

template <int NA>
__device__ __forceinline__ void red_global(unsigned long long* t, const uint64_t (&w)[NA]) {
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    if (umax_word<NA>(a))
      atomicMax(t + a, (unsigned long long)w[a]);
    else
      atomicAdd(t + a, (unsigned long long)w[a]);
  }
}

// Claim-or-accumulate from a first slot whose content k is already loaded.
template <int NA>
__device__ __forceinline__ void global_resolve(const GbParams& p, uint64_t ek, uint64_t s,
                                               uint64_t k, const uint64_t (&w)[NA]) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  for (uint32_t i = 0; i < p.max_probe; ++i) {
    if (k == 0) {
      k = atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek);
      if (k == 0) k = ek;
    }
    if (k == ek) {
      red_global<NA>(p.taggs + s * (uint64_t)NA, w);
      return;
    }
    s = (s + 1) & mask;
    if ((i & 31) == 31 && ld_relaxed_u32(&p.hdr->overflow)) return;  // already overflowed
    k = __ldcg((const unsigned long long*)(p.tkeys + s));
  }
  atomicOr(&p.hdr->overflow, 1u);
}

template <int NA>
__device__ __forceinline__ void global_update(const GbParams& p, uint64_t ek,
                                              const uint64_t (&w)[NA]) {
  const uint64_t s = slot_of(ek, p.log2_slots);
  global_resolve<NA>(p, ek, s, __ldcg((const unsigned long long*)(p.tkeys + s)), w);
}

template <class KT>
struct KeyPair;
template <>
struct KeyPair<int64_t> {
  using V = longlong2;
  __device__ __forceinline__ static void split(const V& v, int64_t& a, int64_t& b) {
    a = v.x;
    b = v.y;
  }
};
template <>
struct KeyPair<int32_t> {
  using V = int2;
  __device__ __forceinline__ static void split(const V& v, int64_t& a, int64_t& b) {
    a = v.x;
    b = v.y;
  }
};

template <class KT, int NA, bool PIN, bool SMT>
__global__ void __launch_bounds__(ST_BLOCK, 6) gb_stream_k(const __grid_constant__ GbParams p) {
  extern __shared__ __align__(16) uint8_t sm[];
  // [pinned keys by slot: 32 x 8 B][dense id by slot: 32 B][key by dense id:
  //  16 x 8 B][CTA sums: 16 x 4 x 8 B][thread-private words: PM x NA x
  //  ST_BLOCK x 8 B][shared table keys: S x 8 B][shared table words: S x NA x 8 B]
  constexpr int PM = pin_max<NA>();
  uint64_t* pk = (uint64_t*)sm;
  uint8_t* dense = sm + 256;
  uint64_t* pkd = (uint64_t*)(sm + 288);
  unsigned long long* csum = (unsigned long long*)(sm + 416);
  uint64_t* acc = (uint64_t*)(sm + 416 + 8 * ST_PIN_LIMIT * 4);
  uint64_t* sk = acc + (PIN ? PM * NA * ST_BLOCK : 0);
  unsigned long long* sa = (unsigned long long*)(sk + (SMT ? p.smem_slots : 0));
  const int tid = threadIdx.x;
  const uint32_t tmask = p.tiny_slots - 1;

  if (PIN) {
    if (tid < 32) {
      const uint64_t k = tid < (int)p.tiny_slots ? p.tiny_init[tid] : 0;
      pk[tid] = k;
      const unsigned occ = __ballot_sync(0xffffffffu, k != 0);
      const int d = __popc(occ & ((1u << tid) - 1u));
      dense[tid] = (uint8_t)d;
      if (k != 0 && d < PM) pkd[d] = k;
    }
    for (int i = tid; i < PM * NA * ST_BLOCK; i += ST_BLOCK) acc[i] = 0;
    for (int i = tid; i < PM * NA; i += ST_BLOCK) csum[i] = 0;
  }
  if (SMT)
    for (uint32_t i = tid; i < p.smem_slots * (1 + NA); i += ST_BLOCK) sk[i] = 0;
  __syncthreads();

  const KT* keys = (const KT*)p.col[p.key_col[0]];
  const int64_t* vals = (const int64_t*)p.col[p.r_a];
  const int64_t n = p.n_rows;
  constexpr int64_t CHUNK = (int64_t)ST_BLOCK * ST_U;
  const bool vec = ((uintptr_t)keys % (2 * sizeof(KT)) == 0) && ((uintptr_t)vals % 16 == 0);

  for (int64_t base = (int64_t)blockIdx.x * CHUNK; base < n; base += (int64_t)gridDim.x * CHUNK) {
    uint64_t ek[ST_U];
    uint64_t val[ST_U];
    bool ok[ST_U];
    // rows base + j * 2 * ST_BLOCK + 2 * tid + {0, 1}: 32 lanes cover a
    // contiguous 2 x 32-row stretch of every column per load
    if (vec && base + CHUNK <= n) {
#pragma unroll
      for (int j = 0; j < ST_U / 2; ++j) {
        const int64_t r = base + (int64_t)j * 2 * ST_BLOCK + 2 * tid;
        const typename KeyPair<KT>::V kv = __ldcs((const typename KeyPair<KT>::V*)(keys + r));
        const longlong2 vv = __ldcs((const longlong2*)(vals + r));
        int64_t k0, k1;
        KeyPair<KT>::split(kv, k0, k1);
        ek[2 * j] = (uint64_t)k0 ^ KEY_FLIP;
        ek[2 * j + 1] = (uint64_t)k1 ^ KEY_FLIP;
        val[2 * j] = (uint64_t)vv.x;
        val[2 * j + 1] = (uint64_t)vv.y;
        ok[2 * j] = ok[2 * j + 1] = true;
      }
    } else {
#pragma unroll
      for (int j = 0; j < ST_U; ++j) {
        const int64_t r = base + (int64_t)(j / 2) * 2 * ST_BLOCK + 2 * tid + (j & 1);
        ok[j] = r < n;
        ek[j] = ok[j] ? ((uint64_t)(int64_t)keys[r] ^ KEY_FLIP) : 0;
        val[j] = ok[j] ? (uint64_t)vals[r] : 0;
      }
    }
    bool need[ST_U];
#pragma unroll
    for (int j = 0; j < ST_U; ++j) {
      need[j] = false;
      if (!ok[j]) continue;
      uint64_t w[NA];
      words_of<NA>(val[j], w);
      if (PIN) {
        const uint32_t s = small_slot_of(ek[j], tmask, p.tiny_mult);
        if (pk[s] == ek[j] && ek[j] != 0) {
          uint64_t* t = acc + (size_t)dense[s] * NA * ST_BLOCK + tid;
#pragma unroll
          for (int a = 0; a < NA; ++a) {
            const uint64_t o = t[a * ST_BLOCK];
            t[a * ST_BLOCK] = umax_word<NA>(a) ? (o > w[a] ? o : w[a]) : o + w[a];
          }
          continue;
        }
      }
      if (ek[j] == 0) {  // INT64_MIN: the side accumulator
        atomicAdd(&p.hdr->n_side, 1ull);
        red_global<NA>(p.hdr->side_aggs, w);
        continue;
      }
      if (SMT) {
        uint32_t s = small_slot_of(ek[j], p.smem_slots - 1, ST_SMEM_MULT);
        bool placed = false;
        for (uint32_t i = 0; i < p.shared_probes; ++i) {
          uint64_t cur = *(volatile uint64_t*)(sk + s);
          if (cur == 0) {
            cur = atomicCAS((unsigned long long*)(sk + s), 0ull, (unsigned long long)ek[j]);
            if (cur == 0) cur = ek[j];
          }
          if (cur == ek[j]) {
            unsigned long long* t = sa + (size_t)s * NA;
#pragma unroll
            for (int a = 0; a < NA; ++a) {
              if (umax_word<NA>(a)) {  // raise only when the row improves it
                if (w[a] > *(volatile unsigned long long*)(t + a))
                  atomicMax(t + a, (unsigned long long)w[a]);
              } else {
                sadd64(t + a, w[a]);
              }
            }
            placed = true;
            break;
          }
          s = (s + 1) & (p.smem_slots - 1);
        }
        if (placed) continue;
      }
      need[j] = true;
    }
    // global table: first slot reads of every remaining row, then resolve
    uint64_t gs[ST_U], gk[ST_U];
#pragma unroll
    for (int j = 0; j < ST_U; ++j) {
      if (!need[j]) continue;
      gs[j] = slot_of(ek[j], p.log2_slots);
      gk[j] = __ldcg((const unsigned long long*)(p.tkeys + gs[j]));
    }
#pragma unroll
    for (int j = 0; j < ST_U; ++j) {
      if (!need[j]) continue;
      uint64_t w[NA];
      words_of<NA>(val[j], w);
      global_resolve<NA>(p, ek[j], gs[j], gk[j], w);
    }
  }

  // fold the thread-private words and the shared table into the global table
  if (PIN) {
    const int lane = tid & 31;
    for (int d = 0; d < PM; ++d) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        uint64_t x = acc[((size_t)d * NA + a) * ST_BLOCK + tid];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const uint64_t y = __shfl_xor_sync(0xffffffffu, x, o);
          x = umax_word<NA>(a) ? (x > y ? x : y) : x + y;
        }
        if (lane == 0 && x) {
          if (umax_word<NA>(a))
            atomicMax(csum + d * NA + a, (unsigned long long)x);
          else
            sadd64(csum + d * NA + a, x);
        }
      }
    }
  }
  __syncthreads();
  if (PIN && tid < PM && csum[tid * NA + 1] != 0) {  // word 1 counts rows
    uint64_t w[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) w[a] = csum[tid * NA + a];
    global_update<NA>(p, pkd[tid], w);
  }
  if (SMT) {
    for (uint32_t s = tid; s < p.smem_slots; s += ST_BLOCK) {
      const uint64_t k = sk[s];
      if (k == 0) continue;
      uint64_t w[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) w[a] = sa[(size_t)s * NA + a];
      global_update<NA>(p, k, w);
    }
  }
}

// Partitioned variant, passes 1 and 2, streaming: a CTA counts its rows per
// partition (pass 1); after the scan, pass 2 writes each row as a (key,
// value) record.  Pinned hot keys never become records: pass 2 aggregates
// them in thread-private words and folds them into the spill table.  INT64_MIN
// rows go to the side accumulator in pass 2.
//
// Writing every record to its own partition costs one L2 write transaction
// per 16-byte record (measured: ~3.5 ms for 1.4e8 records, at any partition
// count from 256 to 16384).  So pass 2 sorts each chunk of SP_TILE records
// by level-1 bin (at most 2^PART_L1_BITS bins of consecutive partitions) in
// shared memory, claims each bin's run with one atomic on the bin's cursor
// and writes the runs contiguously; a second pass (gb_part_l2_k) does the
// same for the partitions inside each bin.  Record order inside a partition
// is arbitrary, which the aggregation does not see.
// Two 256-thread CTAs per SM: while one waits at a barrier of its sort, the
// other streams.
constexpr int SP_BLOCK = 256;
constexpr int SP_MIN_BLOCKS = 2;
constexpr int SP_TILE = SP_BLOCK * ST_U;  // rows of one chunk, records sorted at once
constexpr int SP_BINS = 1 << PART_L1_BITS;
constexpr int SP_BAD = 15;  // wsum[SP_BAD] != 0: a claim overran its bin
static_assert(SP_BLOCK >= SP_BINS, "one thread per level-1 bin");
// shared memory of pass 2 after the pinned words: bin counts, local and
// global bases, bin ends, warp sums, then the tile's records and their bins
constexpr size_t SP_SORT_SMEM = 4 * 4 * SP_BINS + 64 + 16 * SP_TILE + SP_TILE;

template <class KT, int NA, bool PIN, bool SCATTER>
__global__ void __launch_bounds__(SP_BLOCK, SP_MIN_BLOCKS) gb_ppass_stream_k(const __grid_constant__ GbParams p) {
  extern __shared__ __align__(16) uint8_t sm[];
  constexpr int PM = pin_max<NA>();
  uint64_t* pk = (uint64_t*)sm;
  uint8_t* dense = sm + 256;
  uint64_t* pkd = (uint64_t*)(sm + 288);
  unsigned long long* csum = (unsigned long long*)(sm + 416);
  uint64_t* acc = (uint64_t*)(sm + 416 + 8 * ST_PIN_LIMIT * 4);
  uint8_t* const rest = (uint8_t*)(acc + ((PIN && SCATTER) ? PM * NA * SP_BLOCK : 0));
  unsigned int* ctr = (unsigned int*)rest;  // pass 1: [P] counts
  // pass 2
  unsigned int* cnt1 = (unsigned int*)rest;
  unsigned int* lb = cnt1 + SP_BINS;
  unsigned int* gb1 = lb + SP_BINS;
  unsigned int* end1 = gb1 + SP_BINS;
  unsigned int* wsum = end1 + SP_BINS;
  PartRec* recbuf = (PartRec*)(wsum + 16);
  uint8_t* slot_bin = (uint8_t*)(recbuf + SP_TILE);
  const int tid = threadIdx.x;
  const uint32_t P = 1u << p.part_bits;
  const uint32_t shift1 = p.part_bits > PART_L1_BITS ? p.part_bits - PART_L1_BITS : 0;
  const uint32_t B1 = P >> shift1;  // level-1 bins
  PartRec* const out1 = shift1 ? p.recs1 : p.recs;
  const uint32_t tmask = p.tiny_slots - 1;
  if (PIN) {
    if (tid < 32) {
      const uint64_t k = tid < (int)p.tiny_slots ? p.tiny_init[tid] : 0;
      pk[tid] = k;
      const unsigned occ = __ballot_sync(0xffffffffu, k != 0);
      const int d = __popc(occ & ((1u << tid) - 1u));
      dense[tid] = (uint8_t)d;
      if (k != 0 && d < PM) pkd[d] = k;
    }
    if (SCATTER) {
      for (int i = tid; i < PM * NA * SP_BLOCK; i += SP_BLOCK) acc[i] = 0;
      for (int i = tid; i < PM * NA; i += SP_BLOCK) csum[i] = 0;
    }
  }
  if (!SCATTER) {
    for (uint32_t i = tid; i < P; i += SP_BLOCK) ctr[i] = 0;
  } else {
    if (tid < (int)B1) {
      cnt1[tid] = 0;
      end1[tid] = (unsigned int)p.part_start[(tid + 1) << shift1];
    }
    if (tid == 0) wsum[SP_BAD] = 0;
  }
  const int lane = tid & 31, warp = tid >> 5;
  __syncthreads();

  const KT* keys = (const KT*)p.col[p.key_col[0]];
  const int64_t* vals = (const int64_t*)p.col[p.r_a];
  const int64_t n = p.n_rows;
  constexpr int64_t CHUNK = (int64_t)SP_BLOCK * ST_U;
  const bool vec = ((uintptr_t)keys % (2 * sizeof(KT)) == 0) && ((uintptr_t)vals % 16 == 0);
  // rows base + j * 2 * SP_BLOCK + 2 * tid + {0, 1}; the next chunk's loads
  // go out before this chunk is worked on (the pass is bound by load latency)
  auto load = [&](int64_t base, uint64_t(&ek)[ST_U], uint64_t(&val)[ST_U], uint32_t& ok) {
    if (vec && base + CHUNK <= n) {
#pragma unroll
      for (int j = 0; j < ST_U / 2; ++j) {
        const int64_t r = base + (int64_t)j * 2 * SP_BLOCK + 2 * tid;
        int64_t k0, k1;
        KeyPair<KT>::split(__ldcs((const typename KeyPair<KT>::V*)(keys + r)), k0, k1);
        ek[2 * j] = (uint64_t)k0 ^ KEY_FLIP;
        ek[2 * j + 1] = (uint64_t)k1 ^ KEY_FLIP;
        if (SCATTER) {
          const longlong2 vv = __ldcs((const longlong2*)(vals + r));
          val[2 * j] = (uint64_t)vv.x;
          val[2 * j + 1] = (uint64_t)vv.y;
        }
      }
      ok = (1u << ST_U) - 1;
      return;
    }
    ok = 0;
#pragma unroll
    for (int j = 0; j < ST_U; ++j) {
      const int64_t r = base + (int64_t)(j / 2) * 2 * SP_BLOCK + 2 * tid + (j & 1);
      const bool in = r < n;
      ek[j] = in ? ((uint64_t)(int64_t)keys[r] ^ KEY_FLIP) : 0;
      if (SCATTER) val[j] = in ? (uint64_t)vals[r] : 0;
      ok |= (in ? 1u : 0u) << j;
    }
  };
  const int64_t step = (int64_t)gridDim.x * CHUNK;
  uint64_t ek[ST_U], val[ST_U];
  uint32_t okm = 0;
  if ((int64_t)blockIdx.x * CHUNK < n) load((int64_t)blockIdx.x * CHUNK, ek, val, okm);
  for (int64_t base = (int64_t)blockIdx.x * CHUNK; base < n; base += step) {
    uint64_t nek[ST_U], nval[ST_U];
    uint32_t nok = 0;
    if (base + step < n) load(base + step, nek, nval, nok);
    // The chunk's rows go through the steps below together, each step's
    // shared-memory lookups and atomics for all ST_U rows in flight at once
    // (one chain per row would leave the SM waiting on their latency).
    // pinned key? (thread-private accumulation)
    uint32_t pinm = 0;
    if (PIN) {
      uint32_t sl[ST_U];
      uint64_t pv[ST_U];
#pragma unroll
      for (int j = 0; j < ST_U; ++j) {
        sl[j] = small_slot_of(ek[j], tmask, p.tiny_mult);
        pv[j] = pk[sl[j]];
      }
#pragma unroll
      for (int j = 0; j < ST_U; ++j)
        pinm |= ((okm >> j & 1) && pv[j] == ek[j] && ek[j] != 0 ? 1u : 0u) << j;
      if (SCATTER && pinm) {
        uint32_t dd[ST_U];
#pragma unroll
        for (int j = 0; j < ST_U; ++j) dd[j] = dense[sl[j]];
#pragma unroll
        for (int j = 0; j < ST_U; ++j) {
          if (!(pinm >> j & 1)) continue;
          uint64_t w[NA];
          words_of<NA>(val[j], w);
          uint64_t* t = acc + (size_t)dd[j] * NA * SP_BLOCK + tid;
#pragma unroll
          for (int a = 0; a < NA; ++a) {
            const uint64_t o = t[a * SP_BLOCK];
            t[a * SP_BLOCK] = umax_word<NA>(a) ? (o > w[a] ? o : w[a]) : o + w[a];
          }
        }
      }
    }
    // INT64_MIN rows (stored key 0): the side accumulator
    uint32_t sidem = 0;
#pragma unroll
    for (int j = 0; j < ST_U; ++j) sidem |= ((okm >> j & 1) && ek[j] == 0 ? 1u : 0u) << j;
    sidem &= ~pinm;
    if (SCATTER && sidem) {
#pragma unroll
      for (int j = 0; j < ST_U; ++j) {
        if (!(sidem >> j & 1)) continue;
        uint64_t w[NA];
        words_of<NA>(val[j], w);
        atomicAdd(&p.hdr->n_side, 1ull);
        red_global<NA>(p.hdr->side_aggs, w);
      }
    }
    // every other row is a record of its partition
    const uint32_t recm = okm & ~pinm & ~sidem;
    uint32_t part[ST_U];
#pragma unroll
    for (int j = 0; j < ST_U; ++j) part[j] = part_of(ek[j], p.part_bits);
    if (!SCATTER) {
#pragma unroll
      for (int j = 0; j < ST_U; ++j)
        if (recm >> j & 1) atomicAdd(&ctr[part[j]], 1u);
    } else {
      // sort the chunk's records by level-1 bin: ranks within the bins ...
      uint32_t rank[ST_U];
#pragma unroll
      for (int j = 0; j < ST_U; ++j)
        if (recm >> j & 1) rank[j] = atomicAdd(&cnt1[part[j] >> shift1], 1u);
      __syncthreads();
      // ... the bins' local bases (exclusive scan over threads 0..B1-1), one
      // global claim per non-empty bin, and the counts cleared for the next
      // chunk (every thread has read its count by the barrier before) ...
      const uint32_t c = tid < (int)B1 ? cnt1[tid] : 0u;
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31 && warp < SP_BINS / 32) wsum[warp] = incl;
      __syncthreads();
      uint32_t nrec = 0, before = 0;
#pragma unroll
      for (int w = 0; w < SP_BINS / 32; ++w) {
        before += w < warp ? wsum[w] : 0u;
        nrec += wsum[w];
      }
      if (tid < (int)B1) {
        lb[tid] = before + incl - c;
        // output position of local slot i of this bin: i + delta (mod 2^32);
        // a claim past the bin's end (the passes disagreed) voids the call and
        // stops this CTA's writes
        if (c) {
          const uint32_t g = atomicAdd(p.cursor1 + tid, c);
          if (g + c > end1[tid]) {
            atomicOr(&p.hdr->timeout, 2u);
            wsum[SP_BAD] = 1;
          }
          gb1[tid] = g - (before + incl - c);
        }
        cnt1[tid] = 0;
      }
      __syncthreads();
      // ... the records into place in shared memory ...
#pragma unroll
      for (int j = 0; j < ST_U; ++j) {
        if (!(recm >> j & 1)) continue;
        const uint32_t b = part[j] >> shift1;
        const uint32_t sl = lb[b] + rank[j];
        PartRec r;
        r.ek = ek[j];
        r.val = (long long)val[j];
        recbuf[sl] = r;
        slot_bin[sl] = (uint8_t)b;
      }
      __syncthreads();
      // ... and out: consecutive threads write consecutive records of a run.
      // No barrier after: the next chunk touches only the cleared counts
      // before its first barrier, which every thread reaches after this.
      if (!wsum[SP_BAD])  // uniform: never past a bin
        for (uint32_t i = tid; i < nrec; i += SP_BLOCK) out1[i + gb1[slot_bin[i]]] = recbuf[i];
    }
#pragma unroll
    for (int j = 0; j < ST_U; ++j) {
      ek[j] = nek[j];
      if (SCATTER) val[j] = nval[j];
    }
    okm = nok;
  }
  __syncthreads();
  if (!SCATTER) {
    for (uint32_t i = tid; i < P; i += SP_BLOCK) p.hist[(size_t)i * p.fixed_grid + blockIdx.x] = ctr[i];
    return;
  }
  if (PIN) {
    for (int d = 0; d < PM; ++d) {
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        uint64_t x = acc[((size_t)d * NA + a) * SP_BLOCK + tid];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const uint64_t y = __shfl_xor_sync(0xffffffffu, x, o);
          x = umax_word<NA>(a) ? (x > y ? x : y) : x + y;
        }
        if (lane == 0 && x) {
          if (umax_word<NA>(a))
            atomicMax(csum + d * NA + a, (unsigned long long)x);
          else
            sadd64(csum + d * NA + a, x);
        }
      }
    }
    __syncthreads();
    if (tid < PM && csum[tid * NA + 1] != 0) {
      uint64_t w[NA];
#pragma unroll
      for (int a = 0; a < NA; ++a) w[a] = csum[tid * NA + a];
      global_update<NA>(p, pkd[tid], w);
    }
  }
}

size_t ppass_smem(int na, bool pin, bool scatter, uint32_t part_bits) {
  size_t b = 416 + 8 * ST_PIN_LIMIT * 4;
  if (pin && scatter) b += (size_t)8 * (na == 4 ? pin_max<4>() : pin_max<2>()) * na * SP_BLOCK;
  return b + (scatter ? SP_SORT_SMEM : 4ull * (1u << part_bits));
}

// CTAs of a pass that fit on the SMs at once (at most cap), or 0.
template <class KT, int NA, bool PIN, bool SCATTER>
uint32_t ppass_grid(const GbParams& p, uint32_t cap) {
  auto kern = gb_ppass_stream_k<KT, NA, PIN, SCATTER>;
  const size_t smem = ppass_smem(NA, PIN, SCATTER, p.part_bits);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SP_BLOCK, smem) != cudaSuccess)
    return 0;
  const uint32_t g = (uint32_t)relhost::device_sms() * (uint32_t)(occ > 0 ? occ : 0);
  return g < cap ? g : cap;
}

// The histogram pass runs p.fixed_grid CTAs (its counts are laid out per
// CTA); the scatter pass, whose positions come from the bins' cursors, runs
// as many CTAs as fit.
template <class KT, int NA, bool PIN, bool SCATTER>
rel_status launch_ppass(const GbParams& p, cudaStream_t st) {
  auto kern = gb_ppass_stream_k<KT, NA, PIN, SCATTER>;
  const size_t smem = ppass_smem(NA, PIN, SCATTER, p.part_bits);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaFuncSetAttribute(partition pass)");
  const uint32_t grid = SCATTER ? ppass_grid<KT, NA, PIN, SCATTER>(p, 1u << 16) : p.fixed_grid;
  if (grid < 1) return relhost::set_error("group-by: partition pass does not fit"), REL_E_UNSUPPORTED;
  const int id = SCATTER ? relhost::K_GB_PSCATTER : relhost::K_GB_PHIST;
  relhost::launch_begin(id, st);
  kern<<<grid, SP_BLOCK, smem, st>>>(p);
  relhost::launch_end(id, st);
  e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(partition pass)");
}

template <class KT, int NA>
rel_status ppass_dispatch(const GbParams& p, bool scatter, cudaStream_t st) {
  const bool pin = p.tiny_frozen && p.tiny_slots;
  if (pin)
    return scatter ? launch_ppass<KT, NA, true, true>(p, st) : launch_ppass<KT, NA, true, false>(p, st);
  return scatter ? launch_ppass<KT, NA, false, true>(p, st) : launch_ppass<KT, NA, false, false>(p, st);
}

size_t stream_smem(int na, bool pin, bool smt, uint32_t smem_slots) {
  size_t b = 416 + 8 * ST_PIN_LIMIT * 4;
  if (pin) b += (size_t)8 * (na == 4 ? pin_max<4>() : pin_max<2>()) * na * ST_BLOCK;
  if (smt) b += (size_t)8 * smem_slots * (1 + na);
  return b;
}

template <class KT, int NA, bool PIN, bool SMT>
rel_status launch_stream(const GbParams& p, cudaStream_t st) {
  auto kern = gb_stream_k<KT, NA, PIN, SMT>;
  const size_t smem = stream_smem(NA, PIN, SMT, p.smem_slots);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaFuncSetAttribute(stream)");
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, ST_BLOCK, smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "occupancy(stream)");
  if (occ < 1) return relhost::set_error("group-by: stream kernel does not fit"), REL_E_UNSUPPORTED;
  const int64_t chunks = (p.n_rows + (int64_t)ST_BLOCK * ST_U - 1) / ((int64_t)ST_BLOCK * ST_U);
  int64_t grid = (int64_t)relhost::device_sms() * occ;
  if (grid > chunks) grid = chunks;
  if (grid < 1) grid = 1;
  relhost::launch_begin(relhost::K_GB_STREAM, st);
  kern<<<(int)grid, ST_BLOCK, smem, st>>>(p);
  relhost::launch_end(relhost::K_GB_STREAM, st);
  e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(stream)");
}

template <class KT, int NA>
rel_status dispatch_layers(const GbParams& p, cudaStream_t st) {
  const bool pin = p.tiny_frozen && p.tiny_slots;
  const bool smt = p.smem_slots != 0;
  if (pin && smt) return launch_stream<KT, NA, true, true>(p, st);
  if (pin) return launch_stream<KT, NA, true, false>(p, st);
  if (smt) return launch_stream<KT, NA, false, true>(p, st);
  return launch_stream<KT, NA, false, false>(p, st);
}

}  // namespace

bool gb_stream_eligible(const GbParams& p, int shape, int n_hot) {
  const bool kv = shape == SHAPE_KV4_64 || shape == SHAPE_KV4_32 || shape == SHAPE_KV2_64 ||
                  shape == SHAPE_KV2_32;
  if (!kv) return false;
  // thread-private slots only when pinned (a first-come thread-private
  // table is the fused kernel's job)
  const int na = (shape == SHAPE_KV4_64 || shape == SHAPE_KV4_32) ? 4 : 2;
  const bool pin = p.tiny_slots != 0;
  const int pmax = na == 4 ? pin_max<4>() : pin_max<2>();
  if (pin && !(p.tiny_frozen && p.tiny_slots <= 32 && n_hot <= pmax)) return false;
  // a large shared table would leave too few resident threads for the
  // global probes' latency: that case stays with the fused kernel
  return stream_smem(na, pin, p.smem_slots != 0, p.smem_slots) <= 80 * 1024;
}

// Level 2 of the streaming scatter: every tile of PART_TILE level-1 records
// (tiles never straddle a bin) is sorted by partition inside its bin in
// shared memory; each partition's run is claimed with one atomic on the
// partition's cursor and written contiguously.  Persistent grid; tile t
// belongs to the last bin b with l2_tiles[b] <= t.
constexpr int L2_BLOCK = 512;
constexpr int L2_U = PART_TILE / L2_BLOCK;
constexpr int L2_MAX_SUB = 1 << (PART_MAX_BITS - PART_L1_BITS);
constexpr size_t L2_SMEM = 16 * PART_TILE + PART_TILE;

__global__ void __launch_bounds__(L2_BLOCK, 2) gb_part_l2_k(const __grid_constant__ GbParams p) {
  extern __shared__ __align__(16) uint8_t sm[];
  PartRec* recbuf = (PartRec*)sm;
  uint8_t* slot_bin = sm + 16 * PART_TILE;
  __shared__ unsigned int tp[SP_BINS + 1];
  __shared__ unsigned int cnt[L2_MAX_SUB], lb[L2_MAX_SUB], gb[L2_MAX_SUB];
  __shared__ int bad;  // a claim overran its partition: this CTA writes no more
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t shift1 = p.part_bits - PART_L1_BITS;  // > 0: launched only then
  const uint32_t B1 = 1u << PART_L1_BITS;
  const uint32_t B2 = 1u << shift1;
  for (uint32_t i = tid; i <= B1; i += L2_BLOCK) tp[i] = p.l2_tiles[i];
  if (tid < (int)B2) cnt[tid] = 0;
  if (tid == 0) bad = 0;
  __syncthreads();
  const uint32_t T = tp[B1];
  for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
    uint32_t lo = 0, hi = B1;  // tp[lo] <= t < tp[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (tp[mid] <= t) lo = mid; else hi = mid;
    }
    const uint32_t first = lo << shift1;  // first partition of the bin
    const unsigned long long s1 = p.part_start[first];
    const unsigned long long e1 = p.part_start[first + B2];
    const unsigned long long t0 = s1 + (unsigned long long)(t - tp[lo]) * PART_TILE;
    const unsigned long long t1 = t0 + PART_TILE < e1 ? t0 + PART_TILE : e1;
    PartRec r[L2_U];
    uint32_t sr[L2_U];  // partition within the bin | rank within it << 8
#pragma unroll
    for (int u = 0; u < L2_U; ++u) {
      const unsigned long long i = t0 + (unsigned long long)u * L2_BLOCK + tid;
      sr[u] = 0;
      if (i < t1) {
        const longlong2 v = __ldcs((const longlong2*)(p.recs1 + i));
        r[u].ek = (unsigned long long)v.x;
        r[u].val = v.y;
        sr[u] = part_of((uint64_t)v.x, p.part_bits) & (B2 - 1);
      }
    }
#pragma unroll
    for (int u = 0; u < L2_U; ++u)
      if (t0 + (unsigned long long)u * L2_BLOCK + tid < t1) sr[u] |= atomicAdd(&cnt[sr[u]], 1u) << 8;
    __syncthreads();
    // warp 0: local bases, one claim per non-empty partition, partition ends,
    // counts cleared for the next tile
    if (warp == 0) {
      constexpr int PER = L2_MAX_SUB / 32;
      uint32_t cb[PER], sum = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const uint32_t bn = lane * PER + k;
        cb[k] = bn < B2 ? cnt[bn] : 0u;
        sum += cb[k];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t run = incl - sum;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const uint32_t bn = lane * PER + k;
        if (bn < B2) {
          lb[bn] = run;
          if (cb[k]) {  // position of local slot i: i + delta (see the level-1 pass)
            const uint32_t g = atomicAdd(p.cursor + first + bn, cb[k]);
            if (g + cb[k] > (uint32_t)p.part_start[first + bn + 1]) {
              atomicOr(&p.hdr->timeout, 2u);
              bad = 1;
            }
            gb[bn] = g - run;
          }
          cnt[bn] = 0;
        }
        run += cb[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < L2_U; ++u) {
      if (t0 + (unsigned long long)u * L2_BLOCK + tid >= t1) continue;
      const uint32_t sub = sr[u] & 0xFFu;
      const uint32_t sl = lb[sub] + (sr[u] >> 8);
      recbuf[sl] = r[u];
      slot_bin[sl] = (uint8_t)sub;
    }
    __syncthreads();
    // no barrier after the writes: the next tile touches only the cleared
    // counts before its first barrier
    const uint32_t nrec = (uint32_t)(t1 - t0);
    if (!bad)  // uniform: never past a partition
      for (uint32_t i = tid; i < nrec; i += L2_BLOCK) p.recs[i + gb[slot_bin[i]]] = recbuf[i];
  }
}

rel_status gb_launch_part_l2(const GbParams& p, cudaStream_t st) {
  if (p.part_bits <= PART_L1_BITS || p.part_bits > PART_MAX_BITS || !p.recs1)
    return relhost::set_error("group-by: level-2 scatter needs more than 2^%d partitions", PART_L1_BITS),
           REL_E_INVALID;
  cudaError_t e = cudaFuncSetAttribute(gb_part_l2_k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L2_SMEM);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaFuncSetAttribute(level-2 scatter)");
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gb_part_l2_k, L2_BLOCK, L2_SMEM);
  if (e != cudaSuccess || occ < 1) return relhost::cuda_fail(e, "occupancy(level-2 scatter)");
  const int grid = relhost::device_sms() * occ;
  relhost::launch_begin(relhost::K_GB_PL2, st);
  gb_part_l2_k<<<grid, L2_BLOCK, L2_SMEM, st>>>(p);
  relhost::launch_end(relhost::K_GB_PL2, st);
  e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(level-2 scatter)");
}

uint32_t gb_ppass_stream_grid(const GbParams& p, int shape, uint32_t cap) {
  const bool pin = p.tiny_frozen && p.tiny_slots;
  switch (shape) {
    case SHAPE_KV4_64:
      return pin ? ppass_grid<int64_t, 4, true, false>(p, cap) : ppass_grid<int64_t, 4, false, false>(p, cap);
    case SHAPE_KV4_32:
      return pin ? ppass_grid<int32_t, 4, true, false>(p, cap) : ppass_grid<int32_t, 4, false, false>(p, cap);
    case SHAPE_KV2_64:
      return pin ? ppass_grid<int64_t, 2, true, false>(p, cap) : ppass_grid<int64_t, 2, false, false>(p, cap);
    case SHAPE_KV2_32:
      return pin ? ppass_grid<int32_t, 2, true, false>(p, cap) : ppass_grid<int32_t, 2, false, false>(p, cap);
    default: return 0;
  }
}

bool gb_ppass_stream_eligible(const GbParams& p, int shape, int n_hot) {
  const bool kv = shape == SHAPE_KV4_64 || shape == SHAPE_KV4_32 || shape == SHAPE_KV2_64 ||
                  shape == SHAPE_KV2_32;
  if (!kv || p.fixed_grid < 1) return false;
  const int na = (shape == SHAPE_KV4_64 || shape == SHAPE_KV4_32) ? 4 : 2;
  const int pmax = na == 4 ? pin_max<4>() : pin_max<2>();
  if (p.tiny_slots && !(p.tiny_frozen && p.tiny_slots <= 32 && n_hot <= pmax)) return false;
  return ppass_smem(na, p.tiny_slots != 0, true, p.part_bits) * SP_MIN_BLOCKS <= 227 * 1024 &&
         ppass_smem(na, p.tiny_slots != 0, false, p.part_bits) * SP_MIN_BLOCKS <= 227 * 1024;
}

rel_status gb_launch_ppass_stream(const GbParams& p, int shape, bool scatter, cudaStream_t st) {
  switch (shape) {
    case SHAPE_KV4_64: return ppass_dispatch<int64_t, 4>(p, scatter, st);
    case SHAPE_KV4_32: return ppass_dispatch<int32_t, 4>(p, scatter, st);
    case SHAPE_KV2_64: return ppass_dispatch<int64_t, 2>(p, scatter, st);
    case SHAPE_KV2_32: return ppass_dispatch<int32_t, 2>(p, scatter, st);
  }
  relhost::set_error("group-by: partition pass needs a key/value shape");
  return REL_E_INVALID;
}

rel_status gb_launch_stream(const GbParams& p, int shape, cudaStream_t st) {
  if (p.n_rows == 0) return REL_OK;
  switch (shape) {
    case SHAPE_KV4_64: return dispatch_layers<int64_t, 4>(p, st);
    case SHAPE_KV4_32: return dispatch_layers<int32_t, 4>(p, st);
    case SHAPE_KV2_64: return dispatch_layers<int64_t, 2>(p, st);
    case SHAPE_KV2_32: return dispatch_layers<int32_t, 2>(p, st);
  }
  relhost::set_error("group-by: stream kernel needs a key/value shape");
  return REL_E_INVALID;
}

}  // namespace rel
