// Fused filter + hash group-by kernels for sm_103a.
//
// One persistent launch streams every column of the query through shared
// memory with the TMA bulk-copy engine (a ring of 2-4 stages completed on
// mbarriers), evaluates the range filter, the packed group key and the
// product-form aggregate inputs in registers -- no expression interpreter and
// no materialised mask, the instruction overheads the paper attributes to
// compute_column_kernel and transform_kernel (Sec. 7) -- and folds each row
// into a stack of tables, first one that holds the key wins:
//   1. thread-private: up to 32 keys per CTA, each thread owning private
//      accumulator columns in shared memory -- no atomics, so the hottest
//      keys of a skewed input never serialise;
//   2. CTA-shared: an open-addressing table in shared memory updated with
//      shared-memory atomics (the privatised aggregation of
//      single_pass_shmem_aggs_kernel, Sec. 7);
//   3. global: one open-addressing table in device memory (CAS claim, then
//      fire-and-forget RED atomics).
// Rows a per-CTA table cannot hold fall through to the next layer, and both
// per-CTA tables merge into the global one at the end, so every layer
// configuration yields the same exact groups.  A compaction kernel turns
// occupied slots into dense output rows (warp ballot / popc, one atomic per
// warp).  MODE_KEYSET counts distinct keys instead (the exact sizing pass).
#include "groupby.cuh"

namespace rel {

// ------------------------------------------------------------- row access

struct SmemView {
  const uint8_t* base;  // one pipeline stage
  __device__ __forceinline__ int64_t get(const GbParams& p, int c, int r) const {
    const uint8_t* q = base + p.stage_off[c];
    switch (p.ctype[c]) {
      case REL_U8: return (int64_t)q[r];
      case REL_I32: return (int64_t)((const int32_t*)q)[r];
      default: return ((const int64_t*)q)[r];
    }
  }
  template <class T>
  __device__ __forceinline__ const T* ptr(const GbParams& p, int c) const {
    return (const T*)(base + p.stage_off[c]);
  }
};

struct GlobalView {
  int64_t row0;
  __device__ __forceinline__ int64_t get(const GbParams& p, int c, int r) const {
    const int64_t i = row0 + r;
    switch (p.ctype[c]) {
      case REL_U8: return (int64_t)__ldg(p.col[c] + i);
      case REL_I32: return (int64_t)__ldg((const int32_t*)p.col[c] + i);
      default: return (int64_t)__ldg((const long long*)p.col[c] + i);
    }
  }
  template <class T>
  __device__ __forceinline__ const T* ptr(const GbParams& p, int c) const {
    return (const T*)p.col[c] + row0;
  }
};

template <int A>
struct Vals {
  uint64_t v[A];
};

// ------------------------------------------------------------- row shapes
// prep(): per-tile column pointers (hoisted out of the row loop).
// row(): false when the filter rejects the row; else the stored key
// ek = key ^ KEY_FLIP and the encoded aggregate words x.v[0..A).

// Any descriptor within the REL_MAX_* limits, read from the kernel params.
struct ShapeGeneric {
  static constexpr int A = REL_MAX_AGGS;
  static constexpr bool RT = true;  // aggregate kinds known only at run time
  static constexpr uint32_t UMAX = 0;
  template <class V>
  __device__ __forceinline__ static V prep(const GbParams&, const V& v) {
    return v;
  }
  template <class V>
  __device__ __forceinline__ static bool row(const GbParams& p, const V& v, int r, uint64_t& ek,
                                             Vals<A>& x) {
#pragma unroll
    for (int i = 0; i < REL_MAX_PREDS; ++i) {
      if (i < p.n_preds) {
        const int64_t d = v.get(p, p.pred_col[i], r);
        if (d < p.pred_lo[i] || d > p.pred_hi[i]) return false;
      }
    }
    uint64_t key;
    if (p.n_keys == 1) {
      key = (uint64_t)v.get(p, p.key_col[0], r);
    } else {
      key = 0;
#pragma unroll
      for (int i = 0; i < REL_MAX_KEYS; ++i)
        if (i < p.n_keys)
          key |= ((uint64_t)v.get(p, p.key_col[i], r) & p.key_mask[i]) << p.key_shift[i];
    }
    ek = key ^ KEY_FLIP;
#pragma unroll
    for (int a = 0; a < A; ++a) {
      if (a < p.n_aggs) {
        const int op = p.aop[a];
        if (op == REL_COUNT) {
          x.v[a] = 1;
        } else {
          uint64_t val = (uint64_t)v.get(p, p.abase[a], r);
#pragma unroll
          for (int f = 0; f < 2; ++f)
            if (f < p.anf[a])
              val *= (uint64_t)p.ac[a][f] +
                     (uint64_t)p.as[a][f] * (uint64_t)v.get(p, p.afcol[a][f], r);
          x.v[a] = agg_encode(op, (int64_t)val);
        }
      }
    }
    return true;
  }
};

// keep lo <= pred <= hi (int32 column); key = (u8 k0 << 8) | u8 k1;
// sum(a), sum(b), sum(b*(c0 + s0*d)), sum(b*(c0 + s0*d)*(c1 + s1*t)), count.
struct ShapeQ1 {
  static constexpr int A = 5;
  static constexpr bool RT = false;
  static constexpr uint32_t UMAX = 0;
  struct Tile {
    const int32_t* pred;
    const uint8_t *k0, *k1;
    const int64_t *a, *b, *d, *t;
    int64_t lo, hi;
    uint64_t c0, s0, c1, s1;
  };
  template <class V>
  __device__ __forceinline__ static Tile prep(const GbParams& p, const V& v) {
    return Tile{v.template ptr<int32_t>(p, p.r_pred), v.template ptr<uint8_t>(p, p.r_k0),
                v.template ptr<uint8_t>(p, p.r_k1),   v.template ptr<int64_t>(p, p.r_a),
                v.template ptr<int64_t>(p, p.r_b),    v.template ptr<int64_t>(p, p.r_d),
                v.template ptr<int64_t>(p, p.r_t),    p.pred_lo[0],
                p.pred_hi[0],                         (uint64_t)p.ac[2][0],
                (uint64_t)p.as[2][0],                 (uint64_t)p.ac[3][1],
                (uint64_t)p.as[3][1]};
  }
  __device__ __forceinline__ static bool row(const GbParams&, const Tile& q, int r, uint64_t& ek,
                                             Vals<A>& x) {
    const int64_t d = (int64_t)q.pred[r];
    if (d < q.lo || d > q.hi) return false;
    const uint64_t k0 = q.k0[r];
    const uint64_t k1 = q.k1[r];
    ek = ((k0 << 8) | k1) ^ KEY_FLIP;
    const uint64_t qa = (uint64_t)q.a[r];
    const uint64_t pb = (uint64_t)q.b[r];
    const uint64_t dd = (uint64_t)q.d[r];
    const uint64_t tt = (uint64_t)q.t[r];
    const uint64_t f0 = q.c0 + q.s0 * dd;
    const uint64_t f1 = q.c1 + q.s1 * tt;
    const uint64_t dp = pb * f0;
    x.v[0] = qa;
    x.v[1] = pb;
    x.v[2] = dp;
    x.v[3] = dp * f1;
    x.v[4] = 1;
    return true;
  }
};

// key column (int64 / int32) + one int64 value column, runtime ops, no filter.
template <class KT>
struct ShapeKVRT {
  static constexpr int A = 4;
  static constexpr bool RT = true;
  static constexpr uint32_t UMAX = 0;
  struct Tile {
    const KT* k;
    const int64_t* v;
  };
  template <class V>
  __device__ __forceinline__ static Tile prep(const GbParams& p, const V& v) {
    return Tile{v.template ptr<KT>(p, p.key_col[0]), v.template ptr<int64_t>(p, p.r_a)};
  }
  __device__ __forceinline__ static bool row(const GbParams& p, const Tile& q, int r, uint64_t& ek,
                                             Vals<A>& x) {
    const int64_t key = (int64_t)q.k[r];
    const int64_t val = q.v[r];
    ek = (uint64_t)key ^ KEY_FLIP;
#pragma unroll
    for (int a = 0; a < A; ++a)
      if (a < p.n_aggs) x.v[a] = agg_encode(p.aop[a], val);
    return true;
  }
};

// key + int64 value; NA = 4: (sum, count, min, max), NA = 2: (sum, count).
template <class KT, int NA>
struct ShapeKV {
  static constexpr int A = NA;
  static constexpr bool RT = false;
  static constexpr uint32_t UMAX = NA == 4 ? 0xCu : 0u;
  struct Tile {
    const KT* k;
    const int64_t* v;
  };
  template <class V>
  __device__ __forceinline__ static Tile prep(const GbParams& p, const V& v) {
    return Tile{v.template ptr<KT>(p, p.key_col[0]), v.template ptr<int64_t>(p, p.r_a)};
  }
  __device__ __forceinline__ static bool row(const GbParams&, const Tile& q, int r, uint64_t& ek,
                                             Vals<A>& x) {
    const int64_t key = (int64_t)q.k[r];
    const uint64_t val = (uint64_t)q.v[r];
    ek = (uint64_t)key ^ KEY_FLIP;
    from_val(val, x);
    return true;
  }
  // the aggregate words of a row with value val
  __device__ __forceinline__ static void from_val(uint64_t val, Vals<A>& x) {
    x.v[0] = val;
    x.v[1] = 1;
    if constexpr (NA == 4) {
      x.v[2] = val ^ MIN_FLIP;
      x.v[3] = val ^ MAX_FLIP;
    }
  }
};

template <class S>
__device__ __forceinline__ bool is_umax(const GbParams& p, int a) {
  if constexpr (S::RT)
    return (p.umax_mask >> a) & 1u;
  else
    return (S::UMAX >> a) & 1u;
}

template <class S>
__device__ __forceinline__ bool live_agg(const GbParams& p, int a) {
  if constexpr (S::RT)
    return a < p.n_aggs;
  else
    return true;
}

// -------------------------------------------------------------- table ops

template <class S>
__device__ __forceinline__ void red_words(const GbParams& p, unsigned long long* w,
                                          const Vals<S::A>& x) {
#pragma unroll
  for (int a = 0; a < S::A; ++a) {
    if (live_agg<S>(p, a)) {
      if (is_umax<S>(p, a))
        atomicMax(w + a, (unsigned long long)x.v[a]);
      else
        atomicAdd(w + a, (unsigned long long)x.v[a]);
    }
  }
}

// Shared-memory words: a MIN / MAX word is read first and only raised by an
// atomic when the row improves it -- under skew most rows of a hot key do not,
// so most of those atomics (and their serialisation on one address) vanish.
template <class S, bool COUNT32 = false>
__device__ __forceinline__ void red_words_smem(const GbParams& p, unsigned long long* w,
                                               const Vals<S::A>& x) {
  if constexpr (COUNT32 && !S::RT && S::A == 4) {
    // (sum, count, min, max) of a 32-byte slot: the MIN / MAX pair is read
    // with one 16-byte load (w is 32-byte aligned)
    sadd64(w, x.v[0]);
    atomicAdd((unsigned int*)(w + 1), (unsigned int)x.v[1]);
    unsigned long long mn, mx;
    asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];"
                 : "=l"(mn), "=l"(mx)
                 : "r"(smem_u32(w + 2)));
    if ((unsigned long long)x.v[2] > mn) atomicMax(w + 2, (unsigned long long)x.v[2]);
    if ((unsigned long long)x.v[3] > mx) atomicMax(w + 3, (unsigned long long)x.v[3]);
  } else {
#pragma unroll
    for (int a = 0; a < S::A; ++a) {
      if (live_agg<S>(p, a)) {
        if (COUNT32 && a == 1) {
          // key/value shapes: word 1 counts rows; below 2^32 rows per table
          // (a partitioned input has fewer) a 32-bit add on its low half is exact
          atomicAdd((unsigned int*)(w + 1), (unsigned int)x.v[1]);
        } else if (is_umax<S>(p, a)) {
          if ((unsigned long long)x.v[a] > *(volatile unsigned long long*)(w + a))
            atomicMax(w + a, (unsigned long long)x.v[a]);
        } else {
          sadd64(w + a, x.v[a]);
        }
      }
    }
  }
}

// Insert-or-accumulate into the global table; bounded linear probing.
template <class S>
__device__ __forceinline__ bool gtab_update_inl(const GbParams& p, uint64_t ek,
                                                const Vals<S::A>& x) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  uint64_t s = slot_of(ek, p.log2_slots);
  for (uint32_t i = 0; i < p.max_probe; ++i) {
    uint64_t k = ld_relaxed(p.tkeys + s);
    if (k == 0) {
      k = atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek);
      if (k == 0) k = ek;
    }
    if (k == ek) {
      red_words<S>(p, p.taggs + s * (uint64_t)p.n_aggs, x);
      return true;
    }
    s = (s + 1) & mask;
    // a long probe sequence: give up at once if the table already overflowed
    // (the result is then discarded; this bounds the cost of an undersized plan)
    if ((i & 31) == 31 && ld_relaxed_u32(&p.hdr->overflow)) return false;
  }
  atomicOr(&p.hdr->overflow, 1u);
  return false;
}

// Kept inline on every path: an out-of-line call taking the words by
// reference makes the compiler keep them in local memory on every row.
template <class S>
__device__ __forceinline__ bool gtab_update(const GbParams& p, uint64_t ek, const Vals<S::A>& x) {
  return gtab_update_inl<S>(p, ek, x);
}

// Key set for the exact distinct count; false when the set overflowed.
__device__ __noinline__ bool gset_insert(const GbParams& p, uint64_t ek) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  uint64_t s = slot_of(ek, p.log2_slots);
  for (uint32_t i = 0; i < p.max_probe; ++i) {
    uint64_t k = ld_relaxed(p.tkeys + s);
    if (k == ek) return true;
    if (k == 0) {
      k = atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek);
      if (k == 0) {
        atomicAdd(&p.hdr->aux, 1ull);
        return true;
      }
      if (k == ek) return true;
    }
    s = (s + 1) & mask;
    if ((i & 31) == 31 && ld_relaxed_u32(&p.hdr->overflow)) return false;
  }
  atomicOr(&p.hdr->overflow, 1u);
  return false;
}

// ---------------------------------------------------------------- backends

constexpr uint32_t SHARED_MULT = 0x85EBCA77u;

// Thread-private -> CTA-shared -> global, each layer optional.  Only the
// GB_BLOCK consumer threads call these.
template <class S>
struct BeLayered {
  static constexpr int A = S::A;
  static constexpr int ID = relhost::K_GB_LAYERED;
  static constexpr int SIDE = SIDE_AGG;
  uint64_t* tk;              // [tiny_slots] stored keys
  uint64_t* tacc;            // [tiny_slots][A][GB_BLOCK] thread-private words
  uint64_t* tres;            // [tiny_slots][A] reduced words (flush)
  uint64_t* sk;              // [smem_slots] stored keys
  unsigned long long* sacc;  // [smem_slots][A]
  unsigned int* seen_all;    // thread-private slots any row of this CTA used
  uint32_t seen;             // ... by this thread (pinned slots may stay unused)

  __host__ __device__ static uint64_t bytes(uint32_t tiny, uint32_t shared) {
    return 8ull * tiny * (1 + (uint64_t)A * GB_BLOCK + A) + 8ull * shared * (1 + A) + 8ull;
  }
  __device__ void bind(uint8_t* area, const GbParams& p) {
    tk = (uint64_t*)area;
    tacc = tk + p.tiny_slots;
    tres = tacc + (size_t)p.tiny_slots * A * GB_BLOCK;
    sk = tres + (size_t)p.tiny_slots * A;
    sacc = (unsigned long long*)(sk + p.smem_slots);
    seen_all = (unsigned int*)(sacc + (size_t)p.smem_slots * A);
  }
  __device__ void init(const GbParams& p) {
    const uint32_t n1 = p.tiny_slots * (1 + A * GB_BLOCK);
    for (uint32_t i = threadIdx.x; i < n1; i += GB_BLOCK)
      tk[i] = (p.tiny_frozen && i < p.tiny_slots) ? p.tiny_init[i] : 0;
    const uint32_t n2 = p.smem_slots * (1 + A);
    for (uint32_t i = threadIdx.x; i < n2; i += GB_BLOCK) sk[i] = 0;
    seen = 0;
    if (threadIdx.x == 0) *seen_all = 0;
  }
  __device__ __forceinline__ void tiny_rmw(const GbParams& p, uint32_t s, const Vals<A>& x) {
    uint64_t* w = tacc + (size_t)s * A * GB_BLOCK + threadIdx.x;
#pragma unroll
    for (int a = 0; a < A; ++a) {
      if (live_agg<S>(p, a)) {
        const uint64_t o = w[a * GB_BLOCK];
        w[a * GB_BLOCK] = is_umax<S>(p, a) ? (o > x.v[a] ? o : x.v[a]) : o + x.v[a];
      }
    }
  }
  // Find the slot first, then update once: lanes that found their key at
  // different probe depths reconverge before the (long) update sequence.
  // false only when the global table overflowed.
  __device__ __forceinline__ bool update(const GbParams& p, uint64_t ek, const Vals<A>& x) {
    int where = 0;  // 1: thread-private slot s, 2: CTA-shared slot s, 0: neither
    uint32_t s = 0;
    if (p.tiny_slots && p.tiny_frozen) {
      // pinned keys, each at its own hash slot: one probe decides
      s = small_slot_of(ek, p.tiny_slots - 1, p.tiny_mult);
      if (tk[s] == ek) where = 1;
    } else if (p.tiny_slots) {
      const uint32_t mask = p.tiny_slots - 1;
      s = small_slot_of(ek, mask, p.tiny_mult);
#pragma unroll 1
      for (uint32_t i = 0; i < p.tiny_probes; ++i) {
        uint64_t k = *(volatile uint64_t*)(tk + s);
        if (k == 0) {
          k = atomicCAS((unsigned long long*)(tk + s), 0ull, (unsigned long long)ek);
          if (k == 0) k = ek;
        }
        if (k == ek) {
          where = 1;
          break;
        }
        s = (s + 1) & mask;
      }
    }
    if (where == 0 && p.smem_slots) {
      const uint32_t mask = p.smem_slots - 1;
      s = small_slot_of(ek, mask, SHARED_MULT);
#pragma unroll 1
      for (uint32_t i = 0; i < p.shared_probes; ++i) {
        uint64_t k = *(volatile uint64_t*)(sk + s);
        if (k == 0) {
          k = atomicCAS((unsigned long long*)(sk + s), 0ull, (unsigned long long)ek);
          if (k == 0) k = ek;
        }
        if (k == ek) {
          where = 2;
          break;
        }
        s = (s + 1) & mask;
      }
    }
    if (where == 1) {
      seen |= 1u << s;
      tiny_rmw(p, s, x);
      return true;
    }
    if (where == 2) {
      red_words_smem<S>(p, sacc + (size_t)s * A, x);
      return true;
    }
    if (p.tiny_slots || p.smem_slots) return gtab_update<S>(p, ek, x);
    return gtab_update_inl<S>(p, ek, x);
  }
  __device__ void flush(const GbParams& p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ws = __reduce_or_sync(0xffffffffu, seen);
    if (lane == 0 && ws) atomicOr(seen_all, ws);
    named_sync(GB_BLOCK);
    if (p.tiny_slots) {
      for (uint32_t pr = warp; pr < p.tiny_slots * A; pr += GB_BLOCK / 32) {
        const uint32_t s = pr / A, a = pr % A;
        if (tk[s] == 0 || !live_agg<S>(p, a)) continue;
        const bool um = is_umax<S>(p, a);
        const uint64_t* w = tacc + ((size_t)s * A + a) * GB_BLOCK;
        uint64_t v = 0;
        for (int t = lane; t < GB_BLOCK; t += 32) {
          const uint64_t y = w[t];
          v = um ? (v > y ? v : y) : v + y;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const uint64_t y = __shfl_xor_sync(0xffffffffu, v, o);
          v = um ? (v > y ? v : y) : v + y;
        }
        if (lane == 0) tres[s * A + a] = v;
      }
      named_sync(GB_BLOCK);
      if (threadIdx.x < p.tiny_slots && tk[threadIdx.x] != 0 &&
          ((*seen_all >> threadIdx.x) & 1u)) {
        Vals<A> x;
#pragma unroll
        for (int a = 0; a < A; ++a) x.v[a] = tres[threadIdx.x * A + a];
        gtab_update<S>(p, tk[threadIdx.x], x);
      }
    }
    for (uint32_t s = threadIdx.x; s < p.smem_slots; s += GB_BLOCK) {
      const uint64_t k = sk[s];
      if (k == 0) continue;
      Vals<A> x;
#pragma unroll
      for (int a = 0; a < A; ++a) x.v[a] = sacc[(size_t)s * A + a];
      gtab_update<S>(p, k, x);
    }
  }
};

// Pinned keys held in registers: each thread keeps NS x A accumulator words
// in registers and updates the row's group with unrolled, predicated adds and
// maxes -- independent ALU work with no shared-memory dependency chain.  The
// row's key is checked against the pinned table (perfect hash, one probe)
// and mapped to a dense id in [0, NS); a key the plan did not pin goes to the
// global table.  At the end each warp reduces its lanes with shuffles and the
// CTA merges the per-warp partials into the global table.
template <class S, int NS>
struct BeRegs {
  using Shape = S;
  static constexpr int A = S::A;
  static constexpr int ID = relhost::K_GB_REGS;
  static constexpr int SIDE = SIDE_AGG;
  uint64_t acc[NS][A];
  uint32_t seen;            // bit j: this thread updated dense slot j
  uint64_t* tk;             // [tiny_slots] pinned stored keys
  uint64_t* part;           // [GB_BLOCK / 32][NS][A] per-warp partials (flush)
  unsigned int* seen_all;   // OR of every thread's seen bits

  __host__ __device__ static uint64_t bytes(uint32_t tiny, uint32_t) {
    return 8ull * tiny + 8ull * (GB_BLOCK / 32) * NS * A + 8ull;
  }
  __device__ void bind(uint8_t* area, const GbParams& p) {
    tk = (uint64_t*)area;
    part = tk + p.tiny_slots;
    seen_all = (unsigned int*)(part + (GB_BLOCK / 32) * NS * A);
  }
  __device__ void init(const GbParams& p) {
#pragma unroll
    for (int j = 0; j < NS; ++j)
#pragma unroll
      for (int a = 0; a < A; ++a) acc[j][a] = 0;
    seen = 0;
    for (uint32_t i = threadIdx.x; i < p.tiny_slots; i += GB_BLOCK) tk[i] = p.tiny_init[i];
    if (threadIdx.x == 0) *seen_all = 0;
  }
  __device__ __forceinline__ bool update(const GbParams& p, uint64_t ek, const Vals<A>& x) {
    const uint32_t s = small_slot_of(ek, p.tiny_slots - 1, p.tiny_mult);
    if (tk[s] != ek) return gtab_update<S>(p, ek, x);
    const uint32_t d = (uint32_t)(p.tiny_dense >> (4u * s)) & 15u;
    seen |= 1u << d;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const bool hit = d == (uint32_t)j;
#pragma unroll
      for (int a = 0; a < A; ++a) {
        if (!live_agg<S>(p, a)) continue;
        const uint64_t o = acc[j][a];
        if (is_umax<S>(p, a))
          acc[j][a] = (hit && x.v[a] > o) ? x.v[a] : o;
        else
          acc[j][a] = o + (hit ? x.v[a] : 0ull);
      }
    }
    return true;
  }
  __device__ void flush(const GbParams& p) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const bool um = is_umax<S>(p, a);
        uint64_t v = acc[j][a];
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const uint64_t y = __shfl_xor_sync(0xffffffffu, v, o);
          v = um ? (v > y ? v : y) : v + y;
        }
        if (lane == 0) part[(warp * NS + j) * A + a] = v;
      }
    }
    const uint32_t ws = __reduce_or_sync(0xffffffffu, seen);
    if (lane == 0 && ws) atomicOr(seen_all, ws);
    named_sync(GB_BLOCK);
    // thread j merges dense slot j: its key is the pinned key with dense id j
    for (uint32_t s = threadIdx.x; s < p.tiny_slots; s += GB_BLOCK) {
      if (tk[s] == 0) continue;
      const int j = (int)((p.tiny_dense >> (4u * s)) & 15u);
      if (j >= NS || !((*seen_all >> j) & 1u)) continue;  // no row of this key here
      Vals<A> x;
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const bool um = is_umax<S>(p, a);
        uint64_t v = 0;
        for (int w = 0; w < GB_BLOCK / 32; ++w) {
          const uint64_t y = part[(w * NS + j) * A + a];
          v = um ? (v > y ? v : y) : v + y;
        }
        x.v[a] = v;
      }
      gtab_update<S>(p, tk[s], x);
    }
  }
};

// ------------------------------------------------- partitioned variant (P)


__device__ __forceinline__ bool is_pinned(const GbParams& p, const uint64_t* tk, uint64_t ek) {
  if (!p.tiny_frozen) return false;
  return tk[small_slot_of(ek, p.tiny_slots - 1, p.tiny_mult)] == ek;
}

// Pass 1: rows per (partition, CTA), pinned keys excluded.
template <class S>
struct BePartHist {
  static constexpr int A = S::A;
  static constexpr int ID = relhost::K_GB_PHIST;
  static constexpr int SIDE = SIDE_SKIP;
  uint64_t* tk;
  unsigned int* cnt;
  __host__ __device__ static uint64_t bytes(uint32_t tiny, uint32_t) {
    return 8ull * tiny + 4ull * (1u << PART_MAX_BITS);
  }
  __device__ void bind(uint8_t* area, const GbParams& p) {
    tk = (uint64_t*)area;
    cnt = (unsigned int*)(tk + p.tiny_slots);
  }
  __device__ void init(const GbParams& p) {
    for (uint32_t i = threadIdx.x; i < p.tiny_slots; i += GB_BLOCK) tk[i] = p.tiny_init[i];
    for (uint32_t i = threadIdx.x; i < (1u << p.part_bits); i += GB_BLOCK) cnt[i] = 0;
  }
  __device__ __forceinline__ bool update(const GbParams& p, uint64_t ek, const Vals<A>&) {
    if (!is_pinned(p, tk, ek)) atomicAdd(&cnt[part_of(ek, p.part_bits)], 1u);
    return true;
  }
  __device__ void flush(const GbParams& p) {
    named_sync(GB_BLOCK);
    for (uint32_t i = threadIdx.x; i < (1u << p.part_bits); i += GB_BLOCK)
      p.hist[(size_t)i * p.fixed_grid + blockIdx.x] = cnt[i];
  }
};

// Pass 2: pinned keys aggregate in thread-private slots (merged into the
// global table at the end); every other row becomes a (key, value) record
// at its partition's next position for this CTA.
template <class S>
struct BePartScatter {
  static constexpr int A = S::A;
  static constexpr int ID = relhost::K_GB_PSCATTER;
  static constexpr int SIDE = SIDE_AGG;
  BeLayered<S> hot;           // thread-private layer (frozen) only
  unsigned int* cursor;       // [P] next record index of this CTA per partition
                              // (32-bit: a partitioned input has < 2^32 rows,
                              // and a 32-bit shared atomic is native)
  unsigned long long total;   // records the histogram counted (bound check)
  __host__ __device__ static uint64_t bytes(uint32_t tiny, uint32_t) {
    return ((BeLayered<S>::bytes(tiny, 0) + 15) & ~15ull) + 4ull * (1u << PART_MAX_BITS);
  }
  __device__ void bind(uint8_t* area, const GbParams& p) {
    hot.bind(area, p);
    cursor = (unsigned int*)(area + ((BeLayered<S>::bytes(p.tiny_slots, 0) + 15) & ~15ull));
  }
  __device__ void init(const GbParams& p) {
    hot.init(p);
    for (uint32_t i = threadIdx.x; i < (1u << p.part_bits); i += GB_BLOCK)
      cursor[i] = (unsigned int)(p.part_start[i] + p.hist[(size_t)i * p.fixed_grid + blockIdx.x]);
    total = p.part_start[1u << p.part_bits];
  }
  __device__ __forceinline__ bool update(const GbParams& p, uint64_t ek, const Vals<A>& x) {
    if (p.tiny_frozen) {
      const uint32_t s = small_slot_of(ek, p.tiny_slots - 1, p.tiny_mult);
      if (hot.tk[s] == ek) {
        hot.seen |= 1u << s;
        hot.tiny_rmw(p, s, x);
        return true;
      }
    }
    const unsigned long long pos = atomicAdd(&cursor[part_of(ek, p.part_bits)], 1u);
    if (pos >= total) {  // the passes disagreed: report, never write past the buffer
      atomicOr(&p.hdr->timeout, 2u);
      return false;
    }
    PartRec r;
    r.ek = ek;
    r.val = (long long)x.v[0];
    p.recs[pos] = r;
    return true;
  }
  __device__ void flush(const GbParams& p) { hot.flush(p); }
};

// Distinct-key counting: a CTA-shared key filter in front of the global set.
template <class S>
struct BeKeySet {
  static constexpr int A = S::A;
  static constexpr int ID = relhost::K_GB_KEYSET;
  static constexpr int SIDE = SIDE_COUNT;
  uint64_t* tk;
  __host__ __device__ static uint64_t bytes(uint32_t, uint32_t shared) { return 8ull * shared; }
  __device__ void bind(uint8_t* area, const GbParams&) { tk = (uint64_t*)area; }
  __device__ void init(const GbParams& p) {
    for (uint32_t i = threadIdx.x; i < p.smem_slots; i += GB_BLOCK) tk[i] = 0;
  }
  __device__ __forceinline__ bool update(const GbParams& p, uint64_t ek, const Vals<A>&) {
    const uint32_t mask = p.smem_slots - 1;
    uint32_t s = small_slot_of(ek, mask, SHARED_MULT);
    for (uint32_t i = 0; i < p.shared_probes; ++i) {
      uint64_t k = *(volatile uint64_t*)(tk + s);
      if (k == ek) return true;  // this CTA already sent the key to the global set
      if (k == 0) {
        k = atomicCAS((unsigned long long*)(tk + s), 0ull, (unsigned long long)ek);
        if (k == 0) break;  // first sight in this CTA
        if (k == ek) return true;
      }
      s = (s + 1) & mask;
    }
    return gset_insert(p, ek);
  }
  __device__ void flush(const GbParams&) {}
};

// -------------------------------------------------------------- main kernel

// Fold rows [0, nrows) of a tile view into the backend; returns false once
// the global table overflowed (later rows are then pointless).
template <class S, class BE, bool KEYSET, class V>
__device__ __forceinline__ bool run_rows(const GbParams& p, BE& be, const V& v, int nrows) {
  bool ok = true;
  const auto q = S::prep(p, v);
#pragma unroll 4
  for (int r = threadIdx.x; r < nrows; r += GB_BLOCK) {
    uint64_t ek;
    Vals<S::A> x;
    if (!S::row(p, q, r, ek, x)) continue;
    if (ek == 0) {  // the key INT64_MIN: side accumulator (once per row overall)
      if (BE::SIDE != SIDE_SKIP) atomicAdd(&p.hdr->n_side, 1ull);
      if (BE::SIDE == SIDE_AGG) red_words<S>(p, p.hdr->side_aggs, x);
      continue;
    }
    ok &= be.update(p, ek, x);
  }
  return ok;
}

// Persistent, warp-specialised: warps 0..7 consume (GB_BLOCK threads), warp 8
// produces.  The producer streams tile after tile of every column into a
// ring of n_stages shared-memory stages with TMA bulk copies; stage s is
// "full" when its bytes have landed (full[s]) and "empty" again when all
// eight consumer warps have arrived on empty[s].  No CTA-wide barrier runs
// per tile.  Every wait is bounded; a wait that gives up sets hdr->timeout.
template <class S, class BE, bool KEYSET, bool USE_TMA>
__global__ void __launch_bounds__(GB_THREADS) gb_main(const __grid_constant__ GbParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = (uint64_t*)smem;        // [n_stages]
  uint64_t* empty = (uint64_t*)smem + GB_MAX_STAGES;  // [n_stages]
  int* abort_flag = (int*)(smem + 16 * GB_MAX_STAGES);
  uint8_t* area = smem + GB_SMEM_HEAD;
  BE be;
  be.bind(area, p);
  const bool consumer = threadIdx.x < GB_BLOCK;
  if (consumer) be.init(p);
  uint8_t* stages = area + ((BE::bytes(p.tiny_slots, p.smem_slots) + 127) & ~127ull);

  const int64_t T = p.tile_rows;
  const int NS = p.n_stages;
  const int64_t n_tiles = USE_TMA ? p.n_rows / T : (p.n_rows + T - 1) / T;
  const int64_t mine = n_tiles > (int64_t)blockIdx.x
                           ? (n_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1
                           : 0;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    if (USE_TMA) {
      for (int s = 0; s < NS; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], GB_BLOCK / 32);
      }
      fence_mbar_init();
    }
  }
  __syncthreads();

  if (!consumer) {
    // ---- producer warp: one lane issues every copy of this CTA
    if (!USE_TMA || (threadIdx.x & 31) != 0) return;
    const uint64_t policy = l2_evict_first_policy();
    int64_t k = 0;
    for (; k < mine; ++k) {
      const int s = (int)(k % NS);
      if (k >= NS && !mbar_wait_bounded(&empty[s], (uint32_t)((k / NS - 1) & 1), p.wait_ns)) {
        atomicOr(&p.hdr->timeout, 1u);
        break;
      }
      if (*(volatile int*)abort_flag) break;
      const int64_t t = (int64_t)blockIdx.x + k * (int64_t)gridDim.x;
      mbar_arrive_expect_tx(&full[s], p.stage_bytes);
      uint8_t* dst = stages + (size_t)s * p.stage_bytes;
      for (int c = 0; c < p.n_cols; ++c) {
        const uint32_t nb = (uint32_t)(T * p.csize[c]);
        bulk_g2s(dst + p.stage_off[c], p.col[c] + t * T * p.csize[c], nb, &full[s], policy);
      }
    }
    // the CTA's shared memory must outlive every copy issued into it
    for (int64_t j = (k > NS ? k - NS : 0); j < k; ++j)
      mbar_wait_bounded(&full[j % NS], (uint32_t)((j / NS) & 1), p.wait_ns);
    return;
  }

  // ---- consumers
  const int lane = threadIdx.x & 31;
  bool live = true;  // false once the global table overflowed
  if (USE_TMA) {
    for (int64_t k = 0; k < mine; ++k) {
      const int s = (int)(k % NS);
      if (!mbar_wait_bounded(&full[s], (uint32_t)((k / NS) & 1), p.wait_ns)) {
        atomicOr(&p.hdr->timeout, 1u);
        *(volatile int*)abort_flag = 1;
        break;
      }
      if (live) live = run_rows<S, BE, KEYSET>(p, be, SmemView{stages + (size_t)s * p.stage_bytes}, (int)T);
      if ((k & 31) == 31) {  // now and then, notice another CTA's overflow
        uint32_t f = lane == 0 ? ld_relaxed_u32(&p.hdr->overflow) : 0;
        live = live && __shfl_sync(0xffffffffu, f, 0) == 0;
      }
      __syncwarp();
      // (test hook: a ring whose stages never come back, so that the
      // producer's and then the consumers' bounded waits run out)
      if (lane == 0 && !p.test_stall) mbar_arrive(&empty[s]);
    }
    const int64_t tail0 = n_tiles * T;
    if (live && tail0 < p.n_rows && blockIdx.x == (unsigned)(n_tiles % gridDim.x))
      run_rows<S, BE, KEYSET>(p, be, GlobalView{tail0}, (int)(p.n_rows - tail0));
  } else {
    for (int64_t k = 0; k < mine; ++k) {
      const int64_t t = (int64_t)blockIdx.x + k * (int64_t)gridDim.x;
      const int64_t r0 = t * T;
      const int nrows = (int)(p.n_rows - r0 < T ? p.n_rows - r0 : T);
      const bool ok = run_rows<S, BE, KEYSET>(p, be, GlobalView{r0}, nrows);
      uint32_t f = lane == 0 ? ld_relaxed_u32(&p.hdr->overflow) : 0;
      f = __shfl_sync(0xffffffffu, f, 0);
      if (!__all_sync(0xffffffffu, ok) || f) break;  // warp-uniform exit
    }
  }
  // flush unless the result is void anyway (uniform across consumers)
  named_sync(GB_BLOCK);
  if (*(volatile int*)abort_flag) return;
  be.flush(p);
}

// ---------------------------------------------------------------- compaction

__global__ void __launch_bounds__(GB_BLOCK) gb_compact(const __grid_constant__ GbParams p,
                                                        const __grid_constant__ GbOut o) {
  const uint64_t slots = 1ull << p.log2_slots;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (uint64_t base = (uint64_t)blockIdx.x * GB_BLOCK; base < slots;
       base += (uint64_t)gridDim.x * GB_BLOCK) {
    const uint64_t s = base + threadIdx.x;
    const uint64_t ek = s < slots ? p.tkeys[s] : 0;
    const bool occ = ek != 0;
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    if (!m) continue;
    unsigned long long wb = 0;
    if (lane == 0) wb = atomicAdd(&p.hdr->n_out, (unsigned long long)__popc(m));
    wb = __shfl_sync(0xffffffffu, wb, 0);
    if (occ) {
      const uint64_t pos = wb + __popc(m & lt);
      if (pos < (uint64_t)o.capacity) {
        o.keys[pos] = (int64_t)(ek ^ KEY_FLIP);
        const unsigned long long* w = p.taggs + s * (uint64_t)p.n_aggs;
        for (int a = 0; a < p.n_aggs; ++a) o.aggs[a][pos] = agg_decode(p.aop[a], w[a]);
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.hdr->n_side > 0) {
    const unsigned long long pos = atomicAdd(&p.hdr->n_out, 1ull);
    if (pos < (unsigned long long)o.capacity) {
      o.keys[pos] = (int64_t)KEY_FLIP;  // INT64_MIN
      for (int a = 0; a < p.n_aggs; ++a) o.aggs[a][pos] = agg_decode(p.aop[a], p.hdr->side_aggs[a]);
    }
  }
}

// ------------------------------------------- partitioned variant: scan, agg

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024).
__device__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* total) {
  __shared__ unsigned long long warp_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long w = lane < nw ? warp_sum[lane] : 0;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) warp_sum[lane] = wi - w;  // exclusive prefix of warp totals
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const unsigned long long r = warp_sum[warp] + incl - v;
  __syncthreads();
  return r;
}

// hist[part][cta] -> exclusive offsets inside the partition; the partition's
// total goes to part_start[part].  One CTA per partition.
__global__ void __launch_bounds__(1024) gb_part_scan1(const __grid_constant__ GbParams p) {
  __shared__ unsigned long long total;
  const uint32_t G = p.fixed_grid;
  uint32_t* h = p.hist + (size_t)blockIdx.x * G;
  const uint32_t per = (G + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = b + per < G ? b + per : G;
  unsigned long long s = 0;
  for (uint32_t i = b; i < e; ++i) s += h[i];
  unsigned long long run = block_exclusive_scan(s, &total);
  for (uint32_t i = b; i < e; ++i) {
    const uint32_t v = h[i];
    h[i] = (uint32_t)run;
    run += v;
  }
  if (threadIdx.x == 0) p.part_start[blockIdx.x] = total;
}

// hist[part][cta] -> the partition's total in part_start[part] only (the
// streaming passes place records by bin cursors, not by per-CTA offsets).
// One warp per partition.
__global__ void __launch_bounds__(256) gb_part_sum(const __grid_constant__ GbParams p) {
  const uint32_t part = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (part >= (1u << p.part_bits)) return;  // whole warps
  const uint32_t G = p.fixed_grid;
  const uint32_t* h = p.hist + (size_t)part * G;
  unsigned long long s = 0;
  for (uint32_t i = lane; i < G; i += 32) s += h[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) p.part_start[part] = s;
}

// partition totals -> first record of each partition; part_start[P] = all.
// Also the cursors of both scatter levels and the level-2 pass's tiles.
__global__ void __launch_bounds__(1024) gb_part_scan2(const __grid_constant__ GbParams p) {
  __shared__ unsigned long long total, tiles_total;
  const uint32_t P = 1u << p.part_bits;
  const uint32_t per = (P + blockDim.x - 1) / blockDim.x;
  const uint32_t b = threadIdx.x * per, e = b + per < P ? b + per : P;
  unsigned long long s = 0;
  for (uint32_t i = b; i < e; ++i) s += p.part_start[i];
  unsigned long long run = block_exclusive_scan(s, &total);
  for (uint32_t i = b; i < e; ++i) {
    const unsigned long long v = p.part_start[i];
    p.part_start[i] = run;
    p.cursor[i] = (unsigned int)run;
    run += v;
  }
  if (threadIdx.x == 0) p.part_start[P] = total;
  __syncthreads();
  // level-1 bins: 2^shift1 consecutive partitions each
  const uint32_t shift1 = p.part_bits > PART_L1_BITS ? p.part_bits - PART_L1_BITS : 0;
  const uint32_t B1 = P >> shift1;
  unsigned long long tiles = 0;
  if (threadIdx.x < B1) {
    const unsigned long long s1 = p.part_start[threadIdx.x << shift1];
    const unsigned long long e1 = p.part_start[(threadIdx.x + 1) << shift1];
    p.cursor1[threadIdx.x] = (unsigned int)s1;
    tiles = (e1 - s1 + PART_TILE - 1) / PART_TILE;
  }
  const unsigned long long tp = block_exclusive_scan(tiles, &tiles_total);
  if (threadIdx.x < B1) p.l2_tiles[threadIdx.x] = (unsigned int)tp;
  if (threadIdx.x == 0) p.l2_tiles[B1] = (unsigned int)tiles_total;
}

// Insert-or-accumulate into a partition's shared-memory table; a key that
// finds no slot within 32 probes goes to the global table and marks the
// partition as spilled.
template <class S>
__device__ __forceinline__ void part_insert(const GbParams& p, uint64_t* tk, unsigned long long* ta,
                                            uint32_t TS, uint64_t ek, const Vals<S::A>& x,
                                            int* ovf) {
  uint32_t s = small_slot_of(ek, TS - 1, SHARED_MULT);
  for (uint32_t k = 0; k < 32; ++k) {
    uint64_t cur = *(volatile uint64_t*)(tk + s);
    if (cur == 0) {
      cur = atomicCAS((unsigned long long*)(tk + s), 0ull, (unsigned long long)ek);
      if (cur == 0) cur = ek;
    }
    if (cur == ek) {
      red_words_smem<S, true>(p, ta + (size_t)s * S::A, x);
      return;
    }
    s = (s + 1) & (TS - 1);
  }
  *(volatile int*)ovf = 1;
  gtab_update<S>(p, ek, x);
}

// record groups in flight per warp in the aggregation pass (2, 4, 8: 1.36, 1.40
// and 1.94 ms on 2e8 Zipf rows: fewer registers, more warps)
constexpr int PA_R = 2;

// Pass 3: each CTA aggregates whole partitions in a shared-memory table of
// p.smem_slots slots and writes their groups straight to the output (warp
// ballot / popc, one atomic per warp).  Every key lives in one partition, so
// no group is emitted twice -- unless the table overflows: then the whole
// partition is merged into the global table instead, which the compaction
// kernel emits afterwards.
template <class S>
__global__ void __launch_bounds__(GB_BLOCK) gb_part_agg(const __grid_constant__ GbParams p,
                                                         const __grid_constant__ GbOut o) {
  constexpr int A = S::A;
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ int ovf;
  const uint32_t TS = p.smem_slots;
  uint64_t* tk = (uint64_t*)sm;
  unsigned long long* ta = (unsigned long long*)(tk + TS);
  const uint32_t P = 1u << p.part_bits;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // a partition far above the average (skewed keys) is split into up to
  // PART_CHUNKS chunks on different CTAs, which then merge into the global
  // table instead of emitting
  const unsigned long long avg = p.part_start[P] / P;
  const unsigned long long chunk_min = 4 * avg > 4096 ? 4 * avg : 4096;
  for (uint32_t item = blockIdx.x; item < P * PART_CHUNKS; item += gridDim.x) {
    // chunk-major numbering: the first chunks of all partitions come first and
    // spread over every CTA
    const uint32_t part = item % P, c = item / P;
    const unsigned long long pb = p.part_start[part], pe = p.part_start[part + 1];
    const unsigned long long size = pe - pb;
    unsigned long long nch = (size + chunk_min - 1) / chunk_min;
    nch = nch < 1 ? 1 : (nch > PART_CHUNKS ? PART_CHUNKS : nch);
    if (c >= nch) continue;  // uniform across the CTA
    const unsigned long long beg = pb + size * c / nch, end = pb + size * (c + 1) / nch;
    for (uint32_t i = threadIdx.x; i < TS * (1 + A); i += GB_BLOCK) tk[i] = 0;
    if (threadIdx.x == 0) ovf = nch > 1;
    __syncthreads();
    {
      // each warp takes 32 consecutive records at a time, PA_R such groups
      // loaded before any is used, and the next PA_R groups' loads go out
      // before this batch is inserted (the pass waits on load latency).  Lanes
      // of one key are not combined in registers first: on the partitions of
      // skewed keys that did not cost less than the serialised shared-memory
      // atomics it saves (2e8 Zipf(1.1) rows: 2.0 -> 1.9 ms without it)
      const int warp = threadIdx.x >> 5;
      const unsigned long long bstep = (unsigned long long)GB_BLOCK * PA_R;
      longlong2 rec[PA_R];
      unsigned long long b00 = beg + (unsigned long long)warp * 32 * PA_R;
#pragma unroll
      for (int rr = 0; rr < PA_R; ++rr) {
        const unsigned long long i = b00 + (unsigned long long)rr * 32 + lane;
        rec[rr] = i < end ? __ldcs((const longlong2*)(p.recs + i)) : make_longlong2(0, 0);
      }
      for (; b00 < end; b00 += bstep) {
        // the next groups' records go out before this group's are inserted
        longlong2 nxt[PA_R];
#pragma unroll
        for (int rr = 0; rr < PA_R; ++rr) {
          const unsigned long long i = b00 + bstep + (unsigned long long)rr * 32 + lane;
          nxt[rr] = i < end ? __ldcs((const longlong2*)(p.recs + i)) : make_longlong2(0, 0);
        }
#pragma unroll
        for (int rr = 0; rr < PA_R; ++rr) {
          if (b00 + (unsigned long long)rr * 32 + lane >= end) continue;
          Vals<A> x;
          S::from_val((uint64_t)rec[rr].y, x);
          part_insert<S>(p, tk, ta, TS, (uint64_t)rec[rr].x, x, &ovf);
        }
#pragma unroll
        for (int rr = 0; rr < PA_R; ++rr) rec[rr] = nxt[rr];
      }
    }
    __syncthreads();
    const bool spill = ovf != 0;
    for (uint32_t base = 0; base < TS; base += GB_BLOCK) {
      const uint32_t s = base + threadIdx.x;
      const uint64_t ek = s < TS ? tk[s] : 0;
      const bool occ = ek != 0;
      if (spill) {  // partition did not fit: everything to the global table
        if (occ) {
          Vals<A> x;
#pragma unroll
          for (int a = 0; a < A; ++a) x.v[a] = ta[(size_t)s * A + a];
          gtab_update<S>(p, ek, x);
        }
        continue;
      }
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      if (!m) continue;
      unsigned long long wb = 0;
      if (lane == 0) wb = atomicAdd(&p.hdr->n_out, (unsigned long long)__popc(m));
      wb = __shfl_sync(0xffffffffu, wb, 0);
      if (occ) {
        const uint64_t pos = wb + __popc(m & lt);
        if (pos < (uint64_t)o.capacity) {
          o.keys[pos] = (int64_t)(ek ^ KEY_FLIP);
#pragma unroll
          for (int a = 0; a < A; ++a) o.aggs[a][pos] = agg_decode(p.aop[a], ta[(size_t)s * A + a]);
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ launch

namespace {

template <class F>
auto with_shape(int shape, F&& f) {
  switch (shape) {
    case SHAPE_Q1: return f(ShapeQ1{});
    case SHAPE_KVRT64: return f(ShapeKVRT<int64_t>{});
    case SHAPE_KVRT32: return f(ShapeKVRT<int32_t>{});
    case SHAPE_KV4_64: return f(ShapeKV<int64_t, 4>{});
    case SHAPE_KV4_32: return f(ShapeKV<int32_t, 4>{});
    case SHAPE_KV2_64: return f(ShapeKV<int64_t, 2>{});
    case SHAPE_KV2_32: return f(ShapeKV<int32_t, 2>{});
    default: return f(ShapeGeneric{});
  }
}

// The key-set pass only needs keys and filters: it runs on a reduced
// descriptor, so fewer shapes are instantiated for it.
template <class F>
auto with_keyset_shape(int shape, F&& f) {
  switch (shape) {
    case SHAPE_Q1: return f(ShapeQ1{});
    case SHAPE_KVRT64: case SHAPE_KV4_64: case SHAPE_KV2_64: return f(ShapeKVRT<int64_t>{});
    case SHAPE_KVRT32: case SHAPE_KV4_32: case SHAPE_KV2_32: return f(ShapeKVRT<int32_t>{});
    default: return f(ShapeGeneric{});
  }
}

// Partitioned passes: key + int64 value shapes only.
template <class F>
auto with_part_shape(int shape, F&& f) {
  switch (shape) {
    case SHAPE_KV4_32: return f(ShapeKV<int32_t, 4>{});
    case SHAPE_KV2_64: return f(ShapeKV<int64_t, 2>{});
    case SHAPE_KV2_32: return f(ShapeKV<int32_t, 2>{});
    default: return f(ShapeKV<int64_t, 4>{});
  }
}

// Register-privatised kernels: shapes of at most 5 words, 4 or 8 dense slots.
template <class F>
auto with_regs(int shape, uint32_t ns, F&& f) {
  auto pick = [&](auto s) {
    using S = decltype(s);
    return ns <= 4 ? f(BeRegs<S, 4>{}) : f(BeRegs<S, 8>{});
  };
  switch (shape) {
    case SHAPE_Q1: return pick(ShapeQ1{});
    case SHAPE_KV4_32: return pick(ShapeKV<int32_t, 4>{});
    case SHAPE_KV2_64: return pick(ShapeKV<int64_t, 2>{});
    case SHAPE_KV2_32: return pick(ShapeKV<int32_t, 2>{});
    default: return pick(ShapeKV<int64_t, 4>{});
  }
}

template <class S, class BE, bool KEYSET, bool TMA>
size_t smem_of(const GbParams& p) {
  const uint64_t be = (BE::bytes(p.tiny_slots, p.smem_slots) + 127) & ~127ull;
  return GB_SMEM_HEAD + be + (TMA ? (size_t)p.n_stages * p.stage_bytes : 0);
}

template <class S, class BE, bool KEYSET, bool TMA>
int occupancy(const GbParams& p) {
  auto kern = gb_main<S, BE, KEYSET, TMA>;
  const size_t smem = smem_of<S, BE, KEYSET, TMA>(p);
  if (smem > 227 * 1024) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GB_THREADS, smem) != cudaSuccess)
    return 0;
  return per_sm;
}

template <class S, class BE, bool KEYSET, bool TMA>
rel_status launch_one(const GbParams& p, cudaStream_t st) {
  auto kern = gb_main<S, BE, KEYSET, TMA>;
  const size_t smem = smem_of<S, BE, KEYSET, TMA>(p);
  const int per_sm = occupancy<S, BE, KEYSET, TMA>(p);
  if (per_sm < 1) {
    relhost::set_error("group-by: %zu bytes of shared memory per CTA cannot launch", smem);
    return REL_E_UNSUPPORTED;
  }
  const int64_t tiles = (p.n_rows + p.tile_rows - 1) / p.tile_rows;
  int64_t grid = (int64_t)relhost::device_sms() * per_sm;
  if (grid > tiles) grid = tiles > 0 ? tiles : 1;
  if (p.fixed_grid) grid = p.fixed_grid;  // passes that must map rows to CTAs alike
  relhost::launch_begin(BE::ID, st);
  kern<<<(unsigned)grid, GB_THREADS, smem, st>>>(p);
  relhost::launch_end(BE::ID, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return relhost::cuda_fail(e, "launch(group-by)");
  return REL_OK;
}

}  // namespace

int gb_shape_width(int shape) {
  return with_shape(shape, [](auto s) { return decltype(s)::A; });
}

uint64_t gb_backend_smem_bytes(int mode, int shape, uint32_t tiny_slots, uint32_t smem_slots) {
  if (mode == MODE_KEYSET) return 8ull * smem_slots;
  if (mode == MODE_PHIST)
    return with_part_shape(shape, [&](auto s) {
      return BePartHist<decltype(s)>::bytes(tiny_slots, smem_slots);
    });
  if (mode == MODE_PSCATTER)
    return with_part_shape(shape, [&](auto s) {
      return BePartScatter<decltype(s)>::bytes(tiny_slots, smem_slots);
    });
  if (mode == MODE_TINY)
    return with_regs(shape, 8, [&](auto be) { return decltype(be)::bytes(tiny_slots, smem_slots); });
  return with_shape(shape, [&](auto s) {
    return BeLayered<decltype(s)>::bytes(tiny_slots, smem_slots);
  });
}

int gb_ctas_per_sm(const GbParams& p, int shape, int mode, bool tma) {
  if (mode == MODE_PHIST || mode == MODE_PSCATTER)
    return with_part_shape(shape, [&](auto s) {
      using S = decltype(s);
      if (mode == MODE_PHIST)
        return tma ? occupancy<S, BePartHist<S>, false, true>(p)
                   : occupancy<S, BePartHist<S>, false, false>(p);
      return tma ? occupancy<S, BePartScatter<S>, false, true>(p)
                 : occupancy<S, BePartScatter<S>, false, false>(p);
    });
  if (mode == MODE_KEYSET)
    return with_keyset_shape(shape, [&](auto s) {
      using S = decltype(s);
      return tma ? occupancy<S, BeKeySet<S>, true, true>(p)
                 : occupancy<S, BeKeySet<S>, true, false>(p);
    });
  if (mode == MODE_TINY)
    return with_regs(shape, p.tiny_ns, [&](auto be) {
      using BE = decltype(be);
      using S = typename BE::Shape;
      return tma ? occupancy<S, BE, false, true>(p) : occupancy<S, BE, false, false>(p);
    });
  return with_shape(shape, [&](auto s) {
    using S = decltype(s);
    return tma ? occupancy<S, BeLayered<S>, false, true>(p)
               : occupancy<S, BeLayered<S>, false, false>(p);
  });
}

rel_status gb_launch_main(const GbParams& p, int shape, int mode, bool tma, cudaStream_t st) {
  if (p.n_rows == 0 && !p.fixed_grid) return REL_OK;
  if (mode == MODE_PHIST || mode == MODE_PSCATTER)
    return with_part_shape(shape, [&](auto s) {
      using S = decltype(s);
      if (mode == MODE_PHIST)
        return tma ? launch_one<S, BePartHist<S>, false, true>(p, st)
                   : launch_one<S, BePartHist<S>, false, false>(p, st);
      return tma ? launch_one<S, BePartScatter<S>, false, true>(p, st)
                 : launch_one<S, BePartScatter<S>, false, false>(p, st);
    });
  if (mode == MODE_KEYSET)
    return with_keyset_shape(shape, [&](auto s) {
      using S = decltype(s);
      return tma ? launch_one<S, BeKeySet<S>, true, true>(p, st)
                 : launch_one<S, BeKeySet<S>, true, false>(p, st);
    });
  if (mode == MODE_TINY)
    return with_regs(shape, p.tiny_ns, [&](auto be) {
      using BE = decltype(be);
      using S = typename BE::Shape;
      return tma ? launch_one<S, BE, false, true>(p, st) : launch_one<S, BE, false, false>(p, st);
    });
  return with_shape(shape, [&](auto s) {
    using S = decltype(s);
    return tma ? launch_one<S, BeLayered<S>, false, true>(p, st)
               : launch_one<S, BeLayered<S>, false, false>(p, st);
  });
}

rel_status gb_launch_part_scan(const GbParams& p, bool cta_offsets, cudaStream_t st) {
  const uint32_t P = 1u << p.part_bits;
  relhost::launch_begin(relhost::K_GB_PSCAN, st);
  if (cta_offsets)
    gb_part_scan1<<<P, 1024, 0, st>>>(p);
  else
    gb_part_sum<<<(P + 7) / 8, 256, 0, st>>>(p);
  relhost::launch_end(relhost::K_GB_PSCAN, st);
  relhost::launch_begin(relhost::K_GB_PSCAN, st);
  gb_part_scan2<<<1, 1024, 0, st>>>(p);
  relhost::launch_end(relhost::K_GB_PSCAN, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(partition scan)");
}

rel_status gb_launch_part_agg(const GbParams& p, int shape, const GbOut& o, cudaStream_t st) {
  return with_part_shape(shape, [&](auto s) -> rel_status {
    using S = decltype(s);
    auto kern = gb_part_agg<S>;
    const size_t smem = 8ull * p.smem_slots * (1 + S::A);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaFuncSetAttribute(partition agg)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GB_BLOCK, smem);
    if (e != cudaSuccess || per_sm < 1) return relhost::cuda_fail(e, "occupancy(partition agg)");
    const uint32_t P = 1u << p.part_bits;
    uint32_t grid = (uint32_t)relhost::device_sms() * (uint32_t)per_sm;
    if (grid > P) grid = P;
    relhost::launch_begin(relhost::K_GB_PAGG, st);
    kern<<<grid, GB_BLOCK, smem, st>>>(p, o);
    relhost::launch_end(relhost::K_GB_PAGG, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(partition agg)");
  });
}

rel_status gb_launch_compact(const GbParams& p, const GbOut& o, cudaStream_t st) {
  const uint64_t slots = 1ull << p.log2_slots;
  int64_t grid = (int64_t)((slots + GB_BLOCK - 1) / GB_BLOCK);
  const int64_t cap = (int64_t)relhost::device_sms() * 8;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  relhost::launch_begin(relhost::K_GB_COMPACT, st);
  gb_compact<<<(unsigned)grid, GB_BLOCK, 0, st>>>(p, o);
  relhost::launch_end(relhost::K_GB_COMPACT, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return relhost::cuda_fail(e, "launch(compact)");
  return REL_OK;
}

}  // namespace rel
