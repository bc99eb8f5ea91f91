// Fused filter + hash group-by kernels for sm_103a.
//
// One persistent launch streams every column of the query through shared
// memory with the TMA bulk-copy engine (a ring of GB_STAGES stages completed
// on mbarriers), evaluates the range filter, the packed group key and the
// product-form aggregate inputs in registers -- no expression interpreter and
// no materialised mask, the instruction overheads the paper attributes to
// compute_column_kernel and transform_kernel (Sec. 7) -- and folds each row
// into a table:
//   MODE_TINY   : up to 8 groups per CTA, each thread owning private
//                 accumulators in shared memory (no atomics on the hot path);
//   MODE_SHARED : a CTA-shared open-addressing table with shared-memory
//                 atomics (the privatised aggregation of
//                 single_pass_shmem_aggs_kernel, Sec. 7);
//   MODE_GLOBAL : one open-addressing table in global memory;
//   MODE_KEYSET : keys only, counting distinct keys (the exact sizing pass).
// Per-CTA tables spill rows they cannot hold to the global table and merge
// into it at the end, so every mode produces the same exact groups.  A
// compaction kernel then turns occupied slots into dense output rows with a
// warp ballot / popc and one atomic per warp.
#include <algorithm>

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
  __device__ __forceinline__ T at(const GbParams& p, int c, int r) const {
    return ((const T*)(base + p.stage_off[c]))[r];
  }
};

struct GlobalView {
  int64_t row0;
  __device__ __forceinline__ int64_t get(const GbParams& p, int c, int r) const {
    int64_t i = row0 + r;
    switch (p.ctype[c]) {
      case REL_U8: return (int64_t)__ldg(p.col[c] + i);
      case REL_I32: return (int64_t)__ldg((const int32_t*)p.col[c] + i);
      default: return (int64_t)__ldg((const long long*)p.col[c] + i);
    }
  }
  template <class T>
  __device__ __forceinline__ T at(const GbParams& p, int c, int r) const {
    return (T)__ldg((const T*)p.col[c] + row0 + r);
  }
};

template <>
__device__ __forceinline__ int64_t GlobalView::at<int64_t>(const GbParams& p, int c, int r) const {
  return (int64_t)__ldg((const long long*)p.col[c] + row0 + r);
}

// ------------------------------------------------------------- row shapes
// row(): false when the filter rejects the row; else the stored key
// ek = key ^ KEY_FLIP and the encoded aggregate inputs x[0..n_aggs).

// Any descriptor within the REL_MAX_* limits, read from the kernel params.
struct ShapeGeneric {
  template <int A, class V>
  __device__ __forceinline__ static bool row(const GbParams& p, const V& v, int r, uint64_t& ek,
                                             uint64_t (&x)[A]) {
#pragma unroll
    for (int i = 0; i < REL_MAX_PREDS; ++i) {
      if (i < p.n_preds) {
        int64_t d = v.get(p, p.pred_col[i], r);
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
        int op = p.aop[a];
        if (op == REL_COUNT) {
          x[a] = 1;
        } else {
          uint64_t val = (uint64_t)v.get(p, p.abase[a], r);
#pragma unroll
          for (int f = 0; f < 2; ++f)
            if (f < p.anf[a])
              val *= (uint64_t)p.ac[a][f] + (uint64_t)p.as[a][f] * (uint64_t)v.get(p, p.afcol[a][f], r);
          x[a] = agg_encode(op, (int64_t)val);
        }
      }
    }
    return true;
  }
};

// keep lo <= pred[i] <= hi (i32 column); key = (u8 k0 << 8) | u8 k1;
// sum(a), sum(b), sum(b*(c0 + s0*d)), sum(b*(c0 + s0*d)*(c1 + s1*t)), count.
struct ShapeQ1 {
  template <int A, class V>
  __device__ __forceinline__ static bool row(const GbParams& p, const V& v, int r, uint64_t& ek,
                                             uint64_t (&x)[A]) {
    static_assert(A == 5, "Q1 shape has five aggregates");
    int64_t d = (int64_t)v.template at<int32_t>(p, p.r_pred, r);
    if (d < p.pred_lo[0] || d > p.pred_hi[0]) return false;
    uint64_t k0 = v.template at<uint8_t>(p, p.r_k0, r);
    uint64_t k1 = v.template at<uint8_t>(p, p.r_k1, r);
    ek = ((k0 << 8) | k1) ^ KEY_FLIP;
    uint64_t qa = (uint64_t)v.template at<int64_t>(p, p.r_a, r);
    uint64_t pb = (uint64_t)v.template at<int64_t>(p, p.r_b, r);
    uint64_t dd = (uint64_t)v.template at<int64_t>(p, p.r_d, r);
    uint64_t tt = (uint64_t)v.template at<int64_t>(p, p.r_t, r);
    uint64_t f0 = (uint64_t)p.ac[2][0] + (uint64_t)p.as[2][0] * dd;
    uint64_t f1 = (uint64_t)p.ac[3][1] + (uint64_t)p.as[3][1] * tt;
    uint64_t dp = pb * f0;
    x[0] = qa;
    x[1] = pb;
    x[2] = dp;
    x[3] = dp * f1;
    x[4] = 1;
    return true;
  }
};

// key column (int64 or int32), one int64 value column, any ops, no filter.
template <class KT>
struct ShapeKV {
  template <int A, class V>
  __device__ __forceinline__ static bool row(const GbParams& p, const V& v, int r, uint64_t& ek,
                                             uint64_t (&x)[A]) {
    int64_t key = (int64_t)v.template at<KT>(p, p.key_col[0], r);
    int64_t val = v.template at<int64_t>(p, p.r_a, r);
    ek = (uint64_t)key ^ KEY_FLIP;
#pragma unroll
    for (int a = 0; a < A; ++a)
      if (a < p.n_aggs) x[a] = agg_encode(p.aop[a], val);
    return true;
  }
};

// -------------------------------------------------------------- table ops

template <int A>
__device__ __forceinline__ void apply_global(const GbParams& p, unsigned long long* w,
                                             const uint64_t (&x)[A]) {
#pragma unroll
  for (int a = 0; a < A; ++a) {
    if (a < p.n_aggs) {
      if ((p.umax_mask >> a) & 1u)
        atomicMax(w + a, (unsigned long long)x[a]);
      else
        atomicAdd(w + a, (unsigned long long)x[a]);
    }
  }
}

// Insert-or-accumulate into the global table; bounded linear probing.
template <int A>
__device__ __forceinline__ bool gtab_update_inl(const GbParams& p, uint64_t ek,
                                                const uint64_t (&x)[A]) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  uint64_t s = slot_of(ek, p.log2_slots);
  for (uint32_t i = 0; i < p.max_probe; ++i) {
    uint64_t k = ld_relaxed(p.tkeys + s);
    if (k == 0) {
      k = atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek);
      if (k == 0) k = ek;
    }
    if (k == ek) {
      apply_global<A>(p, p.taggs + s * (uint64_t)p.n_aggs, x);
      return true;
    }
    s = (s + 1) & mask;
  }
  atomicOr(&p.hdr->overflow, 1u);
  return false;
}

// Out-of-line copy for the cold paths (spills and end-of-kernel merges).
template <int A>
__device__ __noinline__ bool gtab_update(const GbParams& p, uint64_t ek, const uint64_t (&x)[A]) {
  return gtab_update_inl<A>(p, ek, x);
}

// Key set for the exact distinct count: true when this call claimed the key.
__device__ __noinline__ void gset_insert(const GbParams& p, uint64_t ek) {
  const uint64_t mask = (1ull << p.log2_slots) - 1;
  uint64_t s = slot_of(ek, p.log2_slots);
  for (uint32_t i = 0; i < p.max_probe; ++i) {
    uint64_t k = ld_relaxed(p.tkeys + s);
    if (k == ek) return;
    if (k == 0) {
      k = atomicCAS((unsigned long long*)(p.tkeys + s), 0ull, (unsigned long long)ek);
      if (k == 0) {
        atomicAdd(&p.hdr->aux, 1ull);
        return;
      }
      if (k == ek) return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(&p.hdr->overflow, 1u);
}

template <int A>
__device__ __forceinline__ void side_update(const GbParams& p, const uint64_t (&x)[A]) {
  atomicAdd(&p.hdr->n_side, 1ull);
  apply_global<A>(p, p.hdr->side_aggs, x);
}

// ---------------------------------------------------------------- backends

template <int A>
struct BeGlobal {
  static constexpr int ID = relhost::K_GB_GLOBAL;
  __host__ __device__ static uint64_t bytes(int, uint32_t) { return 0; }
  __device__ void bind(uint8_t*, const GbParams&) {}
  __device__ void init(const GbParams&) {}
  __device__ __forceinline__ void update(const GbParams& p, uint64_t ek, const uint64_t (&x)[A]) {
    gtab_update_inl<A>(p, ek, x);
  }
  __device__ void flush(const GbParams&) {}
};

// Up to TINY_SLOTS keys per CTA; thread-private accumulator columns
// acc[slot][a][thread] in shared memory, reduced and merged at the end.
template <int A>
struct BeTiny {
  static constexpr int ID = relhost::K_GB_TINY;
  uint64_t* tk;
  uint64_t* acc;
  uint64_t* res;
  __host__ __device__ static uint64_t bytes(int, uint32_t) {
    return 8ull * (TINY_SLOTS + (uint64_t)TINY_SLOTS * A * GB_BLOCK + TINY_SLOTS * A);
  }
  __device__ void bind(uint8_t* area, const GbParams&) {
    tk = (uint64_t*)area;
    acc = tk + TINY_SLOTS;
    res = acc + (size_t)TINY_SLOTS * A * GB_BLOCK;
  }
  __device__ void init(const GbParams&) {
    for (int i = threadIdx.x; i < TINY_SLOTS * (1 + A * GB_BLOCK); i += GB_BLOCK) tk[i] = 0;
  }
  __device__ __forceinline__ void update(const GbParams& p, uint64_t ek, const uint64_t (&x)[A]) {
    uint32_t s = small_slot_of(ek, TINY_SLOTS - 1);
#pragma unroll 1
    for (int i = 0; i < TINY_SLOTS; ++i) {
      uint64_t k = *(volatile uint64_t*)(tk + s);
      if (k == 0) {
        k = atomicCAS((unsigned long long*)(tk + s), 0ull, (unsigned long long)ek);
        if (k == 0) k = ek;
      }
      if (k == ek) {
        uint64_t* w = acc + (size_t)s * A * GB_BLOCK + threadIdx.x;
#pragma unroll
        for (int a = 0; a < A; ++a) {
          if (a < p.n_aggs) {
            uint64_t o = w[a * GB_BLOCK];
            w[a * GB_BLOCK] = ((p.umax_mask >> a) & 1u) ? (o > x[a] ? o : x[a]) : o + x[a];
          }
        }
        return;
      }
      s = (s + 1) & (TINY_SLOTS - 1);
    }
    gtab_update<A>(p, ek, x);
  }
  __device__ void flush(const GbParams& p) {
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int pr = warp; pr < TINY_SLOTS * A; pr += GB_BLOCK / 32) {
      const int s = pr / A, a = pr % A;
      if (tk[s] == 0 || a >= p.n_aggs) continue;
      const bool um = (p.umax_mask >> a) & 1u;
      const uint64_t* w = acc + ((size_t)s * A + a) * GB_BLOCK;
      uint64_t v = 0;
      for (int t = lane; t < GB_BLOCK; t += 32) {
        uint64_t y = w[t];
        v = um ? (v > y ? v : y) : v + y;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        uint64_t y = __shfl_xor_sync(0xffffffffu, v, o);
        v = um ? (v > y ? v : y) : v + y;
      }
      if (lane == 0) res[s * A + a] = v;
    }
    __syncthreads();
    if (threadIdx.x < TINY_SLOTS && tk[threadIdx.x] != 0) {
      uint64_t x[A];
#pragma unroll
      for (int a = 0; a < A; ++a) x[a] = res[threadIdx.x * A + a];
      gtab_update<A>(p, tk[threadIdx.x], x);
    }
  }
};

// CTA-shared table of smem_slots keys with shared-memory atomics.
template <int A>
struct BeShared {
  static constexpr int ID = relhost::K_GB_SHARED;
  uint64_t* tk;
  unsigned long long* acc;
  uint32_t mask;
  __host__ __device__ static uint64_t bytes(int, uint32_t slots) {
    return 8ull * slots * (1 + A);
  }
  __device__ void bind(uint8_t* area, const GbParams& p) {
    tk = (uint64_t*)area;
    acc = (unsigned long long*)(tk + p.smem_slots);
    mask = p.smem_slots - 1;
  }
  __device__ void init(const GbParams& p) {
    for (uint32_t i = threadIdx.x; i < p.smem_slots * (1 + A); i += GB_BLOCK) tk[i] = 0;
  }
  __device__ __forceinline__ void update(const GbParams& p, uint64_t ek, const uint64_t (&x)[A]) {
    uint32_t s = small_slot_of(ek, mask);
#pragma unroll 1
    for (int i = 0; i < SHARED_PROBES; ++i) {
      uint64_t k = *(volatile uint64_t*)(tk + s);
      if (k == 0) {
        k = atomicCAS((unsigned long long*)(tk + s), 0ull, (unsigned long long)ek);
        if (k == 0) k = ek;
      }
      if (k == ek) {
        unsigned long long* w = acc + (size_t)s * A;
#pragma unroll
        for (int a = 0; a < A; ++a) {
          if (a < p.n_aggs) {
            if ((p.umax_mask >> a) & 1u)
              atomicMax(w + a, (unsigned long long)x[a]);
            else
              atomicAdd(w + a, (unsigned long long)x[a]);
          }
        }
        return;
      }
      s = (s + 1) & mask;
    }
    gtab_update<A>(p, ek, x);
  }
  __device__ void flush(const GbParams& p) {
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < p.smem_slots; s += GB_BLOCK) {
      uint64_t k = tk[s];
      if (k == 0) continue;
      uint64_t x[A];
#pragma unroll
      for (int a = 0; a < A; ++a) x[a] = acc[(size_t)s * A + a];
      gtab_update<A>(p, k, x);
    }
  }
};

// Distinct-key counting: a CTA-shared key filter in front of the global set.
template <int A>
struct BeKeySet {
  static constexpr int ID = relhost::K_GB_KEYSET;
  uint64_t* tk;
  uint32_t mask;
  __host__ __device__ static uint64_t bytes(int, uint32_t slots) { return 8ull * slots; }
  __device__ void bind(uint8_t* area, const GbParams& p) {
    tk = (uint64_t*)area;
    mask = p.smem_slots - 1;
  }
  __device__ void init(const GbParams& p) {
    for (uint32_t i = threadIdx.x; i < p.smem_slots; i += GB_BLOCK) tk[i] = 0;
  }
  __device__ __forceinline__ void update(const GbParams& p, uint64_t ek, const uint64_t (&)[A]) {
    uint32_t s = small_slot_of(ek, mask);
#pragma unroll 1
    for (int i = 0; i < SHARED_PROBES; ++i) {
      uint64_t k = *(volatile uint64_t*)(tk + s);
      if (k == ek) return;  // this CTA already sent the key to the global set
      if (k == 0) {
        k = atomicCAS((unsigned long long*)(tk + s), 0ull, (unsigned long long)ek);
        if (k == 0) break;  // first sight in this CTA
        if (k == ek) return;
      }
      s = (s + 1) & mask;
    }
    gset_insert(p, ek);
  }
  __device__ void flush(const GbParams&) {}
};

// -------------------------------------------------------------- main kernel

template <class Shape, class BE, int A, bool KEYSET, class V>
__device__ __forceinline__ void run_rows(const GbParams& p, BE& be, const V& v, int nrows) {
#pragma unroll 2
  for (int r = threadIdx.x; r < nrows; r += GB_BLOCK) {
    uint64_t ek;
    uint64_t x[A];
    if (!Shape::template row<A>(p, v, r, ek, x)) continue;
    if (ek == 0) {  // the key INT64_MIN: side accumulator
      if (KEYSET)
        atomicAdd(&p.hdr->n_side, 1ull);
      else
        side_update<A>(p, x);
      continue;
    }
    be.update(p, ek, x);
  }
}

template <class Shape, class BE, int A, bool KEYSET, bool USE_TMA>
__global__ void __launch_bounds__(GB_BLOCK) gb_main(const __grid_constant__ GbParams p) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* full = (uint64_t*)smem;  // GB_STAGES mbarriers
  uint8_t* area = smem + 128;
  BE be;
  be.bind(area, p);
  be.init(p);
  uint8_t* stages = area + ((BE::bytes(p.n_aggs, p.smem_slots) + 127) & ~127ull);

  const int64_t T = p.tile_rows;
  const int64_t n_tiles = USE_TMA ? p.n_rows / T : (p.n_rows + T - 1) / T;
  const int64_t mine = n_tiles > (int64_t)blockIdx.x
                           ? (n_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1
                           : 0;
  uint64_t policy = 0;
  if (USE_TMA && threadIdx.x == 0) {
    for (int s = 0; s < GB_STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    policy = l2_evict_first_policy();
  }
  __syncthreads();

  auto issue = [&](int64_t k, int s) {
    const int64_t t = (int64_t)blockIdx.x + k * (int64_t)gridDim.x;
    mbar_arrive_expect_tx(&full[s], p.stage_bytes);
    uint8_t* dst = stages + (size_t)s * p.stage_bytes;
    for (int c = 0; c < p.n_cols; ++c) {
      const uint32_t nb = (uint32_t)(T * p.csize[c]);
      bulk_g2s(dst + p.stage_off[c], p.col[c] + t * T * p.csize[c], nb, &full[s], policy);
    }
  };

  bool stopped = false;
  if (USE_TMA) {
    if (threadIdx.x == 0)
      for (int64_t k = 0; k < mine && k < GB_STAGES; ++k) issue(k, (int)k);
    int64_t k = 0;
    for (; k < mine; ++k) {
      const int s = (int)(k % GB_STAGES);
      const uint32_t par = (uint32_t)((k / GB_STAGES) & 1);
      const bool ok = mbar_wait_bounded(&full[s], par, WAIT_LIMIT_NS);
      if (ok)
        run_rows<Shape, BE, A, KEYSET>(p, be, SmemView{stages + (size_t)s * p.stage_bytes}, (int)T);
      else
        atomicOr(&p.hdr->timeout, 1u);
      int stop = !ok;
      if (threadIdx.x == 0) stop |= ld_relaxed_u32(&p.hdr->overflow) != 0;
      if (__syncthreads_or(stop)) {
        stopped = true;
        break;
      }
      if (threadIdx.x == 0 && k + GB_STAGES < mine) issue(k + GB_STAGES, s);
    }
    if (stopped) {
      // let the copies already issued land before the CTA's shared memory goes away
      if (threadIdx.x == 0)
        for (int64_t j = k + 1; j < mine && j < k + GB_STAGES; ++j)
          mbar_wait_bounded(&full[j % GB_STAGES], (uint32_t)((j / GB_STAGES) & 1), WAIT_LIMIT_NS);
      __syncthreads();
      return;
    }
    // rows after the last full tile: one CTA, straight from global memory
    const int64_t tail0 = n_tiles * T;
    if (tail0 < p.n_rows && blockIdx.x == (unsigned)(n_tiles % gridDim.x))
      run_rows<Shape, BE, A, KEYSET>(p, be, GlobalView{tail0}, (int)(p.n_rows - tail0));
  } else {
    for (int64_t k = 0; k < mine; ++k) {
      const int64_t t = (int64_t)blockIdx.x + k * (int64_t)gridDim.x;
      const int64_t r0 = t * T;
      const int nrows = (int)(p.n_rows - r0 < T ? p.n_rows - r0 : T);
      run_rows<Shape, BE, A, KEYSET>(p, be, GlobalView{r0}, nrows);
      int stop = 0;
      if (threadIdx.x == 0) stop = ld_relaxed_u32(&p.hdr->overflow) != 0;
      if (__syncthreads_or(stop)) return;
    }
  }
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

// ------------------------------------------------------------------ launch

int gb_shape_width(int shape) {
  return shape == SHAPE_Q1 ? 5 : (shape == SHAPE_KV64 || shape == SHAPE_KV32) ? 4 : REL_MAX_AGGS;
}

uint64_t gb_backend_smem_bytes(int mode, int shape, uint32_t smem_slots) {
  const uint64_t A = (uint64_t)gb_shape_width(shape);
  switch (mode) {
    case MODE_TINY: return 8ull * (TINY_SLOTS + TINY_SLOTS * A * GB_BLOCK + TINY_SLOTS * A);
    case MODE_SHARED: return 8ull * smem_slots * (1 + A);
    case MODE_KEYSET: return 8ull * smem_slots;
    default: return 0;
  }
}

namespace {

template <class Shape, class BE, int A, bool KEYSET, bool TMA>
rel_status launch_one(const GbParams& p, cudaStream_t st) {
  auto kern = gb_main<Shape, BE, A, KEYSET, TMA>;
  const uint64_t be_bytes = (BE::bytes(p.n_aggs, p.smem_slots) + 127) & ~127ull;
  const size_t smem = 128 + be_bytes + (TMA ? (size_t)GB_STAGES * p.stage_bytes : 0);
  if (smem > 227 * 1024) {
    relhost::set_error("group-by: %zu bytes of shared memory exceed the limit", smem);
    return REL_E_UNSUPPORTED;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaFuncSetAttribute(group-by)");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GB_BLOCK, smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "occupancy(group-by)");
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (p.n_rows + p.tile_rows - 1) / p.tile_rows;
  int64_t grid = (int64_t)relhost::device_sms() * per_sm;
  if (grid > tiles) grid = tiles > 0 ? tiles : 1;
  relhost::launch_begin(BE::ID, st);
  kern<<<(unsigned)grid, GB_BLOCK, smem, st>>>(p);
  relhost::launch_end(BE::ID, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return relhost::cuda_fail(e, "launch(group-by)");
  return REL_OK;
}

template <class Shape, int A>
rel_status launch_mode(const GbParams& p, int mode, bool tma, cudaStream_t st) {
#define REL_GB_CASE(BE, KS)                                                         \
  return tma ? launch_one<Shape, BE<A>, A, KS, true>(p, st)                         \
             : launch_one<Shape, BE<A>, A, KS, false>(p, st)
  switch (mode) {
    case MODE_TINY: REL_GB_CASE(BeTiny, false);
    case MODE_SHARED: REL_GB_CASE(BeShared, false);
    case MODE_KEYSET: REL_GB_CASE(BeKeySet, true);
    default: REL_GB_CASE(BeGlobal, false);
  }
#undef REL_GB_CASE
}

}  // namespace

rel_status gb_launch_main(const GbParams& p, int shape, int mode, bool use_tma, cudaStream_t st) {
  if (p.n_rows == 0) return REL_OK;
  switch (shape) {
    case SHAPE_Q1: return launch_mode<ShapeQ1, 5>(p, mode, use_tma, st);
    case SHAPE_KV64: return launch_mode<ShapeKV<int64_t>, 4>(p, mode, use_tma, st);
    case SHAPE_KV32: return launch_mode<ShapeKV<int32_t>, 4>(p, mode, use_tma, st);
    default: return launch_mode<ShapeGeneric, REL_MAX_AGGS>(p, mode, use_tma, st);
  }
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
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return relhost::cuda_fail(e, "launch(compact)");
  return REL_OK;
}

}  // namespace rel
