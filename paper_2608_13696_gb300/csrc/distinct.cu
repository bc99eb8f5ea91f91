// Exact distinct count of one key column: the plain form's sizing pre-pass
// ("count the groups exactly, then size the table"), for one int32 / int64
// key column without a filter.
//
// The paper finds these hash-table kernels bound by instruction issue and
// memory latency rather than by DRAM bandwidth (Sec. 5-6): random probes
// into a table larger than the cache, one slot per step, with a warp waiting
// for its slowest lane.  This kernel is built around the GB300's caches:
//  * the caller's first set is at most 256 MB (measured on 2e8-row inputs:
//    smaller first sets, nearer the L2's size, lose more to the retries of
//    inputs that overflow them than they gain); the key column streams past
//    with evict-first loads and the buckets are marked evict-last;
//  * a key's home is a 32-byte bucket of four slots, read with one 256-bit
//    load, so almost every probe resolves in one L2 request and one compare
//    chain (the paper's recommendation: fewer instructions per memory
//    access);
//  * an optional per-CTA direct-mapped filter of recently sent keys in shared
//    memory drops repeats before they reach the set (off by default: the
//    buckets of frequent keys come from L1 anyway);
//  * every thread issues the bucket loads of several unfiltered rows before
//    resolving any (memory-level parallelism), and the kernel runs at high
//    occupancy so that many chunks of keys are in flight per SM;
//  * keys missing from their home bucket are queued per warp and inserted in
//    one converged pass per chunk, instead of one divergent pass per row slot
//    in which a lane or two walk their probe sequence while the rest wait
//    (2e8-row Zipf column: 1.56 -> 1.19 ms);
//  * when more distinct keys exist than one L2-sized set holds, the host runs
//    several passes, each counting the keys of one hash range in its own set.
// Insert-only linear probing with compare-and-swap claims: every thread that
// inserts key k walks k's slots in the same order and stops at the first slot
// holding k or claims the first empty one, so each distinct key is claimed
// exactly once; the claims are the count.
#include <cmath>

#include "distinct.cuh"

namespace rel {

namespace {

constexpr int DS_BLOCK = 256;
constexpr int DS_U = 8;      // keys per thread per chunk
constexpr int DS_GROUP = 4;  // keys whose home buckets are in flight together

__device__ __forceinline__ uint64_t ds_hash(uint64_t ek) { return ek * 0x9E3779B97F4A7C15ull; }

// Pass of a key under an n-way hash split (a multiplier independent of ds_hash).
__device__ __forceinline__ uint32_t ds_pass(uint64_t ek, uint32_t n_pass) {
  return (uint32_t)__umul64hi(ek * 0xC2B2AE3D27D4EB4Full, (uint64_t)n_pass);
}

// A bucket through L1: a stale copy only ever shows fewer keys than the set
// holds (slots go from empty to a key, never back), which costs at most a
// compare-and-swap that fails -- and the buckets of frequent keys then come
// from L1 instead of hammering one L2 sector.
// In L2 the set is marked evict-last, so the streamed keys (evict-first)
// displace it last.
__device__ __forceinline__ void ld_bucket(const uint64_t* b, uint64_t (&s)[DS_BUCKET_SLOTS],
                                          uint64_t pol) {
  asm volatile("ld.global.L2::cache_hint.v4.u64 {%0, %1, %2, %3}, [%4], %5;"
               : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3])
               : "l"(b), "l"(pol));
}

// A bucket from L2, bypassing L1: the fresh view the insert path works on.
__device__ __forceinline__ void ld_bucket_l2(const uint64_t* b, uint64_t (&s)[DS_BUCKET_SLOTS]) {
  asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3])
               : "l"(b));
}

// The rare path of a key whose home bucket (as loaded) does not hold it:
// walk its probe sequence from bucket b, claiming the first empty slot with a
// compare-and-swap.  Returns 1 when this thread claimed the key, 0 when it
// was present, -1 when DS_MAX_PROBE buckets held neither it nor a gap.  Kept
// out of line so that the unrolled fast path stays small.
__device__ __noinline__ int ds_insert(const DistinctParams& p, uint64_t ek, uint64_t b) {
  for (int i = 0; i < DS_MAX_PROBE; ++i) {
    uint64_t s[DS_BUCKET_SLOTS];
    ld_bucket_l2(p.set + b * DS_BUCKET_SLOTS, s);
    if (s[0] == ek || s[1] == ek || s[2] == ek || s[3] == ek) return 0;
#pragma unroll
    for (int t = 0; t < DS_BUCKET_SLOTS; ++t) {
      if (s[t] != 0) continue;
      const unsigned long long old =
          atomicCAS((unsigned long long*)(p.set + b * DS_BUCKET_SLOTS + t), 0ull,
                    (unsigned long long)ek);
      if (old == 0) return 1;
      if (old == ek) return 0;
      // another key took the slot: go on with the next one
    }
    b = b + 1 == p.n_buckets ? 0 : b + 1;
  }
  return -1;
}

template <class KT>
struct Vec16;
template <>
struct Vec16<int64_t> {
  static constexpr int PER = 2;
  __device__ __forceinline__ static void load(const int64_t* p, uint64_t* out) {
    const longlong2 v = __ldcs((const longlong2*)p);
    out[0] = (uint64_t)v.x ^ KEY_FLIP;
    out[1] = (uint64_t)v.y ^ KEY_FLIP;
  }
};
template <>
struct Vec16<int32_t> {
  static constexpr int PER = 4;
  __device__ __forceinline__ static void load(const int32_t* p, uint64_t* out) {
    const int4 v = __ldcs((const int4*)p);
    out[0] = (uint64_t)(int64_t)v.x ^ KEY_FLIP;
    out[1] = (uint64_t)(int64_t)v.y ^ KEY_FLIP;
    out[2] = (uint64_t)(int64_t)v.z ^ KEY_FLIP;
    out[3] = (uint64_t)(int64_t)v.w ^ KEY_FLIP;
  }
};

// Keys of chunk `base` for this thread: rows base + v * PER * DS_BLOCK +
// PER * tid + e (a warp reads 512 contiguous bytes per vector load); rows past
// the end are marked invalid.
template <class KT, bool VEC>
__device__ __forceinline__ void load_chunk(const KT* keys, int64_t n, int64_t base,
                                           uint64_t (&ek)[DS_U], uint32_t& valid) {
  constexpr int PER = Vec16<KT>::PER;
  const int tid = threadIdx.x;
  if (VEC && base + (int64_t)DS_BLOCK * DS_U <= n) {
#pragma unroll
    for (int v = 0; v < DS_U / PER; ++v)
      Vec16<KT>::load(keys + base + (int64_t)v * PER * DS_BLOCK + PER * tid, ek + v * PER);
    valid = (1u << DS_U) - 1;
    return;
  }
  valid = 0;
#pragma unroll
  for (int j = 0; j < DS_U; ++j) {
    const int64_t r = base + (int64_t)(j / PER) * PER * DS_BLOCK + PER * tid + (j % PER);
    ek[j] = 0;
    if (r < n) {
      ek[j] = (uint64_t)(int64_t)keys[r] ^ KEY_FLIP;
      valid |= 1u << j;
    }
  }
}

// Per warp, the keys whose home bucket (as loaded) held neither them nor a
// gap are queued in shared memory and inserted together once per chunk: one
// pass of the out-of-line insert path with the warp's misses spread over its
// lanes instead of one divergent pass per row slot with a lane or two in it.
struct DsMiss {
  uint64_t key, bucket;
};
constexpr int DS_WARPS = DS_BLOCK / 32;
constexpr int DS_QUEUE = 32 * DS_U;  // every row of a warp's chunk

template <class KT, bool FILTER>
__global__ void __launch_bounds__(DS_BLOCK, 3) distinct_k(const __grid_constant__ DistinctParams p) {
  extern __shared__ __align__(16) uint64_t filt[];
  __shared__ DsMiss queue[DS_WARPS][DS_QUEUE];
  const int lane = threadIdx.x & 31;
  DsMiss* const wq = queue[threadIdx.x >> 5];
  const uint32_t fmask = p.filter_slots - 1;
  if (FILTER)
    for (uint32_t i = threadIdx.x; i < p.filter_slots; i += DS_BLOCK) filt[i] = 0;
  __syncthreads();
  const KT* keys = (const KT*)p.keys;
  const int64_t n = p.n_rows;
  constexpr int64_t CH = (int64_t)DS_BLOCK * DS_U;
  const bool vec = (uintptr_t)keys % 16 == 0;
  unsigned long long claims = 0, side = 0;
  const uint64_t pol = l2_evict_last_policy();
  for (int64_t base = (int64_t)blockIdx.x * CH; base < n; base += (int64_t)gridDim.x * CH) {
    uint64_t ek[DS_U];
    uint32_t ok;
    if (vec) load_chunk<KT, true>(keys, n, base, ek, ok);
    else load_chunk<KT, false>(keys, n, base, ek, ok);
    // the set's overflow flag, read now and tested after the chunk (its
    // latency hides behind the chunk's work)
    const uint32_t ovf = lane == 0 ? ld_relaxed_u32(&p.hdr->overflow) : 0u;
    uint32_t need = 0;
#pragma unroll
    for (int j = 0; j < DS_U; ++j) {
      if (!(ok >> j & 1)) continue;
      if (ek[j] == 0) {  // INT64_MIN: counted apart, once
        side += p.pass == 0;
        continue;
      }
      if (p.n_pass > 1 && ds_pass(ek[j], p.n_pass) != p.pass) continue;
      if (FILTER) {
        uint64_t* f = filt + ((uint32_t)(ds_hash(ek[j]) >> 24) & fmask);
        if (*f == ek[j]) continue;  // this CTA has sent the key already
        *f = ek[j];
      }
      need |= 1u << j;
    }
    // home buckets of DS_GROUP keys in flight together, then resolved; a
    // key not in its home bucket goes to the warp's queue
    uint32_t miss = 0;
#pragma unroll
    for (int g = 0; g < DS_U; g += DS_GROUP) {
      if (!(need >> g & ((1u << DS_GROUP) - 1))) continue;
      uint64_t s[DS_GROUP][DS_BUCKET_SLOTS];
#pragma unroll
      for (int q = 0; q < DS_GROUP; ++q) {
        const uint64_t b = __umul64hi(ds_hash(ek[g + q]), p.n_buckets);
        if (need >> (g + q) & 1) ld_bucket(p.set + b * DS_BUCKET_SLOTS, s[q], pol);
      }
#pragma unroll
      for (int q = 0; q < DS_GROUP; ++q) {
        const uint64_t k = ek[g + q];
        if ((need >> (g + q) & 1) && s[q][0] != k && s[q][1] != k && s[q][2] != k && s[q][3] != k)
          miss |= 1u << (g + q);
      }
    }
    bool bad = false;
    if (__any_sync(0xffffffffu, miss != 0)) {
      const uint32_t nm = __popc(miss);
      uint32_t at = nm;  // inclusive prefix of the lanes' miss counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, at, o);
        if (lane >= o) at += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, at, 31);
      at -= nm;
#pragma unroll
      for (int j = 0; j < DS_U; ++j)
        if (miss >> j & 1) wq[at++] = DsMiss{ek[j], __umul64hi(ds_hash(ek[j]), p.n_buckets)};
      __syncwarp();
      for (uint32_t i = lane; i < total; i += 32) {
        const int r = ds_insert(p, wq[i].key, wq[i].bucket);
        claims += r > 0;
        bad |= r < 0;
      }
      __syncwarp();
    }
    if (bad) atomicOr(&p.hdr->overflow, 1u);
    // once the set overflowed the count is void (the caller retries with more
    // room): stop reading, uniformly per warp
    if (__shfl_sync(0xffffffffu, ovf, 0) || __any_sync(0xffffffffu, bad)) break;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    claims += __shfl_xor_sync(0xffffffffu, claims, o);
    side += __shfl_xor_sync(0xffffffffu, side, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (claims) atomicAdd(&p.hdr->aux, claims);
    if (side) atomicAdd(&p.hdr->n_side, side);
  }
}

// The MurmurHash3 64-bit finalizer (Appleby): a bijective mix of the key.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xFF51AFD7ED558CCDull;
  k ^= k >> 33;
  k *= 0xC4CEB9FE1A85EC53ull;
  k ^= k >> 33;
  return k;
}

template <class KT>
__global__ void __launch_bounds__(DS_BLOCK) hll_k(const KT* __restrict__ keys, int64_t n,
                                                  uint32_t* __restrict__ regs) {
  __shared__ uint32_t r[HLL_REGS];
  for (int i = threadIdx.x; i < HLL_REGS; i += DS_BLOCK) r[i] = 0;
  __syncthreads();
  constexpr int64_t CH = (int64_t)DS_BLOCK * DS_U;
  const bool vec = (uintptr_t)keys % 16 == 0;
  for (int64_t base = (int64_t)blockIdx.x * CH; base < n; base += (int64_t)gridDim.x * CH) {
    uint64_t ek[DS_U];
    uint32_t ok;
    if (vec) load_chunk<KT, true>(keys, n, base, ek, ok);
    else load_chunk<KT, false>(keys, n, base, ek, ok);
#pragma unroll
    for (int j = 0; j < DS_U; ++j) {
      if (!(ok >> j & 1)) continue;
      const uint64_t h = fmix64(ek[j]);
      const uint64_t rest = h << HLL_P;
      const uint32_t rank = rest == 0 ? (uint32_t)(65 - HLL_P) : (uint32_t)__clzll((long long)rest) + 1u;
      uint32_t* x = r + (h >> (64 - HLL_P));
      if (rank > *(volatile uint32_t*)x) atomicMax(x, rank);  // read first: most rows do not raise it
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < HLL_REGS; i += DS_BLOCK)
    if (r[i]) atomicMax(regs + i, r[i]);
}

template <class KT, bool FILTER>
rel_status launch(const DistinctParams& p, cudaStream_t st) {
  auto kern = distinct_k<KT, FILTER>;
  const size_t smem = FILTER ? distinct_smem_bytes(p.filter_slots) : 0;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaFuncSetAttribute(distinct)");
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, DS_BLOCK, smem);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "occupancy(distinct)");
  if (occ < 1) return relhost::set_error("distinct count: kernel does not fit"), REL_E_UNSUPPORTED;
  const int64_t chunks = (p.n_rows + (int64_t)DS_BLOCK * DS_U - 1) / ((int64_t)DS_BLOCK * DS_U);
  int64_t grid = (int64_t)relhost::device_sms() * occ;
  if (grid > chunks) grid = chunks;
  if (grid < 1) grid = 1;
  relhost::launch_begin(relhost::K_GB_KEYSET, st);
  kern<<<(int)grid, DS_BLOCK, smem, st>>>(p);
  relhost::launch_end(relhost::K_GB_KEYSET, st);
  e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(distinct)");
}

}  // namespace

rel_status hll_launch(const void* keys, int key_type, int64_t n, uint32_t* regs, cudaStream_t st) {
  if (n <= 0) return REL_OK;
  if (key_type != REL_I64 && key_type != REL_I32)
    return relhost::set_error("hll: needs an int32 or int64 key"), REL_E_INVALID;
  const int64_t chunks = (n + (int64_t)DS_BLOCK * DS_U - 1) / ((int64_t)DS_BLOCK * DS_U);
  int64_t grid = (int64_t)relhost::device_sms() * 4;
  if (grid > chunks) grid = chunks;
  relhost::launch_begin(relhost::K_HLL, st);
  if (key_type == REL_I64)
    hll_k<int64_t><<<(int)grid, DS_BLOCK, 0, st>>>((const int64_t*)keys, n, regs);
  else
    hll_k<int32_t><<<(int)grid, DS_BLOCK, 0, st>>>((const int32_t*)keys, n, regs);
  relhost::launch_end(relhost::K_HLL, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(hll)");
}

double hll_estimate(const uint32_t* regs) {
  const double m = HLL_REGS;
  double sum = 0.0;
  int zeros = 0;
  for (int i = 0; i < HLL_REGS; ++i) {
    sum += std::ldexp(1.0, -(int)regs[i]);
    zeros += regs[i] == 0;
  }
  const double alpha = 0.7213 / (1.0 + 1.079 / m);
  double e = alpha * m * m / sum;
  if (e <= 2.5 * m && zeros > 0) e = m * std::log(m / zeros);
  return e;
}

rel_status distinct_launch(const DistinctParams& p, int key_type, cudaStream_t st) {
  if (p.n_rows == 0) return REL_OK;
  if (!p.set || p.n_buckets < 1 || p.n_pass < 1 || p.pass >= p.n_pass ||
      (p.filter_slots & (p.filter_slots - 1)) || p.filter_slots > 16384)
    return relhost::set_error("distinct count: bad parameters"), REL_E_INVALID;
  if ((uintptr_t)p.set % 32)
    return relhost::set_error("distinct count: key set not 32-byte aligned"), REL_E_INVALID;
  const bool f = p.filter_slots != 0;
  if (key_type == REL_I64) return f ? launch<int64_t, true>(p, st) : launch<int64_t, false>(p, st);
  if (key_type == REL_I32) return f ? launch<int32_t, true>(p, st) : launch<int32_t, false>(p, st);
  return relhost::set_error("distinct count: needs an int32 or int64 key"), REL_E_INVALID;
}

}  // namespace rel
