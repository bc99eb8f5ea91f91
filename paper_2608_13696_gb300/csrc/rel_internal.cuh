// Internal device utilities shared by the group-by and join kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rel.h"

namespace rel {

// Stored keys are  key ^ KEY_FLIP  so that a zero-filled table is empty.  The
// one key that stores as 0 (INT64_MIN) never enters a table: it takes a side
// path (group-by: a side accumulator; join: a side list of build rows).
constexpr uint64_t KEY_FLIP = 0x8000000000000000ull;

// Zero-initialised aggregate words: SUM and COUNT add; MIN and MAX keep the
// unsigned maximum of an order-mapped input.  MAX maps v -> v ^ 2^63 (signed
// order becomes unsigned order, INT64_MIN -> 0); MIN maps v -> v ^ (2^63 - 1)
// (order reversed, INT64_MAX -> 0).  So 0 is the identity of every word and
// a table can be cleared with a memset.
constexpr uint64_t MIN_FLIP = 0x7FFFFFFFFFFFFFFFull;
constexpr uint64_t MAX_FLIP = 0x8000000000000000ull;

enum : int { KIND_ADD = 0, KIND_UMAX = 1 };

__host__ __device__ __forceinline__ int agg_kind(int op) {
  return (op == REL_MIN || op == REL_MAX) ? KIND_UMAX : KIND_ADD;
}

__device__ __forceinline__ uint64_t agg_encode(int op, int64_t v) {
  switch (op) {
    case REL_COUNT: return 1ull;
    case REL_MIN: return (uint64_t)v ^ MIN_FLIP;
    case REL_MAX: return (uint64_t)v ^ MAX_FLIP;
    default: return (uint64_t)v;
  }
}

__device__ __forceinline__ int64_t agg_decode(int op, uint64_t w) {
  switch (op) {
    case REL_MIN: return (int64_t)(w ^ MIN_FLIP);
    case REL_MAX: return (int64_t)(w ^ MAX_FLIP);
    default: return (int64_t)w;
  }
}

// Slot hash: multiplicative (Fibonacci) hashing, top bits of ek * 2^64/phi.
__device__ __forceinline__ uint64_t slot_of(uint64_t ek, int log2_slots) {
  return (ek * 0x9E3779B97F4A7C15ull) >> (64 - log2_slots);
}

// Hash for the small per-CTA tables: the key folded to 32 bits, then 32-bit
// multiplicative hashing (one IMAD) -- cheap, and independent of slot_of.
__device__ __forceinline__ uint32_t small_slot_of(uint64_t ek, uint32_t mask, uint32_t mult) {
  const uint32_t f = (uint32_t)ek ^ (uint32_t)(ek >> 32);
  return __umulhi(f, mult) & mask;
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 64-bit add to a shared-memory word from two native 32-bit atomics.  A
// 64-bit shared-memory atomicAdd is far slower than a 32-bit one on this
// GPU -- hundreds of times under same-address contention, as on hot keys --
// so the low half is added atomically (returning its old value), and a
// wrap of the low half carries into the high half.  Every wrap is seen by
// exactly the thread whose add caused it, so the final 64-bit word is the
// exact sum mod 2^64.  Read the word only after the adds (a barrier).
__device__ __forceinline__ void sadd64(unsigned long long* w, uint64_t x) {
  unsigned int* h = (unsigned int*)w;  // little-endian: h[0] low, h[1] high
  const unsigned int lo = (unsigned int)x;
  const unsigned int old = atomicAdd(h, lo);
  const unsigned int hi = (unsigned int)(x >> 32) + ((unsigned int)(old + lo) < old ? 1u : 0u);
  if (hi) atomicAdd(h + 1, hi);
}

// ------------------------------------------------------------ mbarrier / TMA

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of an mbarrier, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// L2 policy for data that should stay resident (a hash table probed while a
// column streams past with evict-first loads).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// One-dimensional bulk copy global -> shared (the TMA engine), completing on
// an mbarrier.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// Shared-memory access by 32-bit shared-window address (ordered with every
// other memory access of the thread).
__device__ __forceinline__ uint64_t lds64(uint32_t a) {
  uint64_t v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts64(uint32_t a, uint64_t v) {
  asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

// Barrier among the first `count` threads of the CTA (named barrier 1).
__device__ __forceinline__ void named_sync(uint32_t count) {
  asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}

// ------------------------------------------------------------------ status

// Device-visible status words at the start of every workspace.
struct alignas(128) WsHeader {
  unsigned long long n_out;     // output cursor (groups / pairs)
  unsigned long long n_side;    // group-by: rows whose key is INT64_MIN; join: side rows
  unsigned int overflow;        // a bounded table probe gave up
  unsigned int timeout;         // a bounded wait gave up
  unsigned long long aux;       // spare counter (distinct keys in the exact pre-pass)
  unsigned long long side_aggs[REL_MAX_AGGS];
  unsigned int dups;            // join build: some key occurs twice
  unsigned int pad;
};
static_assert(sizeof(WsHeader) <= 256, "header fits in 256 bytes");
constexpr uint64_t HEADER_BYTES = 256;

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s for any single wait
// the same limit under the test hook REL_PLAN_TEST_STALL
constexpr uint64_t TEST_WAIT_LIMIT_NS = 20000000ull;  // 20 ms

}  // namespace rel

// ------------------------------------------------------------- host helpers

namespace relhost {
void set_error(const char* fmt, ...);
// A workspace must start on a 256-byte boundary (every cudaMalloc and
// PyTorch allocation does): tables in it are read with 32-byte vector loads.
inline bool ws_unaligned(const void* ws) { return ws && ((uintptr_t)ws & 255u) != 0; }
rel_status cuda_fail(cudaError_t e, const char* what);
void count_launch(unsigned n = 1);
int device_sms();

// Kernel ids for launch counting and event timing.
enum KernelId : int {
  K_GB_LAYERED = 0,
  K_GB_KEYSET = 1,
  K_GB_COMPACT = 2,
  K_JOIN_BUILD = 3,
  K_JOIN_PROBE = 4,
  K_JOIN_COUNT = 5,
  K_SKETCH = 6,
  K_GB_REGS = 7,
  K_GB_PHIST = 8,
  K_GB_PSCAN = 9,
  K_GB_PSCATTER = 10,
  K_GB_PAGG = 11,
  K_MLP = 12,
  K_BATCH_A = 13,
  K_BATCH_B = 14,
  K_GB_STREAM = 15,
  K_HLL = 16,
  K_GB_PL2 = 17,
  K_COUNT_IDS = 18
};
// Bracket one launch: counts it and, while profiling, records events.
void launch_begin(int kernel_id, cudaStream_t st);
void launch_end(int kernel_id, cudaStream_t st);
}  // namespace relhost
