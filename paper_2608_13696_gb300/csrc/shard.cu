// Split of a group-by's partial groups by owner rank, for the sharded
// group-by: every rank aggregates its own rows, then sends each partial group
// to the rank that owns its key, where the partials of one key are merged.
// Sum, count, min and max are associative and commutative in exact int64
// arithmetic, so the merged result equals the unsharded one bit for bit.
//
// Owner of key k: floor(h * world / 2^64) with h = (k ^ 2^63) * C mod 2^64, C
// an odd constant independent of the table hashes (the receiving rank's table
// takes its slots from the top bits of another multiplicative hash; an owner
// from those same bits would crowd every received key into one slice of it).
// Three small launches: a count per owner (a shared-memory histogram per CTA,
// then one global add per owner and CTA), the prefix of the counts, and a
// scatter in which each warp reserves its lanes' positions in their owners'
// ranges with one atomic per owner present in the warp.
#include <cstring>

#include "rel_internal.cuh"

namespace rel {

namespace {

constexpr int SH_BLOCK = 256;
constexpr uint64_t OWNER_MULT = 0xD1B54A32D192ED03ull;

__device__ __forceinline__ int owner_of(int64_t key, int world) {
  const uint64_t h = ((uint64_t)key ^ KEY_FLIP) * OWNER_MULT;
  return (int)__umul64hi(h, (uint64_t)world);
}

struct ShardParams {
  const int64_t* keys;
  const int64_t* words[REL_MAX_AGGS];
  int32_t n_words;
  int64_t n;
  int32_t world;
  unsigned long long* count;   // [world] groups per owner
  unsigned long long* cursor;  // [world] next free position per owner
  int64_t* out_keys;
  int64_t* out_words[REL_MAX_AGGS];
};

__global__ void __launch_bounds__(SH_BLOCK) shard_count_k(const __grid_constant__ ShardParams p) {
  __shared__ unsigned int h[REL_SHARD_MAX_WORLD];
  for (int i = threadIdx.x; i < p.world; i += SH_BLOCK) h[i] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * SH_BLOCK + threadIdx.x; i < p.n;
       i += (int64_t)gridDim.x * SH_BLOCK)
    atomicAdd(&h[owner_of(p.keys[i], p.world)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < p.world; i += SH_BLOCK)
    if (h[i]) atomicAdd(&p.count[i], (unsigned long long)h[i]);
}

// Exclusive prefix of the counts: owner r's range starts at cursor[r].
__global__ void shard_scan_k(const __grid_constant__ ShardParams p) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long run = 0;
    for (int r = 0; r < p.world; ++r) {
      p.cursor[r] = run;
      run += p.count[r];
    }
  }
}

__global__ void __launch_bounds__(SH_BLOCK) shard_scatter_k(const __grid_constant__ ShardParams p) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = (int64_t)blockIdx.x * SH_BLOCK; base < p.n;
       base += (int64_t)gridDim.x * SH_BLOCK) {
    const int64_t i = base + threadIdx.x;
    const bool valid = i < p.n;
    const int64_t k = valid ? p.keys[i] : 0;
    const int r = valid ? owner_of(k, p.world) : -1;
    // lanes with the same owner share one reservation
    const unsigned same = __match_any_sync(0xffffffffu, r);
    const int leader = __ffs(same) - 1;
    unsigned long long at = 0;
    if (valid && lane == leader) at = atomicAdd(&p.cursor[r], (unsigned long long)__popc(same));
    at = __shfl_sync(0xffffffffu, at, leader);
    if (!valid) continue;
    const unsigned long long pos = at + __popc(same & lt);
    p.out_keys[pos] = k;
    for (int w = 0; w < p.n_words; ++w) p.out_words[w][pos] = p.words[w][i];
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + SH_BLOCK - 1) / SH_BLOCK;
  const int64_t cap = (int64_t)relhost::device_sms() * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

}  // namespace rel

extern "C" {

uint64_t rel_shard_ws_bytes(int32_t world) {
  if (world < 1 || world > REL_SHARD_MAX_WORLD) return 0;
  return 16ull * (uint64_t)world + 256;
}

rel_status rel_shard_split(const int64_t* keys, const int64_t* const* words, int32_t n_words,
                           int64_t n, int32_t world, int64_t* out_keys, int64_t* const* out_words,
                           int64_t* counts_host, void* ws, size_t ws_bytes, void* stream) {
  if (relhost::ws_unaligned(ws))
    return relhost::set_error("shard: workspace not 256-byte aligned"), REL_E_INVALID;
  using namespace rel;
  if (world < 1 || world > REL_SHARD_MAX_WORLD)
    return relhost::set_error("shard: world must be 1..%d", REL_SHARD_MAX_WORLD), REL_E_UNSUPPORTED;
  if (n < 0 || n_words < 0 || n_words > REL_MAX_AGGS || !counts_host ||
      (n > 0 && (!keys || !out_keys || (n_words > 0 && (!words || !out_words)))))
    return relhost::set_error("shard: bad arguments"), REL_E_INVALID;
  for (int w = 0; w < n_words && n > 0; ++w)
    if (!words[w] || !out_words[w]) return relhost::set_error("shard: NULL word column"), REL_E_INVALID;
  if (!ws || ws_bytes < rel_shard_ws_bytes(world))
    return relhost::set_error("shard: workspace needs %llu bytes",
                              (unsigned long long)rel_shard_ws_bytes(world)),
           REL_E_CAPACITY;
  ShardParams p;
  std::memset(&p, 0, sizeof p);
  p.keys = keys;
  p.n_words = n_words;
  p.n = n;
  p.world = world;
  p.count = (unsigned long long*)ws;
  p.cursor = p.count + world;
  p.out_keys = out_keys;
  for (int w = 0; w < n_words; ++w) {
    p.words[w] = words[w];
    p.out_words[w] = out_words[w];
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(ws, 0, 16ull * world, st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  if (n > 0) {
    relhost::count_launch(3);
    shard_count_k<<<grid_for(n), SH_BLOCK, 0, st>>>(p);
    shard_scan_k<<<1, 32, 0, st>>>(p);
    shard_scatter_k<<<grid_for(n), SH_BLOCK, 0, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return relhost::cuda_fail(e, "launch(shard)");
  }
  unsigned long long c[REL_SHARD_MAX_WORLD];
  e = cudaMemcpyAsync(c, p.count, 8ull * world, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "reading the shard counts");
  for (int r = 0; r < world; ++r) counts_host[r] = (int64_t)c[r];
  return REL_OK;
}

}  // extern "C"
