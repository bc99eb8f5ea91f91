// Sample sketch of a group-by input (one CTA): what a planner needs to size
// the hash table and choose per-CTA layers before touching every row.
//
// Sample: all rows when n_rows <= 4096, otherwise 64 windows of 64
// consecutive rows starting at floor(w * (n_rows - 64) / 63), w = 0..63
// (windows keep runs of equal keys visible, so clustering shows).  Rows the
// filter rejects are dropped.  Over the kept keys the kernel computes:
//   * 256 HyperLogLog registers (p = 8; Flajolet, Fusy, Gandouet & Meunier
//     2007): h = splitmix64(key), register h >> 56, rank = number of leading
//     zeros of the remaining 56 bits + 1 (57 when they are all zero);
//   * exact sample statistics: distinct keys, keys seen once, runs of equal
//     consecutive keys within each window, minimum and maximum key;
//   * the 32 most frequent keys (count descending, key ascending).
// Keys are sorted in shared memory with a bitonic network (warp-local stages
// between warp barriers, CTA barriers only for the long distances); distinct
// keys and their counts come from the run starts of the sorted keys, listed
// with a prefix sum, so no thread walks a long run of equal keys.
#include "sketch.cuh"

namespace rel {

namespace {

constexpr int SK_THREADS = 1024;
constexpr int SK_N = SKETCH_SAMPLE;  // 4096

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t read_col(const SketchParams& p, int c, int64_t i) {
  switch (p.ctype[c]) {
    case REL_U8: return (int64_t)__ldg(p.col[c] + i);
    case REL_I32: return (int64_t)__ldg((const int32_t*)p.col[c] + i);
    default: return (int64_t)__ldg((const long long*)p.col[c] + i);
  }
}

// Bitonic sort of SK_N (a, b) pairs in shared memory by less.  A stage with
// compare distance below 64 only pairs elements inside one aligned 128-element
// block, so warp w sorts block w on its own between two __syncwarp()s; only
// the 21 stages with distance >= 64 need the whole CTA (of 78 in all).
template <class Less>
__device__ void bitonic(int64_t* a, int64_t* b, Less less) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool prev_block = true;
  for (int size = 2; size <= SK_N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const bool block = stride >= 64;
      if (block || prev_block) __syncthreads();
      else __syncwarp();
      prev_block = block;
#pragma unroll
      for (int r = 0; r < SK_N / 2 / SK_THREADS; ++r) {
        // pair number t: block stages spread the pairs over the CTA, warp
        // stages keep warp w on the pairs of its own 128 elements
        const int t = block ? threadIdx.x + r * SK_THREADS : 64 * warp + lane + 32 * r;
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const bool swap = up ? less(a[hi], b[hi], a[lo], b[lo]) : less(a[lo], b[lo], a[hi], b[hi]);
        if (swap) {
          const int64_t ta = a[lo], tb = b[lo];
          a[lo] = a[hi];
          b[lo] = b[hi];
          a[hi] = ta;
          b[hi] = tb;
        }
      }
    }
  }
  __syncthreads();
}

// Exclusive prefix sum of one value per thread over the CTA; *total = the sum.
__device__ int block_scan(int v, int* total) {
  __shared__ int wsum[SK_THREADS / 32];
  __shared__ int all;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = wsum[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    wsum[lane] = wi - w;
    if (lane == 31) all = wi;
  }
  __syncthreads();
  const int r = wsum[warp] + incl - v;
  *total = all;
  __syncthreads();
  return r;
}

// One CTA sketches one input.
__device__ __forceinline__ void sketch_body(const SketchParams& p, DevSketch* out) {
  extern __shared__ int64_t sk_dyn[];
  int64_t* key = sk_dyn;        // [SK_N] sampled keys, then sorted
  int64_t* aux = sk_dyn + SK_N;  // [SK_N] 0 kept / 1 dropped, then counts
  int* start = (int*)(sk_dyn + 2 * SK_N);  // [SK_N + 1] positions of the distinct keys
  __shared__ unsigned int hll[256];
  __shared__ int n_kept, n_ndv, n_single, n_runs;
  __shared__ unsigned long long kmin_u, kmax_u;  // order-mapped (k ^ 2^63)

  const int64_t n = p.n_rows;
  const int S = n < SK_N ? (int)n : SK_N;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 256; i += SK_THREADS) hll[i] = 0;
  if (threadIdx.x == 0) {
    n_kept = n_single = n_runs = 0;
    kmin_u = ~0ull;
    kmax_u = 0ull;
  }
  __syncthreads();

  // every thread reads its SK_N / SK_THREADS sample rows (independent loads)
  int kept = 0;
  uint64_t lo_u = ~0ull, hi_u = 0ull;
#pragma unroll
  for (int r = 0; r < SK_N / SK_THREADS; ++r) {
    const int j = threadIdx.x + r * SK_THREADS;
    bool keep = j < S;
    int64_t k = 0;
    if (keep) {
      const int64_t row = n <= SK_N ? (int64_t)j
                                    : (int64_t)(j / 64) * (n - 64) / 63 + (j % 64);
      for (int i = 0; i < p.n_preds && keep; ++i) {
        const int64_t d = read_col(p, p.pred_col[i], row);
        keep = p.pred_lo[i] <= d && d <= p.pred_hi[i];
      }
      if (keep) {
        if (p.n_keys == 1) {
          k = read_col(p, p.key_col[0], row);
        } else {
          uint64_t u = 0;
          for (int i = 0; i < p.n_keys; ++i)
            u |= ((uint64_t)read_col(p, p.key_col[i], row) & p.key_mask[i]) << p.key_shift[i];
          k = (int64_t)u;
        }
      }
    }
    key[j] = k;
    aux[j] = keep ? 0 : 1;
    if (keep) {
      ++kept;
      const uint64_t h = splitmix64((uint64_t)k);
      const uint64_t rest = h << 8;
      const unsigned rank = rest == 0 ? 57u : (unsigned)__clzll((long long)rest) + 1u;
      atomicMax(&hll[h >> 56], rank);
      const uint64_t u = (uint64_t)k ^ 0x8000000000000000ull;
      lo_u = u < lo_u ? u : lo_u;
      hi_u = u > hi_u ? u : hi_u;
    }
  }
  // per-warp totals, one shared atomic per warp
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kept += __shfl_xor_sync(0xffffffffu, kept, o);
    const uint64_t a = __shfl_xor_sync(0xffffffffu, lo_u, o);
    const uint64_t b = __shfl_xor_sync(0xffffffffu, hi_u, o);
    lo_u = a < lo_u ? a : lo_u;
    hi_u = b > hi_u ? b : hi_u;
  }
  if (lane == 0 && kept) {
    atomicAdd(&n_kept, kept);
    atomicMin(&kmin_u, (unsigned long long)lo_u);
    atomicMax(&kmax_u, (unsigned long long)hi_u);
  }
  __syncthreads();
  // runs of equal consecutive kept keys inside each window (one thread each)
  if (threadIdx.x < 64) {
    const int w0 = threadIdx.x * 64;
    int runs = 0;
    bool have = false;
    int64_t last = 0;
    for (int o = 0; o < 64 && w0 + o < S; ++o) {
      if (aux[w0 + o]) continue;
      if (!have || key[w0 + o] != last) ++runs;
      have = true;
      last = key[w0 + o];
    }
    if (runs) atomicAdd(&n_runs, runs);
  }
  // sort by (dropped, key): kept keys first, ascending
  bitonic(aux, key, [](int64_t a0, int64_t b0, int64_t a1, int64_t b1) {
    return a0 != a1 ? a0 < a1 : b0 < b1;
  });
  const int m = n_kept;
  // distinct keys: the run starts of the sorted prefix, listed in order by a
  // prefix sum (thread t owns positions 4t .. 4t + 3); a key's count is the
  // distance to the next start
  constexpr int PER = SK_N / SK_THREADS;
  const int i0 = PER * threadIdx.x;
  int here = 0;
#pragma unroll
  for (int o = 0; o < PER; ++o) {
    const int i = i0 + o;
    here += (i < m && (i == 0 || key[i] != key[i - 1])) ? 1 : 0;
  }
  int ndv = 0;
  int pos = block_scan(here, &ndv);
#pragma unroll
  for (int o = 0; o < PER; ++o) {
    const int i = i0 + o;
    if (i < m && (i == 0 || key[i] != key[i - 1])) start[pos++] = i;
  }
  if (threadIdx.x == 0) {
    start[ndv] = m;
    n_ndv = ndv;
  }
  __syncthreads();
  int single = 0;
#pragma unroll
  for (int o = 0; o < PER; ++o) {
    const int i = i0 + o;
    aux[i] = 0;  // count at a run start (below), 0 elsewhere
  }
  __syncthreads();
  for (int r = threadIdx.x; r < ndv; r += SK_THREADS) {
    const int c = start[r + 1] - start[r];
    aux[start[r]] = c;
    single += c == 1;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) single += __shfl_xor_sync(0xffffffffu, single, o);
  if (lane == 0 && single) atomicAdd(&n_single, single);
  __syncthreads();
  // top keys: sort by (count descending, key ascending); non-starts (count 0) last
  bitonic(aux, key, [](int64_t c0, int64_t k0, int64_t c1, int64_t k1) {
    return c0 != c1 ? c0 > c1 : k0 < k1;
  });
  for (int i = threadIdx.x; i < SKETCH_TOP; i += SK_THREADS) {
    out->top_key[i] = i < ndv ? key[i] : 0;
    out->top_count[i] = i < ndv ? (int32_t)aux[i] : 0;
  }
  for (int i = threadIdx.x; i < 256; i += SK_THREADS) out->hll[i] = (uint8_t)hll[i];
  if (threadIdx.x == 0) {
    out->sample_rows = S;
    out->kept = m;
    out->ndv = ndv;
    out->singletons = n_single;
    out->runs = n_runs;
    out->key_min = m ? (int64_t)(kmin_u ^ 0x8000000000000000ull) : 0;
    out->key_max = m ? (int64_t)(kmax_u ^ 0x8000000000000000ull) : 0;
  }
}

__global__ void __launch_bounds__(SK_THREADS) sketch_k(const __grid_constant__ SketchParams p,
                                                        DevSketch* out) {
  sketch_body(p, out);
}

// Many inputs in one launch: CTA b sketches input b.
__global__ void __launch_bounds__(SK_THREADS) sketch_many_k(const SketchParams* __restrict__ ps,
                                                             DevSketch* outs) {
  sketch_body(ps[blockIdx.x], outs + blockIdx.x);
}

}  // namespace

rel_status sketch_many_launch(const SketchParams* ps, DevSketch* outs, int n, cudaStream_t st) {
  if (n <= 0) return REL_OK;
  const int smem = 2 * SK_N * (int)sizeof(int64_t) + (SK_N + 4) * (int)sizeof(int);
  cudaError_t e0 =
      cudaFuncSetAttribute(sketch_many_k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e0 != cudaSuccess) return relhost::cuda_fail(e0, "cudaFuncSetAttribute(sketch)");
  relhost::launch_begin(relhost::K_SKETCH, st);
  sketch_many_k<<<n, SK_THREADS, smem, st>>>(ps, outs);
  relhost::launch_end(relhost::K_SKETCH, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(sketch, batched)");
}

rel_status sketch_launch(const SketchParams& p, DevSketch* out, cudaStream_t st) {
  const int smem = 2 * SK_N * (int)sizeof(int64_t) + (SK_N + 4) * (int)sizeof(int);
  cudaError_t e0 = cudaFuncSetAttribute(sketch_k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e0 != cudaSuccess) return relhost::cuda_fail(e0, "cudaFuncSetAttribute(sketch)");
  relhost::launch_begin(relhost::K_SKETCH, st);
  sketch_k<<<1, SK_THREADS, smem, st>>>(p, out);
  relhost::launch_end(relhost::K_SKETCH, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(sketch)");
}

}  // namespace rel
