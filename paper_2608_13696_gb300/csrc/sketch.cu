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
// Distinct keys and their counts come from a shared-memory hash table of
// sample positions (no sort); the top keys from a histogram of the counts
// (the cut at the 32nd largest count) and a bitonic sort of only the keys
// counted at least that often -- a handful for a skewed sample, every key
// when all are seen once.
#include "sketch.cuh"

namespace rel {

namespace {

constexpr int SK_THREADS = 1024;
constexpr int SK_N = SKETCH_SAMPLE;  // 4096
constexpr int SK_TAB = 2 * SK_N;     // hash table entries (load <= 1/2)

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

// Bitonic sort of the first n (a power of two, <= SK_N) pairs, a CTA
// barrier per stage (the candidate lists are short for skewed samples).
template <class Less>
__device__ void bitonic_n(int64_t* a, int64_t* b, int n, Less less) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < n / 2; t += SK_THREADS) {
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
  int64_t* key = sk_dyn;          // [SK_N] sampled keys
  int64_t* aux = sk_dyn + SK_N;    // [SK_N] 0 kept / 1 dropped, then candidate counts
  int64_t* key2 = sk_dyn + 2 * SK_N;  // [SK_N] candidate keys
  int* tab = (int*)(sk_dyn + 3 * SK_N);  // [SK_TAB] 1 + sample position of a key
  int* tcnt = tab + SK_TAB;              // [SK_TAB] its count
  int* start = tcnt + SK_TAB;            // [SK_N + 4] count histogram
  __shared__ unsigned int hll[256];
  __shared__ int n_kept, n_ndv, n_single, n_runs, s_cut;
  __shared__ unsigned long long kmin_u, kmax_u;  // order-mapped (k ^ 2^63)

  const int64_t n = p.n_rows;
  const int S = n < SK_N ? (int)n : SK_N;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 256; i += SK_THREADS) hll[i] = 0;
  if (threadIdx.x == 0) {
    n_kept = n_ndv = n_single = n_runs = 0;
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
  const int m = n_kept;
  // distinct keys and their counts: a shared-memory hash table of sample
  // positions (load <= 1/2), entry = 1 + the position of the key's first
  // insert; equal keys meet at the same entry and add to its count
  constexpr int PER = SK_N / SK_THREADS;
  for (int i = threadIdx.x; i < SK_TAB; i += SK_THREADS) {
    tab[i] = 0;
    tcnt[i] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int j = threadIdx.x + r * SK_THREADS;
    if (j >= S || aux[j]) continue;
    const int64_t k = key[j];
    uint32_t t = (uint32_t)(splitmix64((uint64_t)k) >> 32) & (SK_TAB - 1);
    for (int probe = 0; probe < SK_TAB; ++probe) {
      int cur = tab[t];
      if (cur == 0) {
        cur = atomicCAS(&tab[t], 0, j + 1);
        if (cur == 0) {
          atomicAdd(&tcnt[t], 1);
          break;
        }
      }
      if (key[cur - 1] == k) {
        atomicAdd(&tcnt[t], 1);
        break;
      }
      t = (t + 1) & (SK_TAB - 1);
    }
  }
  __syncthreads();
  // distinct and single keys; histogram of the counts (bins 1 .. SK_N)
  int* hist = start;  // [SK_N + 1]
  for (int i = threadIdx.x; i <= SK_N; i += SK_THREADS) hist[i] = 0;
  __syncthreads();
  int nd = 0, single = 0;
  for (int i = threadIdx.x; i < SK_TAB; i += SK_THREADS) {
    const int c = tcnt[i];
    if (c == 0) continue;
    ++nd;
    single += c == 1;
    atomicAdd(&hist[c], 1);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    nd += __shfl_xor_sync(0xffffffffu, nd, o);
    single += __shfl_xor_sync(0xffffffffu, single, o);
  }
  if (lane == 0 && nd) atomicAdd(&n_ndv, nd);
  if (lane == 0 && single) atomicAdd(&n_single, single);
  __syncthreads();
  const int ndv = n_ndv;
  // cut: the SKETCH_TOP-th largest count (every key counted at least that
  // often is a candidate, so ties at the cut are all present); thread t owns
  // the bins 4t + 1 .. 4t + 4
  int mine = 0;
#pragma unroll
  for (int o = 1; o <= PER; ++o) mine += hist[PER * threadIdx.x + o];
  int all = 0;
  const int below = block_scan(mine, &all);  // keys counted <= 4t times
  int above = all - below - mine;             // keys counted > 4t + 4 times
  if (threadIdx.x == 0) s_cut = 1;
  __syncthreads();
  if (ndv > SKETCH_TOP) {
#pragma unroll
    for (int o = PER; o >= 1; --o) {
      const int c = PER * threadIdx.x + o, h = hist[c];
      if (above < SKETCH_TOP && above + h >= SKETCH_TOP) s_cut = c;
      above += h;
    }
  }
  __syncthreads();
  const int cut = s_cut;
  // the candidates (count >= cut), listed with a prefix sum, then sorted by
  // (count descending, key ascending); the padding sorts last
  int here = 0;
  for (int i = PER * 2 * threadIdx.x; i < PER * 2 * (threadIdx.x + 1); ++i) here += tcnt[i] >= cut;
  int n_cand = 0;
  int pos = block_scan(here, &n_cand);
  for (int i = PER * 2 * threadIdx.x; i < PER * 2 * (threadIdx.x + 1); ++i) {
    if (tcnt[i] >= cut && tcnt[i] > 0) {
      aux[pos] = tcnt[i];
      key2[pos] = key[tab[i] - 1];
      ++pos;
    }
  }
  int n2 = 2;
  while (n2 < n_cand) n2 <<= 1;
  for (int i = n_cand + threadIdx.x; i < n2; i += SK_THREADS) {
    aux[i] = -1;
    key2[i] = 0;
  }
  bitonic_n(aux, key2, n2, [](int64_t c0, int64_t k0, int64_t c1, int64_t k1) {
    return c0 != c1 ? c0 > c1 : k0 < k1;
  });
  for (int i = threadIdx.x; i < SKETCH_TOP; i += SK_THREADS) {
    out->top_key[i] = i < ndv ? key2[i] : 0;
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
  const int smem = 3 * SK_N * (int)sizeof(int64_t) + (2 * SK_TAB + SK_N + 4) * (int)sizeof(int);
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
  const int smem = 3 * SK_N * (int)sizeof(int64_t) + (2 * SK_TAB + SK_N + 4) * (int)sizeof(int);
  cudaError_t e0 = cudaFuncSetAttribute(sketch_k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e0 != cudaSuccess) return relhost::cuda_fail(e0, "cudaFuncSetAttribute(sketch)");
  relhost::launch_begin(relhost::K_SKETCH, st);
  sketch_k<<<1, SK_THREADS, smem, st>>>(p, out);
  relhost::launch_end(relhost::K_SKETCH, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "launch(sketch)");
}

}  // namespace rel
