/*
 * Seeded synthetic key/value columns generated on the GPU, for workloads too
 * large to generate on the host for every instance (many instances of up to
 * tens of millions of rows each).
 *
 * Input production only, like gen.c: nothing here hashes keys into tables,
 * aggregates or matches.  The counter-based generator is the same splitmix64
 * stream as gen.c (stream_key(seed, tag) + i), so the uniform family and the
 * values are bit-identical to gen.c's syn_uniform_mixed / syn_uniform.
 *
 * Key families over a domain of D ranks (key = splitmix64(rank), a bijective
 * scramble over all of int64):
 *   0 uniform    rank = U[1, D];
 *   1 Zipf(s)    P(rank = k) proportional to k^-s on [1, D], sampled by
 *                rejection-inversion (Hoermann & Derflinger 1996) with at most
 *                64 attempts per row (then the last candidate is kept);
 *   2 clustered  runs of equal keys: each row starts a new run with
 *                probability 1/64 (geometric run lengths, mean 64; a run is
 *                cut after 4096 rows), the run's rank = U[1, D] drawn at its
 *                first row.
 * Values: U[-10^6, 10^6].
 *
 * Join sides: the build and probe streams of gen.c (40-bit Feistel
 * permutation keys, Bernoulli hits), bit-identical to syn_join_build and
 * syn_join_probe.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr uint64_t TAG_KEY = 0x21, TAG_VAL = 0x22, TAG_RUN = 0x23;

__host__ __device__ inline uint64_t mix64(uint64_t x) {
  uint64_t z = x + GAMMA;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t stream_key(uint64_t seed, uint64_t tag) {
  return mix64(mix64(seed) ^ tag);
}

__device__ inline int64_t uniform_in(uint64_t r, int64_t lo, int64_t hi) {
  const uint64_t span = (uint64_t)hi - (uint64_t)lo + 1u;
  if (span == 0) return (int64_t)((uint64_t)lo + r);
  return (int64_t)((uint64_t)lo + __umul64hi(r, span));
}

// (0, 1]: 53 random bits
__device__ inline double unit(uint64_t r) { return ((double)(r >> 11) + 1.0) * 0x1.0p-53; }

// Hat function h(x) = x^-s, its antiderivative H and the inverse of H.
struct ZipfHat {
  double s, one_minus_s;
  bool log_form;  // s == 1
  __device__ double h(double x) const { return pow(x, -s); }
  __device__ double H(double x) const {
    return log_form ? log(x) : (pow(x, one_minus_s) - 1.0) / one_minus_s;
  }
  __device__ double Hinv(double y) const {
    return log_form ? exp(y) : pow(1.0 + one_minus_s * y, 1.0 / one_minus_s);
  }
};

__global__ void kv_kernel(int family, double s, int64_t n, int64_t domain, uint64_t seed,
                          int64_t* __restrict__ keys, int64_t* __restrict__ vals) {
  const uint64_t kkey = stream_key(seed, TAG_KEY), kval = stream_key(seed, TAG_VAL),
                 krun = stream_key(seed, TAG_RUN);
  ZipfHat z;
  z.s = s;
  z.one_minus_s = 1.0 - s;
  z.log_form = s == 1.0;
  const double D = (double)domain;
  // the candidate interval of rank k is [H(k - 1/2), H(k + 1/2)]; rank 1's
  // is cut to width h(1) = 1 so that it is accepted outright
  const double u_lo = family == 1 ? z.H(1.5) - 1.0 : 0.0;
  const double u_hi = family == 1 ? z.H(D + 0.5) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rank;
    if (family == 1) {
      int64_t k = 1;
      for (int a = 0; a < 64; ++a) {
        const double u = u_lo + unit(mix64(kkey + ((uint64_t)i << 6) + (uint64_t)a)) * (u_hi - u_lo);
        const double x = z.Hinv(u);
        k = (int64_t)(x + 0.5);
        if (k < 1) k = 1;
        if (k > domain) k = domain;
        if (k == 1 || u >= z.H((double)k + 0.5) - z.h((double)k)) break;
      }
      rank = k;
    } else if (family == 2) {
      int64_t j = i;
      while (j > 0 && i - j < 4096 && (mix64(krun + (uint64_t)j) >> 58) != 0) --j;
      rank = uniform_in(mix64(kkey + (uint64_t)j), 1, domain);
    } else {
      rank = uniform_in(mix64(kkey + (uint64_t)i), 1, domain);
    }
    keys[i] = (int64_t)mix64((uint64_t)rank);
    if (vals) vals[i] = uniform_in(mix64(kval + (uint64_t)i), -1000000, 1000000);
  }
}

// The join streams of gen.c, row for row (see syn_join_build / syn_join_probe).
constexpr uint64_t TAG_PERM = 0x50, TAG_PAYLOAD = 0x51, TAG_HIT = 0x52, TAG_PICK = 0x53,
                   TAG_MISS = 0x54;

__device__ inline uint64_t perm40(uint64_t x, uint64_t pkey) {
  const uint64_t M = (1ull << 20) - 1;
  uint64_t L = (x >> 20) & M, R = x & M;
  for (uint64_t k = 0; k < 4; k++) {
    const uint64_t rk = mix64(pkey ^ (k + 1));
    const uint64_t F = mix64(rk ^ R) & M;
    const uint64_t nL = R, nR = L ^ F;
    L = nL;
    R = nR;
  }
  return (L << 20) | R;
}

__global__ void join_build_kernel(int64_t n_b, uint64_t seed, int64_t* keys, int64_t* pay) {
  const uint64_t pk = stream_key(seed, TAG_PERM), payk = stream_key(seed, TAG_PAYLOAD);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_b;
       j += (int64_t)gridDim.x * blockDim.x) {
    keys[j] = (int64_t)perm40((uint64_t)j, pk);
    if (pay) pay[j] = uniform_in(mix64(payk + (uint64_t)j), 0, INT64_MAX);
  }
}

__global__ void join_probe_kernel(int64_t n_p, int64_t n_b, uint64_t thr, uint64_t seed,
                                  int64_t* keys) {
  const uint64_t pk = stream_key(seed, TAG_PERM), hk = stream_key(seed, TAG_HIT),
                 ck = stream_key(seed, TAG_PICK), mk = stream_key(seed, TAG_MISS);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_p;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool hit = mix64(hk + (uint64_t)i) < thr;
    const uint64_t src = hit ? (uint64_t)uniform_in(mix64(ck + (uint64_t)i), 0, n_b - 1)
                             : (uint64_t)uniform_in(mix64(mk + (uint64_t)i), n_b,
                                                    (int64_t)(1ull << 40) - 1);
    keys[i] = (int64_t)perm40(src, pk);
  }
}

unsigned grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  return (unsigned)(blocks > cap ? cap : blocks);
}

}  // namespace

/* Join build side as gen.c's syn_join_build (keys distinct): keys[n_b],
 * payload[n_b] (NULL to skip), device memory.  1 <= n_b < 2^40. */
extern "C" int syn_gpu_join_build(int64_t n_b, uint64_t seed, int64_t* keys, int64_t* payload,
                                  void* stream) {
  if (n_b < 0 || n_b >= (1ll << 40) || (n_b > 0 && !keys)) return (int)cudaErrorInvalidValue;
  if (n_b == 0) return 0;
  join_build_kernel<<<grid_for(n_b), 256, 0, (cudaStream_t)stream>>>(n_b, seed, keys, payload);
  return (int)cudaGetLastError();
}

/* Join probe side as gen.c's syn_join_probe (without the present flags). */
extern "C" int syn_gpu_join_probe(int64_t n_p, int64_t n_b, uint64_t hit_threshold, uint64_t seed,
                                  int64_t* keys, void* stream) {
  if (n_p < 0 || n_b < 1 || n_b >= (1ll << 40) || (n_p > 0 && !keys))
    return (int)cudaErrorInvalidValue;
  if (n_p == 0) return 0;
  join_probe_kernel<<<grid_for(n_p), 256, 0, (cudaStream_t)stream>>>(n_p, n_b, hit_threshold, seed,
                                                                     keys);
  return (int)cudaGetLastError();
}

/* keys[n] (and vals[n] unless NULL), device memory.  family 0/1/2 as above,
 * s the Zipf exponent (> 0; family 1 only), domain >= 1.  Returns a
 * cudaError_t value (0 = success). */
extern "C" int syn_gpu_kv(int family, double s, int64_t n, int64_t domain, uint64_t seed,
                          int64_t* keys, int64_t* vals, void* stream) {
  if (n < 0 || domain < 1 || family < 0 || family > 2 || (family == 1 && !(s > 0.0)) ||
      (n > 0 && !keys) || n >= (1ll << 56))
    return (int)cudaErrorInvalidValue;
  if (n == 0) return 0;
  kv_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(family, s, n, domain, seed, keys,
                                                           vals);
  return (int)cudaGetLastError();
}
