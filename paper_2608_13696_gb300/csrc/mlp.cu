// The planner's network: 264 sketch features -> 64 -> 64 -> 4 outputs
// (log2 of the number of groups, and logits of the three group-by variants:
// CTA-private tables, one global table, partitioned).  Weights are stored in
// FP32 (the optimiser's master copy) with a BF16 copy used by the forward and
// backward passes; the BF16 operands are multiplied and accumulated in FP32
// (a BF16 x BF16 product is exact in FP32).  Inputs and hidden activations
// are rounded to BF16 where they enter a layer.  Hidden layers use ReLU.
//
// Loss per sample: (y0 - log2 ndv)^2 + cross-entropy(softmax(y1..y3), label),
// averaged over the batch.  The network is tiny (21,380 parameters), so the
// kernels are plain per-thread dot products; nothing here is a contraction
// worth tensor cores.
#include <cuda_bf16.h>

#include "mlp.cuh"

namespace rel {

namespace {

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float wbf(const __nv_bfloat16* w, int i) {
  return __bfloat162float(w[i]);
}

// One CTA per sample, MLP_H threads.
__global__ void __launch_bounds__(MLP_H) mlp_fwd_k(const __nv_bfloat16* __restrict__ wb,
                                                   const float* __restrict__ pf,
                                                   const float* __restrict__ x, int batch,
                                                   float* __restrict__ out,
                                                   float* __restrict__ acts) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= batch) return;
  __shared__ float xin[MLP_IN], h1[MLP_H], h2[MLP_H];
  for (int k = j; k < MLP_IN; k += MLP_H) xin[k] = bf(x[(size_t)b * MLP_IN + k]);
  __syncthreads();
  float z = 0.f;
  for (int k = 0; k < MLP_IN; ++k) z = fmaf(wbf(wb, OFF_W1 + j * MLP_IN + k), xin[k], z);
  z += pf[OFF_B1 + j];
  const float a1 = bf(z > 0.f ? z : 0.f);
  h1[j] = a1;
  if (acts) acts[(size_t)b * ACT_STRIDE + j] = z;
  __syncthreads();
  z = 0.f;
  for (int k = 0; k < MLP_H; ++k) z = fmaf(wbf(wb, OFF_W2 + j * MLP_H + k), h1[k], z);
  z += pf[OFF_B2 + j];
  const float a2 = bf(z > 0.f ? z : 0.f);
  h2[j] = a2;
  if (acts) acts[(size_t)b * ACT_STRIDE + MLP_H + j] = z;
  __syncthreads();
  if (j < MLP_OUT) {
    float y = 0.f;
    for (int k = 0; k < MLP_H; ++k) y = fmaf(wbf(wb, OFF_W3 + j * MLP_H + k), h2[k], y);
    out[(size_t)b * MLP_OUT + j] = y + pf[OFF_B3 + j];
  }
}

// Per-sample part of the backward pass: output gradient, then dz2, dz1
// (gradients at the hidden pre-activations), and the sample's loss.
__global__ void __launch_bounds__(MLP_H) mlp_bwd_sample_k(
    const __nv_bfloat16* __restrict__ wb, const float* __restrict__ acts,
    const float* __restrict__ out, const float* __restrict__ t_ndv,
    const int32_t* __restrict__ t_var, int batch, float* __restrict__ dz, float* __restrict__ loss) {
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= batch) return;
  __shared__ float dout[MLP_OUT], d2[MLP_H];
  const float inv_b = 1.f / (float)batch;
  if (j == 0) {
    const float* y = out + (size_t)b * MLP_OUT;
    const float e = y[0] - t_ndv[b];
    float m = fmaxf(y[1], fmaxf(y[2], y[3]));
    const float s1 = expf(y[1] - m), s2 = expf(y[2] - m), s3 = expf(y[3] - m);
    const float sum = s1 + s2 + s3;
    const int lab = t_var[b];
    const float p[3] = {s1 / sum, s2 / sum, s3 / sum};
    dout[0] = 2.f * e * inv_b;
    for (int c = 0; c < 3; ++c) dout[1 + c] = (p[c] - (c == lab ? 1.f : 0.f)) * inv_b;
    const float ce = logf(sum) + m - y[1 + lab];
    atomicAdd(loss, (e * e + ce) * inv_b);
    for (int c = 0; c < MLP_OUT; ++c) dz[(size_t)b * DZ_STRIDE + 2 * MLP_H + c] = dout[c];
  }
  __syncthreads();
  // dh2[j] = sum_o W3[o][j] dout[o]; dz2 = dh2 where z2 > 0
  float g = 0.f;
  for (int o = 0; o < MLP_OUT; ++o) g = fmaf(wbf(wb, OFF_W3 + o * MLP_H + j), dout[o], g);
  const float z2 = acts[(size_t)b * ACT_STRIDE + MLP_H + j];
  const float g2 = z2 > 0.f ? g : 0.f;
  d2[j] = g2;
  dz[(size_t)b * DZ_STRIDE + MLP_H + j] = g2;
  __syncthreads();
  // dh1[j] = sum_i W2[i][j] dz2[i]; dz1 = dh1 where z1 > 0
  g = 0.f;
  for (int i = 0; i < MLP_H; ++i) g = fmaf(wbf(wb, OFF_W2 + i * MLP_H + j), d2[i], g);
  const float z1 = acts[(size_t)b * ACT_STRIDE + j];
  dz[(size_t)b * DZ_STRIDE + j] = z1 > 0.f ? g : 0.f;
}

// Parameter gradients: one thread per parameter, summing over the batch.
__global__ void mlp_bwd_param_k(const float* __restrict__ x, const float* __restrict__ acts,
                                const float* __restrict__ dz, int batch, float* __restrict__ grad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MLP_PARAMS) return;
  float s = 0.f;
  if (q < OFF_B1) {  // W1[j][k]: dz1[j] * x[k]
    const int j = q / MLP_IN, k = q % MLP_IN;
    for (int b = 0; b < batch; ++b)
      s = fmaf(dz[(size_t)b * DZ_STRIDE + j], bf(x[(size_t)b * MLP_IN + k]), s);
  } else if (q < OFF_W2) {
    const int j = q - OFF_B1;
    for (int b = 0; b < batch; ++b) s += dz[(size_t)b * DZ_STRIDE + j];
  } else if (q < OFF_B2) {  // W2[j][k]: dz2[j] * h1[k]
    const int j = (q - OFF_W2) / MLP_H, k = (q - OFF_W2) % MLP_H;
    for (int b = 0; b < batch; ++b) {
      const float z1 = acts[(size_t)b * ACT_STRIDE + k];
      s = fmaf(dz[(size_t)b * DZ_STRIDE + MLP_H + j], bf(z1 > 0.f ? z1 : 0.f), s);
    }
  } else if (q < OFF_W3) {
    const int j = q - OFF_B2;
    for (int b = 0; b < batch; ++b) s += dz[(size_t)b * DZ_STRIDE + MLP_H + j];
  } else if (q < OFF_B3) {  // W3[o][k]: dout[o] * h2[k]
    const int o = (q - OFF_W3) / MLP_H, k = (q - OFF_W3) % MLP_H;
    for (int b = 0; b < batch; ++b) {
      const float z2 = acts[(size_t)b * ACT_STRIDE + MLP_H + k];
      s = fmaf(dz[(size_t)b * DZ_STRIDE + 2 * MLP_H + o], bf(z2 > 0.f ? z2 : 0.f), s);
    }
  } else {
    const int o = q - OFF_B3;
    for (int b = 0; b < batch; ++b) s += dz[(size_t)b * DZ_STRIDE + 2 * MLP_H + o];
  }
  grad[q] = s;
}

// AdamW (Loshchilov & Hutter 2019): decoupled weight decay on the weights
// (not the biases), bias-corrected moments; refreshes the BF16 copy.
__global__ void mlp_adamw_k(float* __restrict__ p, __nv_bfloat16* __restrict__ wb,
                            float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, MlpAdamW h) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MLP_PARAMS) return;
  const bool is_bias = (q >= OFF_B1 && q < OFF_W2) || (q >= OFF_B2 && q < OFF_W3) || q >= OFF_B3;
  const float gq = g[q];
  const float mq = h.beta1 * m[q] + (1.f - h.beta1) * gq;
  const float vq = h.beta2 * v[q] + (1.f - h.beta2) * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float mhat = mq / h.bc1, vhat = vq / h.bc2;
  float pq = p[q];
  if (!is_bias) pq -= h.lr * h.wd * pq;
  pq -= h.lr * mhat / (sqrtf(vhat) + h.eps);
  p[q] = pq;
  wb[q] = __float2bfloat16_rn(pq);
}

__global__ void mlp_round_k(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < MLP_PARAMS) wb[q] = __float2bfloat16_rn(p[q]);
}

rel_status done(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, what);
}

}  // namespace

rel_status mlp_round(const float* p, void* wb, cudaStream_t st) {
  relhost::launch_begin(relhost::K_MLP, st);
  mlp_round_k<<<(MLP_PARAMS + 255) / 256, 256, 0, st>>>(p, (__nv_bfloat16*)wb);
  relhost::launch_end(relhost::K_MLP, st);
  return done("launch(mlp round)");
}

rel_status mlp_forward(const void* wb, const float* p, const float* x, int batch, float* out,
                       float* acts, cudaStream_t st) {
  if (batch == 0) return REL_OK;
  relhost::launch_begin(relhost::K_MLP, st);
  mlp_fwd_k<<<batch, MLP_H, 0, st>>>((const __nv_bfloat16*)wb, p, x, batch, out, acts);
  relhost::launch_end(relhost::K_MLP, st);
  return done("launch(mlp forward)");
}

rel_status mlp_backward(const void* wb, const float* x, const float* acts, const float* out,
                        const float* t_ndv, const int32_t* t_var, int batch, float* dz,
                        float* grad, float* loss, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return relhost::cuda_fail(e, "cudaMemsetAsync");
  if (batch == 0) {
    e = cudaMemsetAsync(grad, 0, sizeof(float) * MLP_PARAMS, st);
    return e == cudaSuccess ? REL_OK : relhost::cuda_fail(e, "cudaMemsetAsync");
  }
  relhost::launch_begin(relhost::K_MLP, st);
  mlp_bwd_sample_k<<<batch, MLP_H, 0, st>>>((const __nv_bfloat16*)wb, acts, out, t_ndv, t_var,
                                             batch, dz, loss);
  relhost::launch_end(relhost::K_MLP, st);
  rel_status r = done("launch(mlp backward)");
  if (r) return r;
  relhost::launch_begin(relhost::K_MLP, st);
  mlp_bwd_param_k<<<(MLP_PARAMS + 255) / 256, 256, 0, st>>>(x, acts, dz, batch, grad);
  relhost::launch_end(relhost::K_MLP, st);
  return done("launch(mlp gradients)");
}

rel_status mlp_adamw(float* p, void* wb, float* m, float* v, const float* g, const MlpAdamW& h,
                     cudaStream_t st) {
  relhost::launch_begin(relhost::K_MLP, st);
  mlp_adamw_k<<<(MLP_PARAMS + 255) / 256, 256, 0, st>>>(p, (__nv_bfloat16*)wb, m, v, g, h);
  relhost::launch_end(relhost::K_MLP, st);
  return done("launch(mlp adamw)");
}

}  // namespace rel
