// The planner network's layout and launchers (mlp.cu), used by api.cu.
#pragma once

#include "rel_internal.cuh"

namespace rel {

constexpr int MLP_IN = REL_MLP_IN;        // 264 sketch features
constexpr int MLP_H = REL_MLP_HIDDEN;     // 64
constexpr int MLP_OUT = REL_MLP_OUT;      // log2 ndv + 3 variant logits
// parameter layout (FP32 master copy and BF16 copy alike):
//   W1[64][264] b1[64] W2[64][64] b2[64] W3[4][64] b3[4]
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_H;
constexpr int MLP_PARAMS = OFF_B3 + MLP_OUT;
static_assert(MLP_PARAMS == REL_MLP_PARAMS, "parameter count");
constexpr int ACT_STRIDE = 2 * MLP_H;          // z1, z2 per sample
constexpr int DZ_STRIDE = 2 * MLP_H + MLP_OUT;  // dz1, dz2, dout per sample

struct MlpAdamW {
  float lr, beta1, beta2, eps, wd, bc1, bc2;  // bc = 1 - beta^step
};

rel_status mlp_round(const float* p, void* wb, cudaStream_t st);
rel_status mlp_forward(const void* wb, const float* p, const float* x, int batch, float* out,
                       float* acts, cudaStream_t st);
rel_status mlp_backward(const void* wb, const float* x, const float* acts, const float* out,
                        const float* t_ndv, const int32_t* t_var, int batch, float* dz,
                        float* grad, float* loss, cudaStream_t st);
rel_status mlp_adamw(float* p, void* wb, float* m, float* v, const float* g, const MlpAdamW& h,
                     cudaStream_t st);

}  // namespace rel
