// Smoothing-length MLP: sizes and launchers (kernels in mlp.cu).
#pragma once

#include "nl_internal.cuh"

namespace nlg {

constexpr int kMlpF = 8;    // input features per cluster
constexpr int kMlpH = 64;   // hidden width
// packed parameters: W1 (64x8) b1 W2 (64x64) b2 W3 (64x64) b3 W4 (64) b4
constexpr int kMlpParams = kMlpH * kMlpF + kMlpH + 2 * (kMlpH * kMlpH + kMlpH) + kMlpH + 1;

size_t mlp_train_smem();
size_t mlp_predict_smem();
// features X (ncl x 8) and e64 (per super-cluster) of a prepared list
cudaError_t mlp_features(uint32_t nsc, int M, const SysTables &t, const float4 *clo,
                         const float4 *chi, const uint32_t *perm_pad, float4 *slo, float4 *shi,
                         float *X, float *e64, cudaStream_t s);
// targets y (ncl) and weights w (1 real cluster, 0 empty) from h (caller order)
cudaError_t mlp_targets(uint32_t ncl, int M, const uint32_t *perm_pad, const float *h,
                        const float *e64, float *y, float *w, cudaStream_t s);
// hq (padded order) = e64 * exp(pred of the cluster)
cudaError_t mlp_apply_h0(uint32_t npad, int M, const uint32_t *perm_pad, const float *pred,
                         const float *e64, float *hq, cudaStream_t s);
cudaError_t mlp_predict(int64_t n, const float *X, const float *P, float *out, int num_sms,
                        cudaStream_t s);
// one minibatch (samples idx[0..nb)): gradient of sum_r w_r (pred_r - y_r)^2 * inv_n
// into grad (if not NULL) and, when adam != 0, one Adam step of P (step >= 1)
cudaError_t mlp_train_step(int64_t nb, const int64_t *idx, const float *X, const float *Y,
                           const float *W, float *P, float *m, float *v, float *partial,
                           int slots, float *grad, float *loss, int adam, float lr, int step,
                           float inv_n, cudaStream_t s);

}  // namespace nlg
