// Learned-priority MLP (12 -> 64 -> 64 -> 1): inference and training.
#pragma once

#include "common.cuh"

namespace gbch {

constexpr int MLP_NIN = 12;
constexpr int MLP_NH = 64;
constexpr int MLP_NPARAM = MLP_NIN * MLP_NH + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NH + 1;
static_assert(MLP_NPARAM == CH_MLP_NPARAM, "parameter count of ch.h");

// sign(x) * log2(1 + |x|), the transform applied to every integer feature.
__host__ __device__ __forceinline__ float feature_transform(long long x) {
    const double a = x < 0 ? -(double)x : (double)x;
    const float v = (float)log2(1.0 + a);
    return x < 0 ? -v : v;
}

// Weights resident on the device: FP32 copy and the BF16 tensor-core
// fragments of W1 and W2.
struct MlpDevice {
    DevBuf<float> weights;
    DevBuf<uint32_t> frag;
    MlpDevice();
    ~MlpDevice();
    void load(const float *host_weights, cudaStream_t st);
    // y[r] = MLP(x[r]); x holds 16 floats per row (12 transformed features).
    void infer(const float *x, uint64_t rows, float *y, cudaStream_t st) const;
};

// x[r] = transformed features of trace rows (round, vertex, 12 features).
void rows_to_features(const long long *rows, uint64_t n, float *x, cudaStream_t st);

// y[r] = training target of trace row r: sign(x) * log2(1 + |x|) of
// x = edge difference + 2 * hierarchy depth at that rescoring.
void mlp_targets(const long long *rows, uint64_t n, float *y, cudaStream_t st);

// Adam training (or, with epochs = 0, the gradient of the first batch).
void mlp_train(const long long *rows, const float *labels, uint64_t n, const ch_train_params_t *tp,
               float *weights_io, float *loss_out, float *grad_out, cudaStream_t st);

}  // namespace gbch
