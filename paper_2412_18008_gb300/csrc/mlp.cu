// Learned vertex priority: a 12 -> 64 -> 64 -> 1 MLP over integer-derived
// per-vertex features, used in place of the edge difference (the paper's
// Alg. 4 score) when CH_PRIO_LEARNED is set. The paper has no learned
// priority; any priority yields a valid hierarchy (Alg. 5 only needs a
// strict order), so the network can only change the hierarchy's quality.
//
// Inference runs on the tensor cores: BF16 weights and activations, FP32
// accumulation (mma.sync m16n8k16), one warp per 16 vertices; layer 1's
// accumulators are re-packed in registers as layer 2's A fragments.
// Training runs forward passes with the same BF16 roundings, backward passes
// in FP32 (rounding treated as identity), gradient sums in a fixed order
// (deterministic), and Adam on FP32 master weights.
//
// Weight layout (FP32, CH_MLP_NPARAM values): W1[12][64] (input-major),
// b1[64], W2[64][64] (input-major), b2[64], W3[64], b3.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "mlp.cuh"

namespace gbch {

namespace {

constexpr int NIN = MLP_NIN, NH = MLP_NH;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
static_assert(OFF_B3 + 1 == MLP_NPARAM, "parameter layout");

__device__ __forceinline__ float bf16_round(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// The copy of parameter p the forward pass uses: W1 and W2 in BF16 (as the
// tensor-core inference uses them), biases and W3 in FP32.
__device__ __forceinline__ float quantised(uint32_t p, float w) {
    return (p < (uint32_t)OFF_B1 || (p >= (uint32_t)OFF_W2 && p < (uint32_t)OFF_B2)) ? bf16_round(w) : w;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// D = A * B + C for one m16n8k16 tile (A row-major BF16, B column-major BF16).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragments of W1 (K = 16 rows, 12 used) and W2 (K = 64), per lane:
// frag1[j][lane] for n-tile j (8 columns); frag2[kk][j][lane] for k-tile kk.
struct MlpFrag {
    uint2 w1[NH / 8][32];
    uint2 w2[NH / 16][NH / 8][32];
    float b1[NH], b2[NH], w3[NH], b3;
};

__global__ void k_mlp_prepare(const float *w, MlpFrag *f) {
    const uint32_t lane = threadIdx.x & 31u, grp = lane >> 2, tig = lane & 3u;
    const uint32_t warp = threadIdx.x >> 5;
    // W1: element (k, n) = W1[k][n] for k < 12, 0 above
    auto w1 = [&](uint32_t k, uint32_t n) { return k < (uint32_t)NIN ? w[OFF_W1 + k * NH + n] : 0.f; };
    for (uint32_t j = warp; j < NH / 8; j += blockDim.x >> 5) {
        const uint32_t n = 8 * j + grp;
        f->w1[j][lane] = make_uint2(pack_bf16(w1(2 * tig, n), w1(2 * tig + 1, n)),
                                    pack_bf16(w1(2 * tig + 8, n), w1(2 * tig + 9, n)));
    }
    for (uint32_t t = warp; t < (NH / 16) * (NH / 8); t += blockDim.x >> 5) {
        const uint32_t kk = t / (NH / 8), j = t % (NH / 8);
        const uint32_t n = 8 * j + grp, k0 = 16 * kk + 2 * tig;
        const float *W2 = w + OFF_W2;
        f->w2[kk][j][lane] = make_uint2(pack_bf16(W2[k0 * NH + n], W2[(k0 + 1) * NH + n]),
                                        pack_bf16(W2[(k0 + 8) * NH + n], W2[(k0 + 9) * NH + n]));
    }
    for (uint32_t i = threadIdx.x; i < (uint32_t)NH; i += blockDim.x) {
        f->b1[i] = w[OFF_B1 + i];
        f->b2[i] = w[OFF_B2 + i];
        f->w3[i] = w[OFF_W3 + i];
    }
    if (threadIdx.x == 0) f->b3 = w[OFF_B3];
}

constexpr int INF_WARPS = 4;

// y[r] = MLP(x[r]) for rows of 16 transformed features (12 used). Each warp
// takes 16 rows at a time.
__global__ void __launch_bounds__(INF_WARPS * 32)
k_mlp_infer(const float *x, uint64_t rows, const MlpFrag *fg, float *y) {
    __shared__ MlpFrag f;
    for (uint32_t i = threadIdx.x; i < sizeof(MlpFrag) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(&f)[i] = reinterpret_cast<const uint32_t *>(fg)[i];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, grp = lane >> 2, tig = lane & 3u;
    const uint64_t warp = blockIdx.x * (uint64_t)INF_WARPS + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * INF_WARPS;
    for (uint64_t r0 = warp * 16; r0 < rows; r0 += nwarps * 16) {
        const uint64_t ra = r0 + grp, rb = r0 + grp + 8;
        auto xv = [&](uint64_t r, uint32_t c) { return r < rows ? x[r * 16 + c] : 0.f; };
        uint32_t a[4];
        a[0] = pack_bf16(xv(ra, 2 * tig), xv(ra, 2 * tig + 1));
        a[1] = pack_bf16(xv(rb, 2 * tig), xv(rb, 2 * tig + 1));
        a[2] = pack_bf16(xv(ra, 2 * tig + 8), xv(ra, 2 * tig + 9));
        a[3] = pack_bf16(xv(rb, 2 * tig + 8), xv(rb, 2 * tig + 9));
        // layer 1: 8 n-tiles of 8 columns
        float h1[NH / 8][4];
#pragma unroll
        for (int j = 0; j < NH / 8; ++j) {
            const float bl = f.b1[8 * j + 2 * tig], bh = f.b1[8 * j + 2 * tig + 1];
            h1[j][0] = bl;
            h1[j][1] = bh;
            h1[j][2] = bl;
            h1[j][3] = bh;
            mma_bf16(h1[j], a, f.w1[j][lane].x, f.w1[j][lane].y);
        }
        // relu, and re-pack as layer 2's A fragments (k-tile kk = n-tiles 2kk, 2kk+1)
        uint32_t a2[NH / 16][4];
#pragma unroll
        for (int kk = 0; kk < NH / 16; ++kk) {
            const float *c0 = h1[2 * kk], *c1 = h1[2 * kk + 1];
            a2[kk][0] = pack_bf16(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
            a2[kk][1] = pack_bf16(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
            a2[kk][2] = pack_bf16(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
            a2[kk][3] = pack_bf16(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
        }
        // layer 2 and layer 3 (a dot product with W3, on the CUDA cores)
        float ya = 0.f, yb = 0.f;
#pragma unroll
        for (int j = 0; j < NH / 8; ++j) {
            const float bl = f.b2[8 * j + 2 * tig], bh = f.b2[8 * j + 2 * tig + 1];
            float h2[4] = {bl, bh, bl, bh};
#pragma unroll
            for (int kk = 0; kk < NH / 16; ++kk) mma_bf16(h2, a2[kk], f.w2[kk][j][lane].x, f.w2[kk][j][lane].y);
            const float wl = f.w3[8 * j + 2 * tig], wh = f.w3[8 * j + 2 * tig + 1];
            ya += fmaxf(h2[0], 0.f) * wl + fmaxf(h2[1], 0.f) * wh;
            yb += fmaxf(h2[2], 0.f) * wl + fmaxf(h2[3], 0.f) * wh;
        }
        // sum over the 4 lanes of a group (they hold the row's 64 columns)
        ya += __shfl_xor_sync(FULL, ya, 1);
        ya += __shfl_xor_sync(FULL, ya, 2);
        yb += __shfl_xor_sync(FULL, yb, 1);
        yb += __shfl_xor_sync(FULL, yb, 2);
        if (tig == 0) {
            if (ra < rows) y[ra] = ya + f.b3;
            if (rb < rows) y[rb] = yb + f.b3;
        }
    }
}

// ----- training -----------------------------------------------------------

constexpr int TR_THREADS = 256;

// Per sample: transformed features x (16, 12 used), the forward pass with
// the inference's roundings (inputs, W1, W2 and the first hidden layer in
// BF16; W3, biases, the second hidden layer and the output in FP32), and the
// backward pass down to the pre-activation gradients of both hidden layers.
__global__ void __launch_bounds__(TR_THREADS)
k_train_fwd_bwd(const float *x, const float *label, uint64_t b0, uint32_t bsz, const float *wq,
                float *h1o, float *h2o, float *g1o, float *g2o, float *dyo, float *loss_part) {
    __shared__ float W[MLP_NPARAM];
    for (uint32_t i = threadIdx.x; i < (uint32_t)MLP_NPARAM; i += blockDim.x) W[i] = wq[i];
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float lsum = 0.f;
    if (i < bsz) {
        const uint64_t r = b0 + i;
        float xi[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k) xi[k] = bf16_round(x[r * 16 + k]);
        float h1[NH], h2[NH];
        for (int j = 0; j < NH; ++j) {
            float s = W[OFF_B1 + j];
#pragma unroll
            for (int k = 0; k < NIN; ++k) s += xi[k] * W[OFF_W1 + k * NH + j];
            h1[j] = bf16_round(fmaxf(s, 0.f));
        }
        for (int j = 0; j < NH; ++j) {
            float s = W[OFF_B2 + j];
            for (int k = 0; k < NH; ++k) s += h1[k] * W[OFF_W2 + k * NH + j];
            h2[j] = fmaxf(s, 0.f);
        }
        float y = W[OFF_B3];
        for (int j = 0; j < NH; ++j) y += h2[j] * W[OFF_W3 + j];
        const float diff = y - label[r];
        lsum = diff * diff;
        const float dy = 2.f * diff / (float)bsz;
        dyo[i] = dy;
        float g2[NH];
        for (int j = 0; j < NH; ++j) {
            g2[j] = h2[j] > 0.f ? dy * W[OFF_W3 + j] : 0.f;
            h1o[(uint64_t)i * NH + j] = h1[j];
            h2o[(uint64_t)i * NH + j] = h2[j];
            g2o[(uint64_t)i * NH + j] = g2[j];
        }
        for (int k = 0; k < NH; ++k) {
            float s = 0.f;
            for (int j = 0; j < NH; ++j) s += g2[j] * W[OFF_W2 + k * NH + j];
            g1o[(uint64_t)i * NH + k] = h1[k] > 0.f ? s : 0.f;
        }
    }
    // block sum of the squared errors, in a fixed order
    __shared__ float red[TR_THREADS];
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (uint32_t st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

constexpr uint32_t TR_SLICE = 512;  // samples per partial-gradient block

// Partial gradients over a slice of samples: one thread per parameter
// group, summing the slice in sample order.
__global__ void __launch_bounds__(TR_THREADS)
k_train_grad_part(const float *x, uint64_t b0, uint32_t bsz, const float *h1, const float *h2,
                  const float *g1, const float *g2, const float *dy, float *part) {
    const uint32_t s0 = blockIdx.x * TR_SLICE;
    const uint32_t s1 = min(bsz, s0 + TR_SLICE);
    float *out = part + (uint64_t)blockIdx.x * MLP_NPARAM;
    for (uint32_t p = threadIdx.x; p < (uint32_t)MLP_NPARAM; p += blockDim.x) {
        float s = 0.f;
        if (p < (uint32_t)OFF_B1) {  // W1[k][j] += x_k * g1_j
            const uint32_t k = p / NH, j = p % NH;
            for (uint32_t i = s0; i < s1; ++i) s += bf16_round(x[(b0 + i) * 16 + k]) * g1[(uint64_t)i * NH + j];
        } else if (p < (uint32_t)OFF_W2) {
            const uint32_t j = p - OFF_B1;
            for (uint32_t i = s0; i < s1; ++i) s += g1[(uint64_t)i * NH + j];
        } else if (p < (uint32_t)OFF_B2) {  // W2[k][j] += h1_k * g2_j
            const uint32_t k = (p - OFF_W2) / NH, j = (p - OFF_W2) % NH;
            for (uint32_t i = s0; i < s1; ++i) s += h1[(uint64_t)i * NH + k] * g2[(uint64_t)i * NH + j];
        } else if (p < (uint32_t)OFF_W3) {
            const uint32_t j = p - OFF_B2;
            for (uint32_t i = s0; i < s1; ++i) s += g2[(uint64_t)i * NH + j];
        } else if (p < (uint32_t)OFF_B3) {  // W3[j] += h2_j * dy
            const uint32_t j = p - OFF_W3;
            for (uint32_t i = s0; i < s1; ++i) s += h2[(uint64_t)i * NH + j] * dy[i];
        } else {
            for (uint32_t i = s0; i < s1; ++i) s += dy[i];
        }
        out[p] = s;
    }
}

// grad[p] = sum of the partials in slice order; then Adam on the FP32
// master weights and a BF16-rounded copy for the next forward pass.
__global__ void k_train_adam(const float *part, uint32_t nparts, float *grad, float *w, float *wq,
                             float *m, float *v, float lr, float b1, float b2, float eps,
                             float b1t, float b2t, int apply) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < (uint32_t)MLP_NPARAM;
         p += gridDim.x * blockDim.x) {
        float g = 0.f;
        for (uint32_t k = 0; k < nparts; ++k) g += part[(uint64_t)k * MLP_NPARAM + p];
        grad[p] = g;
        if (!apply) continue;
        const float mi = b1 * m[p] + (1.f - b1) * g;
        const float vi = b2 * v[p] + (1.f - b2) * g * g;
        m[p] = mi;
        v[p] = vi;
        const float mh = mi / (1.f - b1t), vh = vi / (1.f - b2t);
        const float wi = w[p] - lr * mh / (sqrtf(vh) + eps);
        w[p] = wi;
        wq[p] = quantised(p, wi);
    }
}

__global__ void k_round_weights(const float *w, float *wq) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < (uint32_t)MLP_NPARAM;
         p += gridDim.x * blockDim.x)
        wq[p] = quantised(p, w[p]);
}

// Transformed features of trace rows (round, vertex, 12 features).
__global__ void k_rows_to_x(const long long *rows, uint64_t n, float *x) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 16; ++k) x[r * 16 + k] = k < NIN ? feature_transform(rows[r * 14 + 2 + k]) : 0.f;
    }
}

// Training target of trace rows: the transformed score
// x = edge difference + 2 * hierarchy depth (features 4 and 6).
__global__ void k_targets(const long long *rows, uint64_t n, float *y) {
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x)
        y[r] = feature_transform(rows[r * 14 + 2 + 4] + 2 * rows[r * 14 + 2 + 6]);
}

}  // namespace

void mlp_targets(const long long *rows, uint64_t n, float *y, cudaStream_t st) {
    if (n == 0) return;
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sm_count() * 8);
    k_targets<<<(unsigned)blocks, 256, 0, st>>>(rows, n, y);
    CH_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------

MlpDevice::MlpDevice() = default;
MlpDevice::~MlpDevice() = default;

void MlpDevice::load(const float *host_weights, cudaStream_t st) {
    weights.alloc(MLP_NPARAM);
    frag.alloc((sizeof(MlpFrag) + 3) / 4);
    CH_CUDA_TRY(cudaMemcpyAsync(weights.ptr, host_weights, MLP_NPARAM * sizeof(float),
                                cudaMemcpyHostToDevice, st));
    k_mlp_prepare<<<1, 256, 0, st>>>(weights.ptr, reinterpret_cast<MlpFrag *>(frag.ptr));
    CH_CHECK_LAUNCH();
}

void MlpDevice::infer(const float *x, uint64_t rows, float *y, cudaStream_t st) const {
    if (!rows) return;
    const int blocks = grid_for((rows + 15) / 16, INF_WARPS, device_sm_count() * 8);
    k_mlp_infer<<<blocks, INF_WARPS * 32, 0, st>>>(x, rows, reinterpret_cast<const MlpFrag *>(frag.ptr), y);
    CH_CHECK_LAUNCH();
}

void rows_to_features(const long long *rows, uint64_t n, float *x, cudaStream_t st) {
    if (!n) return;
    k_rows_to_x<<<grid_for(n, 256, device_sm_count() * 8), 256, 0, st>>>(rows, n, x);
    CH_CHECK_LAUNCH();
}

void mlp_train(const long long *rows, const float *labels, uint64_t n, const ch_train_params_t *tp,
               float *weights_io, float *loss_out, float *grad_out, cudaStream_t st) {
    DevBuf<float> x, w, wq, m, v, grad, h1, h2, g1, g2, dy, part, lpart;
    x.alloc(n * 16);
    rows_to_features(rows, n, x.ptr, st);
    w.alloc(MLP_NPARAM);
    wq.alloc(MLP_NPARAM);
    m.alloc(MLP_NPARAM);
    v.alloc(MLP_NPARAM);
    grad.alloc(MLP_NPARAM);
    m.zero(st);
    v.zero(st);
    CH_CUDA_TRY(cudaMemcpyAsync(w.ptr, weights_io, MLP_NPARAM * 4, cudaMemcpyDeviceToDevice, st));
    k_round_weights<<<20, 256, 0, st>>>(w.ptr, wq.ptr);
    CH_CHECK_LAUNCH();
    const uint32_t B = std::max<uint32_t>(1, std::min<uint64_t>(tp->batch, n));
    h1.alloc((uint64_t)B * MLP_NH);
    h2.alloc((uint64_t)B * MLP_NH);
    g1.alloc((uint64_t)B * MLP_NH);
    g2.alloc((uint64_t)B * MLP_NH);
    dy.alloc(B);
    const uint32_t nparts = (B + TR_SLICE - 1) / TR_SLICE;
    part.alloc((uint64_t)nparts * MLP_NPARAM);
    const uint32_t fb_blocks = (B + TR_THREADS - 1) / TR_THREADS;
    lpart.alloc(fb_blocks);
    std::vector<float> hl(fb_blocks);
    float b1t = 1.f, b2t = 1.f;
    const bool apply = tp->epochs > 0;
    const uint32_t epochs = apply ? tp->epochs : 1;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        double ep_loss = 0;
        for (uint64_t b0 = 0; b0 < n; b0 += B) {
            const uint32_t bsz = (uint32_t)std::min<uint64_t>(B, n - b0);
            const uint32_t fbb = (bsz + TR_THREADS - 1) / TR_THREADS;
            k_train_fwd_bwd<<<fbb, TR_THREADS, 0, st>>>(x.ptr, labels, b0, bsz, wq.ptr, h1.ptr,
                                                        h2.ptr, g1.ptr, g2.ptr, dy.ptr, lpart.ptr);
            CH_CHECK_LAUNCH();
            const uint32_t np = (bsz + TR_SLICE - 1) / TR_SLICE;
            k_train_grad_part<<<np, TR_THREADS, 0, st>>>(x.ptr, b0, bsz, h1.ptr, h2.ptr, g1.ptr,
                                                         g2.ptr, dy.ptr, part.ptr);
            CH_CHECK_LAUNCH();
            b1t *= tp->beta1;
            b2t *= tp->beta2;
            k_train_adam<<<20, 256, 0, st>>>(part.ptr, np, grad.ptr, w.ptr, wq.ptr, m.ptr, v.ptr,
                                              tp->lr, tp->beta1, tp->beta2, tp->eps, b1t, b2t,
                                              apply ? 1 : 0);
            CH_CHECK_LAUNCH();
            CH_CUDA_TRY(cudaMemcpyAsync(hl.data(), lpart.ptr, fbb * 4, cudaMemcpyDeviceToHost, st));
            CH_CUDA_TRY(cudaStreamSynchronize(st));
            for (uint32_t k = 0; k < fbb; ++k) ep_loss += hl[k];
            if (!apply) break;  // gradient of the first batch only
        }
        if (loss_out) loss_out[ep] = (float)(ep_loss / (double)(apply ? n : std::min<uint64_t>(B, n)));
    }
    if (apply)
        CH_CUDA_TRY(cudaMemcpyAsync(weights_io, w.ptr, MLP_NPARAM * 4, cudaMemcpyDeviceToDevice, st));
    if (grad_out)
        CH_CUDA_TRY(cudaMemcpyAsync(grad_out, grad.ptr, MLP_NPARAM * 4, cudaMemcpyDeviceToDevice, st));
    CH_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace gbch
