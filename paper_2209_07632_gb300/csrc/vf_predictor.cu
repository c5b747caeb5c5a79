// The learned part of assembly (not in the paper): a small MLP that
// predicts, from a candidate block's cluster geometry, the rank bin of its
// truncated SVD or that the SVD cannot win (Algorithm 3's probe outcome).
// Assembly uses the prediction as the probe's starting rank and to skip
// probes predicted to lose; the probe and the byte test still decide.
//
// Network: x (VF_PRED_NFEAT) -> standardise -> W1 (64) ReLU -> W2 (64) ReLU
// -> W3 (VF_PRED_NCLASS) -> softmax; loss = mean cross-entropy.  The forward
// pass uses FP16-rounded weights with FP32 activations and accumulation;
// training keeps FP32 master weights and treats the rounding as identity
// in the backward pass (the gradient is taken at the rounded weights).
// Every sum has a fixed order, so training is bit-reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_fp16.h>

#include "vf_internal.cuh"
#include "vf_predictor.cuh"

struct vf_rank_predictor {
    int device = 0;
    uint64_t seed = 0;
    std::vector<float> w;                      // master weights, VF_PRED_NPARAM
    std::vector<float> mu, sd;                 // feature standardisation
    std::vector<float> m1, m2;                 // Adam moments
    int64_t step = 0;
};

namespace vf {

constexpr int kH = 64;
constexpr int kF = VF_PRED_NFEAT;
constexpr int kC = VF_PRED_NCLASS;
// flat parameter layout
constexpr int oW1 = 0, oB1 = oW1 + kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kC * kH, kNP = oB3 + kC;
static_assert(kNP == VF_PRED_NPARAM, "parameter count");

// Forward for the samples idx[0..n) (or 0..n when idx is NULL): logits ->
// probabilities p (n x C); the hidden activations h1, h2 (n x 64) are kept
// for the backward pass when non-NULL.  One thread per sample; weights
// (FP16-rounded) and the standardisation in shared memory.
__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ X, const int64_t* __restrict__ idx,
                                                 int64_t n, const __half* __restrict__ wh,
                                                 const float* __restrict__ mu, const float* __restrict__ sd,
                                                 float* __restrict__ P, float* __restrict__ H1,
                                                 float* __restrict__ H2) {
    __shared__ float w[kNP];
    __shared__ float smu[kF], ssd[kF];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) w[i] = __half2float(wh[i]);
    for (int i = threadIdx.x; i < kF; i += blockDim.x) {
        smu[i] = mu[i];
        ssd[i] = sd[i];
    }
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t r = idx ? idx[s] : s;
    float x[kF];
#pragma unroll
    for (int f = 0; f < kF; ++f) x[f] = (X[r * kF + f] - smu[f]) / ssd[f];
    float h1[kH], h2[kH];
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
        float a = w[oB1 + j];
#pragma unroll
        for (int f = 0; f < kF; ++f) a = fmaf(w[oW1 + j * kF + f], x[f], a);
        h1[j] = fmaxf(a, 0.f);
    }
#pragma unroll 2
    for (int j = 0; j < kH; ++j) {
        float a = w[oB2 + j];
#pragma unroll
        for (int k = 0; k < kH; ++k) a = fmaf(w[oW2 + j * kH + k], h1[k], a);
        h2[j] = fmaxf(a, 0.f);
    }
    float z[kC];
    float zmax = -INFINITY;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        float a = w[oB3 + c];
#pragma unroll
        for (int k = 0; k < kH; ++k) a = fmaf(w[oW3 + c * kH + k], h2[k], a);
        z[c] = a;
        zmax = fmaxf(zmax, a);
    }
    float den = 0.f;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        z[c] = expf(z[c] - zmax);
        den += z[c];
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) P[s * kC + c] = z[c] / den;
    if (H1)
#pragma unroll
        for (int j = 0; j < kH; ++j) H1[s * kH + j] = h1[j];
    if (H2)
#pragma unroll
        for (int j = 0; j < kH; ++j) H2[s * kH + j] = h2[j];
}

// Backward through the activations: dZ = (p - onehot(y)) / n, dA2 = W3^T dZ
// masked by h2 > 0, dA1 = W2^T dA2 masked by h1 > 0; also the standardised
// inputs for the first layer's weight gradient.  One thread per sample.
__global__ void __launch_bounds__(128) k_mlp_bwd(const float* __restrict__ X, const int64_t* __restrict__ idx,
                                                 const int32_t* __restrict__ labels, int64_t n,
                                                 const __half* __restrict__ wh, const float* __restrict__ mu,
                                                 const float* __restrict__ sd, const float* __restrict__ P,
                                                 const float* __restrict__ H1, const float* __restrict__ H2,
                                                 float* __restrict__ DZ, float* __restrict__ DA2,
                                                 float* __restrict__ DA1, float* __restrict__ XS,
                                                 float* __restrict__ nll) {
    __shared__ float w[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) w[i] = __half2float(wh[i]);
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t r = idx ? idx[s] : s;
    const int y = labels[r];
    const float inv = 1.f / (float)n;
    float dz[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) {
        const float p = P[s * kC + c];
        dz[c] = (p - (c == y ? 1.f : 0.f)) * inv;
        DZ[s * kC + c] = dz[c];
    }
    nll[s] = -logf(fmaxf(P[s * kC + y], 1e-30f));
    float da2[kH];
#pragma unroll 4
    for (int k = 0; k < kH; ++k) {
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < kC; ++c) a = fmaf(w[oW3 + c * kH + k], dz[c], a);
        da2[k] = H2[s * kH + k] > 0.f ? a : 0.f;
        DA2[s * kH + k] = da2[k];
    }
#pragma unroll 2
    for (int k = 0; k < kH; ++k) {
        float a = 0.f;
#pragma unroll
        for (int j = 0; j < kH; ++j) a = fmaf(w[oW2 + j * kH + k], da2[j], a);
        DA1[s * kH + k] = H1[s * kH + k] > 0.f ? a : 0.f;
    }
#pragma unroll
    for (int f = 0; f < kF; ++f) XS[s * kF + f] = (X[r * kF + f] - mu[f]) / sd[f];
}

// Parameter gradients: one thread per parameter, summing over the samples
// in order (dW = sum_s delta_s a_s^T, db = sum_s delta_s).
__global__ void k_mlp_wgrad(int64_t n, const float* __restrict__ XS, const float* __restrict__ H1,
                            const float* __restrict__ H2, const float* __restrict__ DZ,
                            const float* __restrict__ DA2, const float* __restrict__ DA1,
                            float* __restrict__ g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNP) return;
    const float* D;
    const float* A = nullptr;
    int ld, la, row, col;
    if (i < oB1) { D = DA1; ld = kH; A = XS; la = kF; row = (i - oW1) / kF; col = (i - oW1) % kF; }
    else if (i < oW2) { D = DA1; ld = kH; row = i - oB1; col = 0; la = 0; }
    else if (i < oB2) { D = DA2; ld = kH; A = H1; la = kH; row = (i - oW2) / kH; col = (i - oW2) % kH; }
    else if (i < oW3) { D = DA2; ld = kH; row = i - oB2; col = 0; la = 0; }
    else if (i < oB3) { D = DZ; ld = kC; A = H2; la = kH; row = (i - oW3) / kH; col = (i - oW3) % kH; }
    else { D = DZ; ld = kC; row = i - oB3; col = 0; la = 0; }
    float acc = 0.f;
    if (A)
        for (int64_t s = 0; s < n; ++s) acc = fmaf(D[s * ld + row], A[s * la + col], acc);
    else
        for (int64_t s = 0; s < n; ++s) acc += D[s * ld + row];
    g[i] = acc;
}

// Adam on the master weights, then the FP16 copy the forward pass uses.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ g, __half* __restrict__ wh, float lr, float b1c, float b2c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float v = w[i] - lr * (a / b1c) / (sqrtf(b / b2c) + eps);
    w[i] = v;
    wh[i] = __float2half_rn(v);
}

__global__ void k_to_half(const float* __restrict__ w, __half* __restrict__ wh) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNP) wh[i] = __float2half_rn(w[i]);
}

// Device state of one pass over n samples.
struct MlpBufs {
    dbuf<float> X, P, H1, H2, DZ, DA2, DA1, XS, nll, g, w, m1, m2, mu, sd;
    dbuf<__half> wh;
    dbuf<int32_t> labels;
    dbuf<int64_t> idx;
};

static vf_status upload_model(const vf_rank_predictor* p, MlpBufs& b) {
    VF_TRY(b.w.upload(p->w));
    VF_TRY(b.mu.upload(p->mu));
    VF_TRY(b.sd.upload(p->sd));
    VF_TRY(b.wh.alloc(kNP));
    k_to_half<<<(kNP + 255) / 256, 256>>>(b.w.p, b.wh.p);
    VF_TRY_CUDA(cudaGetLastError());
    return VF_OK;
}

static vf_status alloc_pass(MlpBufs& b, int64_t n, bool backward) {
    VF_TRY(b.P.alloc(std::max<int64_t>(n, 1) * kC));
    if (backward) {
        VF_TRY(b.H1.alloc(std::max<int64_t>(n, 1) * kH));
        VF_TRY(b.H2.alloc(std::max<int64_t>(n, 1) * kH));
        VF_TRY(b.DZ.alloc(std::max<int64_t>(n, 1) * kC));
        VF_TRY(b.DA2.alloc(std::max<int64_t>(n, 1) * kH));
        VF_TRY(b.DA1.alloc(std::max<int64_t>(n, 1) * kH));
        VF_TRY(b.XS.alloc(std::max<int64_t>(n, 1) * kF));
        VF_TRY(b.nll.alloc(std::max<int64_t>(n, 1)));
        VF_TRY(b.g.alloc(kNP));
    }
    return VF_OK;
}

// forward + backward + parameter gradient on the samples idx (device) of
// b.X / b.labels; the mean loss (host, FP64 sum of the per-sample terms)
static vf_status grad_pass(MlpBufs& b, const int64_t* d_idx, int64_t n, double* loss) {
    const unsigned g = (unsigned)ceil_div(n, 128);
    k_mlp_fwd<<<g, 128>>>(b.X.p, d_idx, n, b.wh.p, b.mu.p, b.sd.p, b.P.p, b.H1.p, b.H2.p);
    k_mlp_bwd<<<g, 128>>>(b.X.p, d_idx, b.labels.p, n, b.wh.p, b.mu.p, b.sd.p, b.P.p, b.H1.p, b.H2.p, b.DZ.p,
                          b.DA2.p, b.DA1.p, b.XS.p, b.nll.p);
    k_mlp_wgrad<<<(kNP + 127) / 128, 128>>>(n, b.XS.p, b.H1.p, b.H2.p, b.DZ.p, b.DA2.p, b.DA1.p, b.g.p);
    VF_TRY_CUDA(cudaGetLastError());
    if (loss) {
        std::vector<float> nl;
        VF_TRY(b.nll.download(nl));
        double s = 0;
        for (int64_t i = 0; i < n; ++i) s += nl[i];
        *loss = s / (double)n;
    }
    return VF_OK;
}

vf_status predictor_classify(const vf_rank_predictor* p, const std::vector<float>& feats, int64_t n,
                             std::vector<int32_t>& cls, std::vector<float>& prob) {
    cls.assign(n, 0);
    prob.assign(n * kC, 0.f);
    if (n == 0) return VF_OK;
    MlpBufs b;
    VF_TRY(upload_model(p, b));
    VF_TRY(b.X.upload(feats));
    VF_TRY(alloc_pass(b, n, false));
    k_mlp_fwd<<<(unsigned)ceil_div(n, 128), 128>>>(b.X.p, nullptr, n, b.wh.p, b.mu.p, b.sd.p, b.P.p, nullptr,
                                                    nullptr);
    VF_TRY_CUDA(cudaGetLastError());
    VF_TRY(b.P.download(prob));
    prob.resize(n * kC);
    for (int64_t i = 0; i < n; ++i) {
        int best = 0;
        for (int c = 1; c < kC; ++c)
            if (prob[i * kC + c] > prob[i * kC + best]) best = c;  // ties: the lower class
        cls[i] = best;
    }
    return VF_OK;
}

// Glorot-uniform initial weights from a counter-based generator.
static void init_weights(vf_rank_predictor* p) {
    p->w.assign(kNP, 0.f);
    auto fill = [&](int off, int fan_out, int fan_in, uint64_t tag) {
        const float a = std::sqrt(6.f / (float)(fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) {
            const uint64_t r = splitmix64(p->seed ^ (tag << 40) ^ (uint64_t)i);
            const float u = (float)((r >> 11) * (1.0 / 9007199254740992.0));  // [0, 1)
            p->w[off + i] = (2.f * u - 1.f) * a;
        }
    };
    fill(oW1, kH, kF, 1);
    fill(oW2, kH, kH, 2);
    fill(oW3, kC, kH, 3);
    p->mu.assign(kF, 0.f);
    p->sd.assign(kF, 1.f);
    p->m1.assign(kNP, 0.f);
    p->m2.assign(kNP, 0.f);
    p->step = 0;
}

}  // namespace vf

using namespace vf;

extern "C" vf_status vf_predictor_create(int32_t device, uint64_t seed, vf_rank_predictor** out) {
    clear_error();
    VF_CHECK(out, VF_E_INVAL, "vf_predictor_create: null argument");
    int nd = 0;
    VF_TRY_CUDA(cudaGetDeviceCount(&nd));
    VF_CHECK(device >= 0 && device < nd, VF_E_INVAL, "vf_predictor_create: no device %d", device);
    auto p = new vf_rank_predictor();
    p->device = device;
    p->seed = seed;
    init_weights(p);
    *out = p;
    return VF_OK;
}

extern "C" void vf_predictor_destroy(vf_rank_predictor* p) { delete p; }

extern "C" vf_status vf_predictor_params(vf_rank_predictor* p, float* get, const float* set) {
    clear_error();
    VF_CHECK(p, VF_E_INVAL, "vf_predictor_params: null predictor");
    if (get) {
        std::copy(p->w.begin(), p->w.end(), get);
        std::copy(p->mu.begin(), p->mu.end(), get + kNP);
        std::copy(p->sd.begin(), p->sd.end(), get + kNP + kF);
    }
    if (set) {
        for (int i = kNP + kF; i < kNP + 2 * kF; ++i)
            VF_CHECK(set[i] > 0.f && std::isfinite(set[i]), VF_E_INVAL,
                     "vf_predictor_params: feature scales must be positive");
        p->w.assign(set, set + kNP);
        p->mu.assign(set + kNP, set + kNP + kF);
        p->sd.assign(set + kNP + kF, set + kNP + 2 * kF);
        p->m1.assign(kNP, 0.f);
        p->m2.assign(kNP, 0.f);
        p->step = 0;
    }
    return VF_OK;
}

extern "C" vf_status vf_predictor_grad(vf_rank_predictor* p, const float* feats, const int32_t* labels, int64_t n,
                                       double* loss, float* grad) {
    clear_error();
    VF_CHECK(p && feats && labels && n > 0, VF_E_INVAL, "vf_predictor_grad: bad argument");
    for (int64_t i = 0; i < n; ++i)
        VF_CHECK(labels[i] >= 0 && labels[i] < kC, VF_E_INVAL, "vf_predictor_grad: label out of range");
    device_guard g(p->device);
    MlpBufs b;
    VF_TRY(upload_model(p, b));
    VF_TRY(b.X.upload(std::vector<float>(feats, feats + n * kF)));
    VF_TRY(b.labels.upload(std::vector<int32_t>(labels, labels + n)));
    VF_TRY(alloc_pass(b, n, true));
    VF_TRY(grad_pass(b, nullptr, n, loss));
    if (grad) {
        std::vector<float> hg;
        VF_TRY(b.g.download(hg));
        std::copy(hg.begin(), hg.begin() + kNP, grad);
    }
    return VF_OK;
}

extern "C" vf_status vf_predictor_train(vf_rank_predictor* p, const float* feats, const int32_t* labels, int64_t n,
                                        int32_t epochs, int32_t batch, float lr, double* final_loss) {
    clear_error();
    VF_CHECK(p && feats && labels && n > 0 && epochs >= 0 && batch > 0 && lr > 0.f, VF_E_INVAL,
             "vf_predictor_train: bad argument");
    for (int64_t i = 0; i < n; ++i)
        VF_CHECK(labels[i] >= 0 && labels[i] < kC, VF_E_INVAL, "vf_predictor_train: label out of range");
    device_guard g(p->device);
    // standardisation from the training set (FP64 sums)
    for (int f = 0; f < kF; ++f) {
        double s = 0, s2 = 0;
        for (int64_t i = 0; i < n; ++i) {
            s += feats[i * kF + f];
            s2 += (double)feats[i * kF + f] * feats[i * kF + f];
        }
        const double m = s / n, v = std::max(s2 / n - m * m, 0.0);
        p->mu[f] = (float)m;
        p->sd[f] = (float)std::max(std::sqrt(v), 1e-6);
    }
    MlpBufs b;
    VF_TRY(upload_model(p, b));
    VF_TRY(b.m1.upload(p->m1));
    VF_TRY(b.m2.upload(p->m2));
    VF_TRY(b.X.upload(std::vector<float>(feats, feats + n * kF)));
    VF_TRY(b.labels.upload(std::vector<int32_t>(labels, labels + n)));
    const int64_t bs = std::min<int64_t>(batch, n);
    VF_TRY(alloc_pass(b, std::max<int64_t>(bs, n), true));
    VF_TRY(b.idx.alloc(n));
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    for (int32_t e = 0; e < epochs; ++e) {
        // Fisher-Yates with a counter-based generator: the same seed, the same order
        for (int64_t i = n - 1; i > 0; --i) {
            const uint64_t r = splitmix64(p->seed ^ ((uint64_t)(e + 1) << 32) ^ (uint64_t)i);
            std::swap(order[i], order[(int64_t)(r % (uint64_t)(i + 1))]);
        }
        VF_TRY_CUDA(cudaMemcpy(b.idx.p, order.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
        for (int64_t s0 = 0; s0 + bs <= n; s0 += bs) {
            VF_TRY(grad_pass(b, b.idx.p + s0, bs, nullptr));
            p->step++;
            const float b1c = 1.f - std::pow(0.9f, (float)p->step), b2c = 1.f - std::pow(0.999f, (float)p->step);
            k_adam<<<(kNP + 255) / 256, 256>>>(b.w.p, b.m1.p, b.m2.p, b.g.p, b.wh.p, lr, b1c, b2c);
            VF_TRY_CUDA(cudaGetLastError());
        }
    }
    VF_TRY(b.w.download(p->w));
    VF_TRY(b.m1.download(p->m1));
    VF_TRY(b.m2.download(p->m2));
    if (final_loss) VF_TRY(grad_pass(b, nullptr, n, final_loss));
    VF_TRY_CUDA(cudaDeviceSynchronize());
    return VF_OK;
}

extern "C" vf_status vf_predictor_predict(const vf_rank_predictor* p, const float* feats, int64_t n, int32_t* cls,
                                          float* prob) {
    clear_error();
    VF_CHECK(p && feats && n >= 0 && cls, VF_E_INVAL, "vf_predictor_predict: bad argument");
    device_guard g(p->device);
    std::vector<int32_t> c;
    std::vector<float> pr;
    VF_TRY(predictor_classify(p, std::vector<float>(feats, feats + n * kF), n, c, pr));
    std::copy(c.begin(), c.end(), cls);
    if (prob) std::copy(pr.begin(), pr.end(), prob);
    return VF_OK;
}
