// Learned cost model: a small MLP that predicts the log time of a
// contraction step (GEMM under a tile configuration, or a permutation) from
// the step's shape features.  Trained on the autotuner's own timings, on the
// GPU, by the kernels below (FP32, deterministic: every reduction is a fixed
// loop, no atomics); used to rank tile configurations without timing them
// and to compare slicing plans by predicted time.
//
// Layout: in -> H -> H -> H -> 1, ReLU on the hidden layers.  Parameters are
// one flat FP32 vector: W1[in][H], b1[H], W2[H][H], b2[H], W3[H][H], b3[H],
// W4[H][1], b4[1] (row-major, "x W + b").
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "plan.h"

namespace {

constexpr int kLayers = 4;

__global__ void linear_fwd(const float *__restrict__ X, const float *__restrict__ W,
                           const float *__restrict__ b, float *__restrict__ Y, int B, int I, int O,
                           int relu) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (o >= O || r >= B) return;
    float acc = b[o];
    const float *x = X + (int64_t)r * I;
    for (int i = 0; i < I; ++i) acc = fmaf(x[i], W[(int64_t)i * O + o], acc);
    Y[(int64_t)r * O + o] = relu ? fmaxf(acc, 0.0f) : acc;
}

// dX[b][i] = sum_o dZ[b][o] W[i][o], then times the ReLU mask of X (the
// previous layer's output, > 0 where its pre-activation was > 0)
__global__ void linear_bwd_data(const float *__restrict__ dZ, const float *__restrict__ W,
                                const float *__restrict__ Xprev, float *__restrict__ dX, int B,
                                int I, int O) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= I || r >= B) return;
    float acc = 0.0f;
    const float *dz = dZ + (int64_t)r * O;
    const float *w = W + (int64_t)i * O;
    for (int o = 0; o < O; ++o) acc = fmaf(dz[o], w[o], acc);
    dX[(int64_t)r * I + i] = Xprev[(int64_t)r * I + i] > 0.0f ? acc : 0.0f;
}

// dW[i][o] = sum_b X[b][i] dZ[b][o]; db[o] = sum_b dZ[b][o] (i == I row)
__global__ void linear_bwd_weight(const float *__restrict__ X, const float *__restrict__ dZ,
                                  float *__restrict__ dW, float *__restrict__ db, int B, int I,
                                  int O) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;   // 0..I (I = bias row)
    if (o >= O || i > I) return;
    float acc = 0.0f;
    if (i < I) {
        for (int r = 0; r < B; ++r) acc = fmaf(X[(int64_t)r * I + i], dZ[(int64_t)r * O + o], acc);
        dW[(int64_t)i * O + o] = acc;
    } else {
        for (int r = 0; r < B; ++r) acc += dZ[(int64_t)r * O + o];
        db[o] = acc;
    }
}

// mean squared error over B predictions: dY = 2 (y - t) / B, loss[0]
__global__ void mse_loss(const float *__restrict__ y, const float *__restrict__ t, float *dy,
                         double *loss, int B) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < B; r += blockDim.x) {
        const float d = y[r] - t[r];
        dy[r] = 2.0f * d / (float)B;
        s += (double)d * (double)d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = sh[0] / (double)B;
}

__global__ void adam_step(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                          float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                          float bc1, float bc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void gather_rows(const float *__restrict__ src, const int32_t *__restrict__ idx,
                            float *__restrict__ dst, int B, int width) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c >= width || r >= B) return;
    dst[(int64_t)r * width + c] = src[(int64_t)idx[r] * width + c];
}

uint64_t splitmix(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct tn_cost_model_s {
    int in = TN_COST_NFEAT, hidden = 128;
    int dims[kLayers + 1];
    int64_t off_w[kLayers], off_b[kLayers], n_params = 0;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    int64_t adam_t = 0;
    // activations for a batch (sized on demand)
    int cap_b = 0;
    float *d_act[kLayers + 1] = {};   // layer inputs/outputs: act[0] = X, act[L] = y
    float *d_dz[kLayers + 1] = {};
    float *d_t = nullptr;
    double *d_loss = nullptr;
    int32_t *d_idx = nullptr;
};

namespace {

int fail_msg(int code, const std::string &m) { return tn::record_error(code, m); }

void free_batch(tn_cost_model_s *M) {
    for (int l = 0; l <= kLayers; ++l) {
        cudaFree(M->d_act[l]);
        cudaFree(M->d_dz[l]);
        M->d_act[l] = M->d_dz[l] = nullptr;
    }
    cudaFree(M->d_t);
    cudaFree(M->d_loss);
    cudaFree(M->d_idx);
    M->d_t = nullptr;
    M->d_loss = nullptr;
    M->d_idx = nullptr;
    M->cap_b = 0;
}

cudaError_t ensure_batch(tn_cost_model_s *M, int B) {
    if (B <= M->cap_b) return cudaSuccess;
    free_batch(M);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l <= kLayers && e == cudaSuccess; ++l) {
        e = cudaMalloc(&M->d_act[l], (size_t)B * M->dims[l] * 4);
        if (e == cudaSuccess) e = cudaMalloc(&M->d_dz[l], (size_t)B * M->dims[l] * 4);
    }
    if (e == cudaSuccess) e = cudaMalloc(&M->d_t, (size_t)B * 4);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_loss, 8);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_idx, (size_t)B * 4);
    if (e == cudaSuccess) M->cap_b = B;
    return e;
}

// forward over d_act[0] (B rows) -> d_act[L]
void forward(tn_cost_model_s *M, int B, cudaStream_t s) {
    for (int l = 0; l < kLayers; ++l) {
        const int I = M->dims[l], O = M->dims[l + 1];
        dim3 g((O + 127) / 128, B);
        linear_fwd<<<g, 128, 0, s>>>(M->d_act[l], M->d_p + M->off_w[l], M->d_p + M->off_b[l],
                                     M->d_act[l + 1], B, I, O, l < kLayers - 1);
    }
}

// loss and gradient (into d_g) for targets in d_t
void backward(tn_cost_model_s *M, int B, cudaStream_t s) {
    mse_loss<<<1, 256, 0, s>>>(M->d_act[kLayers], M->d_t, M->d_dz[kLayers], M->d_loss, B);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int I = M->dims[l], O = M->dims[l + 1];
        linear_bwd_weight<<<dim3((O + 127) / 128, I + 1), 128, 0, s>>>(
            M->d_act[l], M->d_dz[l + 1], M->d_g + M->off_w[l], M->d_g + M->off_b[l], B, I, O);
        if (l > 0)
            linear_bwd_data<<<dim3((I + 127) / 128, B), 128, 0, s>>>(M->d_dz[l + 1], M->d_p + M->off_w[l],
                                                                     M->d_act[l], M->d_dz[l], B, I, O);
    }
}

}  // namespace

extern "C" {

int tn_cost_model_create(int32_t hidden, uint64_t seed, tn_cost_model_t **out) {
    if (!out || hidden < 1 || hidden > 1024) return fail_msg(TN_EINVAL, "hidden must be in 1..1024");
    auto *M = new tn_cost_model_s();
    M->hidden = hidden;
    M->dims[0] = TN_COST_NFEAT;
    for (int l = 1; l < kLayers; ++l) M->dims[l] = hidden;
    M->dims[kLayers] = 1;
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        M->off_w[l] = off;
        off += (int64_t)M->dims[l] * M->dims[l + 1];
        M->off_b[l] = off;
        off += M->dims[l + 1];
    }
    M->n_params = off;
    // He-uniform initialisation from a splitmix64 stream; biases zero
    std::vector<float> h(off, 0.0f);
    uint64_t st = seed;
    for (int l = 0; l < kLayers; ++l) {
        const float lim = std::sqrt(6.0f / (float)M->dims[l]);
        for (int64_t k = 0; k < (int64_t)M->dims[l] * M->dims[l + 1]; ++k) {
            const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
            h[M->off_w[l] + k] = (float)((2.0 * u - 1.0) * lim);
        }
    }
    cudaError_t e = cudaMalloc(&M->d_p, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_g, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_m, off * 4);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_v, off * 4);
    if (e == cudaSuccess) e = cudaMemcpy(M->d_p, h.data(), off * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(M->d_m, 0, off * 4);
    if (e == cudaSuccess) e = cudaMemset(M->d_v, 0, off * 4);
    if (e != cudaSuccess) {
        tn_cost_model_destroy(M);
        return fail_msg(TN_ECUDA, std::string("cost model allocation: ") + cudaGetErrorString(e));
    }
    *out = M;
    return TN_OK;
}

void tn_cost_model_destroy(tn_cost_model_t *M) {
    if (!M) return;
    free_batch(M);
    cudaFree(M->d_p);
    cudaFree(M->d_g);
    cudaFree(M->d_m);
    cudaFree(M->d_v);
    delete M;
}

int tn_cost_model_params(tn_cost_model_t *M, float *h_params, int64_t capacity, int64_t *n_params,
                         int32_t set) {
    if (!M) return fail_msg(TN_EINVAL, "NULL model");
    if (n_params) *n_params = M->n_params;
    if (!h_params) return TN_OK;
    if (capacity < M->n_params) return fail_msg(TN_EINVAL, "capacity below the parameter count");
    const cudaError_t e = set ? cudaMemcpy(M->d_p, h_params, M->n_params * 4, cudaMemcpyHostToDevice)
                              : cudaMemcpy(h_params, M->d_p, M->n_params * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_msg(TN_ECUDA, cudaGetErrorString(e));
    if (set) {
        cudaMemset(M->d_m, 0, M->n_params * 4);
        cudaMemset(M->d_v, 0, M->n_params * 4);
        M->adam_t = 0;
    }
    return TN_OK;
}

int tn_cost_model_grad(tn_cost_model_t *M, const float *h_x, const float *h_t, int32_t n, float *h_grad,
                       double *loss, void *stream) {
    if (!M || !h_x || !h_t || n < 1) return fail_msg(TN_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = ensure_batch(M, n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M->d_act[0], h_x, (size_t)n * M->dims[0] * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M->d_t, h_t, (size_t)n * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail_msg(TN_ECUDA, cudaGetErrorString(e));
    forward(M, n, s);
    backward(M, n, s);
    if (h_grad) e = cudaMemcpyAsync(h_grad, M->d_g, M->n_params * 4, cudaMemcpyDeviceToHost, s);
    double l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, M->d_loss, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_msg(TN_ECUDA, cudaGetErrorString(e));
    if (loss) *loss = l;
    return TN_OK;
}

int tn_cost_model_train(tn_cost_model_t *M, const float *h_x, const float *h_t, int64_t n, int32_t epochs,
                        int32_t batch, float lr, uint64_t seed, double *final_loss, void *stream) {
    if (!M || !h_x || !h_t || n < 1 || epochs < 1 || batch < 1) return fail_msg(TN_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int B = (int)std::min<int64_t>(batch, n);
    float *d_x = nullptr, *d_tt = nullptr;
    cudaError_t e = cudaMalloc(&d_x, (size_t)n * M->dims[0] * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_tt, (size_t)n * 4);
    if (e == cudaSuccess) e = ensure_batch(M, B);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, h_x, (size_t)n * M->dims[0] * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tt, h_t, (size_t)n * 4, cudaMemcpyHostToDevice, s);
    std::vector<int32_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    uint64_t st = seed;
    int32_t *d_order = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_order, (size_t)n * 4);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int64_t i = n - 1; i > 0; --i) std::swap(order[i], order[splitmix(st) % (uint64_t)(i + 1)]);
        e = cudaMemcpyAsync(d_order, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s);
        for (int64_t b0 = 0; b0 + B <= n && e == cudaSuccess; b0 += B) {
            gather_rows<<<dim3((M->dims[0] + 127) / 128, B), 128, 0, s>>>(d_x, d_order + b0, M->d_act[0], B, M->dims[0]);
            gather_rows<<<dim3(1, B), 128, 0, s>>>(d_tt, d_order + b0, M->d_t, B, 1);
            forward(M, B, s);
            backward(M, B, s);
            ++M->adam_t;
            const float b1 = 0.9f, b2 = 0.999f;
            const float bc1 = 1.0f - std::pow(b1, (float)M->adam_t);
            const float bc2 = 1.0f - std::pow(b2, (float)M->adam_t);
            adam_step<<<(int)std::min<int64_t>((M->n_params + 255) / 256, 1024), 256, 0, s>>>(
                M->d_p, M->d_g, M->d_m, M->d_v, M->n_params, lr, b1, b2, 1e-8f, bc1, bc2);
            e = cudaGetLastError();
        }
        // the order buffer is rewritten next epoch: finish this one first
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    double l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, M->d_loss, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_x);
    cudaFree(d_tt);
    cudaFree(d_order);
    if (e != cudaSuccess) return fail_msg(TN_ECUDA, cudaGetErrorString(e));
    if (final_loss) *final_loss = l;
    return TN_OK;
}

int tn_cost_model_predict(tn_cost_model_t *M, const float *h_x, int64_t n, float *h_y, void *stream) {
    if (!M || !h_x || !h_y || n < 0) return fail_msg(TN_EINVAL, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = 4096;
    cudaError_t e = ensure_batch(M, (int)std::min<int64_t>(std::max<int64_t>(n, 1), chunk));
    for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += chunk) {
        const int B = (int)std::min<int64_t>(chunk, n - r0);
        e = cudaMemcpyAsync(M->d_act[0], h_x + r0 * M->dims[0], (size_t)B * M->dims[0] * 4,
                            cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        forward(M, B, s);
        e = cudaMemcpyAsync(h_y + r0, M->d_act[kLayers], (size_t)B * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return fail_msg(TN_ECUDA, cudaGetErrorString(e));
    return TN_OK;
}

}  // extern "C"
