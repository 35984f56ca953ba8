// Surrogate split selector: a 4-64-64-2 multilayer perceptron trained on the
// GPU by its own forward / backward / Adam kernels (no library).
//
// The network maps a split's parameters (log2 nside, log FWHM, log l_cut,
// log theta_cut) to (log10 eps_C, log10 time): the measured power-spectrum
// error of the split convolution and its cost, so that a split meeting an error
// bound can be chosen from a candidate grid without trial runs (the paper's
// Sec. 2 scan uses the Eq. 6 estimate and the Eq. 7-8 cost models instead).
//
// Parameters live in one flat FP32 array (row-major):
//   W1 [4][64] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64][2] | b3 [2]
// with tanh after the two hidden layers.  Inputs and targets are standardised
// inside the kernels with per-feature mean / standard deviation held by the
// model.  Loss: mean over samples and both outputs of the squared error of the
// standardised targets.  One CTA of 256 threads takes a tile of 64 samples:
// forward into shared memory, backward through the same tile, per-tile weight
// gradients as small matrix products, then one atomic add per parameter.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr int kIn = 4, kH = 64, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kIn * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kOut,
              kParams = kOffB3 + kOut;  // 4610
constexpr int kTile = 64;      // samples per CTA
constexpr int kThreads = 256;

struct Norm {
    float xm[kIn], xs[kIn], ym[kOut], ys[kOut];
};

struct TileSmem {
    float p[kParams];
    float x[kTile][kIn];
    float t[kTile][kOut];
    float h1[kTile][kH];
    float h2[kTile][kH];
    float d2[kTile][kH];   // dL/dz2, then reused
    float d1[kTile][kH];   // dL/dz1
    float y[kTile][kOut];  // prediction, then dL/dy
    float red[kThreads / 32];
};

// Forward pass of one tile into shared memory (rows beyond n are zero inputs).
__device__ void tile_forward(TileSmem &S, const Norm &nm, const float *__restrict__ X,
                             const float *__restrict__ T, int s0, int n) {
    const int tid = threadIdx.x;
    for (int i = tid; i < kTile * kIn; i += kThreads) {
        const int s = i / kIn, f = i % kIn;
        const int g = s0 + s;
        S.x[s][f] = g < n ? (X[(size_t)g * kIn + f] - nm.xm[f]) / nm.xs[f] : 0.0f;
    }
    if (T) {
        for (int i = tid; i < kTile * kOut; i += kThreads) {
            const int s = i / kOut, o = i % kOut;
            const int g = s0 + s;
            S.t[s][o] = g < n ? (T[(size_t)g * kOut + o] - nm.ym[o]) / nm.ys[o] : 0.0f;
        }
    }
    __syncthreads();
    for (int i = tid; i < kTile * kH; i += kThreads) {
        const int s = i / kH, u = i % kH;
        float z = S.p[kOffB1 + u];
#pragma unroll
        for (int f = 0; f < kIn; ++f) z = fmaf(S.x[s][f], S.p[kOffW1 + f * kH + u], z);
        S.h1[s][u] = tanhf(z);
    }
    __syncthreads();
    for (int i = tid; i < kTile * kH; i += kThreads) {
        const int s = i / kH, v = i % kH;
        float z = S.p[kOffB2 + v];
        for (int u = 0; u < kH; ++u) z = fmaf(S.h1[s][u], S.p[kOffW2 + u * kH + v], z);
        S.h2[s][v] = tanhf(z);
    }
    __syncthreads();
    for (int i = tid; i < kTile * kOut; i += kThreads) {
        const int s = i / kOut, o = i % kOut;
        float z = S.p[kOffB3 + o];
        for (int v = 0; v < kH; ++v) z = fmaf(S.h2[s][v], S.p[kOffW3 + v * kOut + o], z);
        S.y[s][o] = z;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
mlp_predict_kernel(const float *__restrict__ params, Norm nm, const float *__restrict__ X, int n,
                   float *__restrict__ Y) {
    extern __shared__ __align__(16) unsigned char raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(raw);
    for (int i = threadIdx.x; i < kParams; i += kThreads) S.p[i] = params[i];
    __syncthreads();
    const int s0 = blockIdx.x * kTile;
    tile_forward(S, nm, X, nullptr, s0, n);
    for (int i = threadIdx.x; i < kTile * kOut; i += kThreads) {
        const int s = i / kOut, o = i % kOut;
        if (s0 + s < n) Y[(size_t)(s0 + s) * kOut + o] = S.y[s][o] * nm.ys[o] + nm.ym[o];
    }
}

// Forward + backward of one tile; adds the tile's gradient (of the mean loss
// over all n samples) into grad[kParams] and its loss share into *loss.
__global__ void __launch_bounds__(kThreads)
mlp_grad_kernel(const float *__restrict__ params, Norm nm, const float *__restrict__ X,
                const float *__restrict__ T, int n, float *__restrict__ grad,
                float *__restrict__ loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < kParams; i += kThreads) S.p[i] = params[i];
    __syncthreads();
    const int s0 = blockIdx.x * kTile;
    tile_forward(S, nm, X, T, s0, n);
    const float scale = 2.0f / ((float)n * (float)kOut);  // d(mean sq err)/dy
    // dL/dy and the loss
    float lsum = 0.0f;
    for (int i = tid; i < kTile * kOut; i += kThreads) {
        const int s = i / kOut, o = i % kOut;
        const bool in = s0 + s < n;
        const float e = in ? S.y[s][o] - S.t[s][o] : 0.0f;
        lsum += e * e;
        S.y[s][o] = scale * e;
    }
    __syncthreads();
    // dL/dz2 = (dL/dy W3^T) (1 - h2^2)
    for (int i = tid; i < kTile * kH; i += kThreads) {
        const int s = i / kH, v = i % kH;
        float g = 0.0f;
#pragma unroll
        for (int o = 0; o < kOut; ++o) g = fmaf(S.y[s][o], S.p[kOffW3 + v * kOut + o], g);
        const float h = S.h2[s][v];
        S.d2[s][v] = g * (1.0f - h * h);
    }
    __syncthreads();
    // dL/dz1 = (dL/dz2 W2^T) (1 - h1^2)
    for (int i = tid; i < kTile * kH; i += kThreads) {
        const int s = i / kH, u = i % kH;
        float g = 0.0f;
        for (int v = 0; v < kH; ++v) g = fmaf(S.d2[s][v], S.p[kOffW2 + u * kH + v], g);
        const float h = S.h1[s][u];
        S.d1[s][u] = g * (1.0f - h * h);
    }
    __syncthreads();
    // parameter gradients of the tile: sums over its samples
    for (int i = tid; i < kParams; i += kThreads) {
        float g = 0.0f;
        if (i < kOffB1) {                 // W1[f][u] = sum_s x[s][f] d1[s][u]
            const int f = i / kH, u = i % kH;
            for (int s = 0; s < kTile; ++s) g = fmaf(S.x[s][f], S.d1[s][u], g);
        } else if (i < kOffW2) {          // b1[u]
            const int u = i - kOffB1;
            for (int s = 0; s < kTile; ++s) g += S.d1[s][u];
        } else if (i < kOffB2) {          // W2[u][v] = sum_s h1[s][u] d2[s][v]
            const int k = i - kOffW2, u = k / kH, v = k % kH;
            for (int s = 0; s < kTile; ++s) g = fmaf(S.h1[s][u], S.d2[s][v], g);
        } else if (i < kOffW3) {          // b2[v]
            const int v = i - kOffB2;
            for (int s = 0; s < kTile; ++s) g += S.d2[s][v];
        } else if (i < kOffB3) {          // W3[v][o] = sum_s h2[s][v] dy[s][o]
            const int k = i - kOffW3, v = k / kOut, o = k % kOut;
            for (int s = 0; s < kTile; ++s) g = fmaf(S.h2[s][v], S.y[s][o], g);
        } else {                          // b3[o]
            const int o = i - kOffB3;
            for (int s = 0; s < kTile; ++s) g += S.y[s][o];
        }
        atomicAdd(&grad[i], g);
    }
    // loss: warp shuffles, then one atomic per CTA
    for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    if ((tid & 31) == 0) S.red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) t += S.red[w];
        atomicAdd(loss, t / ((float)n * (float)kOut));
    }
}

// Adam (Kingma & Ba 2015) with bias correction; *step counts the updates
// already made (advanced afterwards by mlp_step_kernel, so every block of this
// launch reads the same value).
__global__ void mlp_adam_kernel(float *__restrict__ params, const float *__restrict__ grad,
                                float *__restrict__ m1, float *__restrict__ m2,
                                const int *__restrict__ step, float lr, float beta1, float beta2,
                                float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = *step + 1;
    if (i < kParams) {
        const float g = grad[i];
        const float a = beta1 * m1[i] + (1.0f - beta1) * g;
        const float b = beta2 * m2[i] + (1.0f - beta2) * g * g;
        m1[i] = a;
        m2[i] = b;
        const float ah = a / (1.0f - powf(beta1, (float)t));
        const float bh = b / (1.0f - powf(beta2, (float)t));
        params[i] -= lr * ah / (sqrtf(bh) + eps);
    }
}

__global__ void mlp_step_kernel(int *step) { *step += 1; }

} // namespace
} // namespace ksc

// ---------------------------------------------------------------------------
// Model object and C ABI.
// ---------------------------------------------------------------------------
struct ksc_mlp {
    ksc::Norm norm{};
    float *d_params = nullptr;  // kParams
    float *d_grad = nullptr;    // kParams + 1 (loss last)
    float *d_m1 = nullptr, *d_m2 = nullptr;
    int *d_step = nullptr;
};

namespace {

int mfail(int code, const std::string &msg) {
    ksc::set_last_error(msg);
    return code;
}

int mcuda(cudaError_t e, const char *what) {
    return mfail(KSC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// splitmix64 (Steele, Lea & Flood 2014): the counter-based generator behind the
// initial weights, so a seed fixes them on any machine.
unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

size_t tile_smem() { return sizeof(ksc::TileSmem); }

void mlp_free(ksc_mlp *m) {
    if (!m) return;
    cudaFree(m->d_params);
    cudaFree(m->d_grad);
    cudaFree(m->d_m1);
    cudaFree(m->d_m2);
    cudaFree(m->d_step);
    delete m;
}

cudaError_t set_smem_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(ksc::mlp_grad_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tile_smem());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ksc::mlp_predict_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem());
    done = e == cudaSuccess;
    return e;
}

} // namespace

extern "C" {

int ksc_mlp_n_params(void) { return ksc::kParams; }

int ksc_mlp_create(unsigned long long seed, ksc_mlp **out) {
    if (!out) return mfail(KSC_ERR_ARG, "null output pointer");
    *out = nullptr;
    ksc_mlp *m = new (std::nothrow) ksc_mlp();
    if (!m) return mfail(KSC_ERR_NOMEM, "host allocation");
    for (int f = 0; f < ksc::kIn; ++f) { m->norm.xm[f] = 0.0f; m->norm.xs[f] = 1.0f; }
    for (int o = 0; o < ksc::kOut; ++o) { m->norm.ym[o] = 0.0f; m->norm.ys[o] = 1.0f; }
    // Glorot-uniform weights, zero biases
    std::vector<float> p(ksc::kParams, 0.0f);
    unsigned long long ctr = seed * 0x100000001B3ull;
    auto uni = [&]() {  // uniform in [-1, 1)
        const unsigned long long r = splitmix64(ctr++);
        return (float)((double)(r >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    };
    auto fill = [&](int off, int fan_in, int fan_out) {
        const float a = std::sqrt(6.0f / (float)(fan_in + fan_out));
        for (int i = 0; i < fan_in * fan_out; ++i) p[off + i] = a * uni();
    };
    fill(ksc::kOffW1, ksc::kIn, ksc::kH);
    fill(ksc::kOffW2, ksc::kH, ksc::kH);
    fill(ksc::kOffW3, ksc::kH, ksc::kOut);
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_params, sizeof(float) * ksc::kParams)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_grad, sizeof(float) * (ksc::kParams + 1))) != cudaSuccess ||
        (e = cudaMalloc(&m->d_m1, sizeof(float) * ksc::kParams)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_m2, sizeof(float) * ksc::kParams)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_step, sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(m->d_params, p.data(), sizeof(float) * ksc::kParams,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(m->d_m1, 0, sizeof(float) * ksc::kParams)) != cudaSuccess ||
        (e = cudaMemset(m->d_m2, 0, sizeof(float) * ksc::kParams)) != cudaSuccess ||
        (e = cudaMemset(m->d_step, 0, sizeof(int))) != cudaSuccess) {
        mlp_free(m);
        return mcuda(e, "surrogate device state");
    }
    *out = m;
    return KSC_OK;
}

int ksc_mlp_set_norm(ksc_mlp *m, const float *x_mean, const float *x_std, const float *y_mean,
                     const float *y_std) {
    if (!m || !x_mean || !x_std || !y_mean || !y_std) return mfail(KSC_ERR_ARG, "null argument");
    for (int f = 0; f < ksc::kIn; ++f) {
        if (!(x_std[f] > 0.0f)) return mfail(KSC_ERR_ARG, "standard deviations must be > 0");
        m->norm.xm[f] = x_mean[f];
        m->norm.xs[f] = x_std[f];
    }
    for (int o = 0; o < ksc::kOut; ++o) {
        if (!(y_std[o] > 0.0f)) return mfail(KSC_ERR_ARG, "standard deviations must be > 0");
        m->norm.ym[o] = y_mean[o];
        m->norm.ys[o] = y_std[o];
    }
    return KSC_OK;
}

int ksc_mlp_get_params(const ksc_mlp *m, float *h_params) {
    if (!m || !h_params) return mfail(KSC_ERR_ARG, "null argument");
    cudaError_t e = cudaMemcpy(h_params, m->d_params, sizeof(float) * ksc::kParams,
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? KSC_OK : mcuda(e, "parameter download");
}

int ksc_mlp_set_params(ksc_mlp *m, const float *h_params) {
    if (!m || !h_params) return mfail(KSC_ERR_ARG, "null argument");
    cudaError_t e = cudaMemcpy(m->d_params, h_params, sizeof(float) * ksc::kParams,
                               cudaMemcpyHostToDevice);
    return e == cudaSuccess ? KSC_OK : mcuda(e, "parameter upload");
}

int ksc_mlp_predict(const ksc_mlp *m, const float *d_x, int n, float *d_y, void *stream) {
    if (!m || !d_x || !d_y || n < 0) return mfail(KSC_ERR_ARG, "bad argument");
    if (n == 0) return KSC_OK;
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return mcuda(e, "surrogate kernel attribute");
    const int blocks = (n + ksc::kTile - 1) / ksc::kTile;
    ksc::mlp_predict_kernel<<<blocks, ksc::kThreads, tile_smem(), (cudaStream_t)stream>>>(
        m->d_params, m->norm, d_x, n, d_y);
    e = cudaGetLastError();
    return e == cudaSuccess ? KSC_OK : mcuda(e, "surrogate predict launch");
}

int ksc_mlp_grad(const ksc_mlp *m, const float *d_x, const float *d_t, int n, float *h_grad,
                 float *h_loss) {
    if (!m || !d_x || !d_t || !h_grad || n < 1) return mfail(KSC_ERR_ARG, "bad argument");
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return mcuda(e, "surrogate kernel attribute");
    if ((e = cudaMemset(m->d_grad, 0, sizeof(float) * (ksc::kParams + 1))) != cudaSuccess)
        return mcuda(e, "gradient reset");
    const int blocks = (n + ksc::kTile - 1) / ksc::kTile;
    ksc::mlp_grad_kernel<<<blocks, ksc::kThreads, tile_smem()>>>(m->d_params, m->norm, d_x, d_t, n,
                                                                m->d_grad,
                                                                m->d_grad + ksc::kParams);
    if ((e = cudaGetLastError()) != cudaSuccess) return mcuda(e, "surrogate gradient launch");
    if ((e = cudaMemcpy(h_grad, m->d_grad, sizeof(float) * ksc::kParams,
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
        return mcuda(e, "gradient download");
    if (h_loss &&
        (e = cudaMemcpy(h_loss, m->d_grad + ksc::kParams, sizeof(float), cudaMemcpyDeviceToHost)) !=
            cudaSuccess)
        return mcuda(e, "loss download");
    return KSC_OK;
}

int ksc_mlp_train(ksc_mlp *m, const float *d_x, const float *d_t, int n, int epochs, float lr,
                  void *stream, float *h_loss) {
    if (!m || !d_x || !d_t || n < 1 || epochs < 0 || !(lr > 0.0f))
        return mfail(KSC_ERR_ARG, "bad argument");
    cudaError_t e = set_smem_attr();
    if (e != cudaSuccess) return mcuda(e, "surrogate kernel attribute");
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (n + ksc::kTile - 1) / ksc::kTile;
    // one epoch (full-batch gradient, one Adam step) captured once as a CUDA graph
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return mcuda(e, "capture stream");
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(m->d_grad, 0, sizeof(float) * (ksc::kParams + 1), cs);
        ksc::mlp_grad_kernel<<<blocks, ksc::kThreads, tile_smem(), cs>>>(
            m->d_params, m->norm, d_x, d_t, n, m->d_grad, m->d_grad + ksc::kParams);
        ksc::mlp_adam_kernel<<<(ksc::kParams + 255) / 256, 256, 0, cs>>>(
            m->d_params, m->d_grad, m->d_m1, m->d_m2, m->d_step, lr, 0.9f, 0.999f, 1e-8f);
        ksc::mlp_step_kernel<<<1, 1, 0, cs>>>(m->d_step);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    for (int ep = 0; e == cudaSuccess && ep < epochs; ++ep) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess && h_loss) {
        // loss of the last epoch's parameters before its update
        e = cudaMemcpyAsync(h_loss, m->d_grad + ksc::kParams, sizeof(float),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return e == cudaSuccess ? KSC_OK : mcuda(e, "surrogate training");
}

int ksc_mlp_select(const ksc_mlp *m, const float *h_x, int n, double log10_bound, double margin,
                   const double *h_host_ms, int *best, float *h_pred) {
    if (!m || !h_x || !best || n < 1) return mfail(KSC_ERR_ARG, "bad argument");
    *best = -1;
    float *d_x = nullptr, *d_y = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_x, sizeof(float) * (size_t)ksc::kIn * (size_t)n)) != cudaSuccess)
        return mfail(KSC_ERR_NOMEM, "candidate buffer");
    if ((e = cudaMalloc(&d_y, sizeof(float) * 2 * (size_t)n)) != cudaSuccess) {
        cudaFree(d_x);
        return mfail(KSC_ERR_NOMEM, "prediction buffer");
    }
    std::vector<float> y(2 * (size_t)n);
    int rc = KSC_OK;
    e = cudaMemcpy(d_x, h_x, sizeof(float) * (size_t)ksc::kIn * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        rc = ksc_mlp_predict(m, d_x, n, d_y, nullptr);
        if (rc == KSC_OK)
            e = cudaMemcpy(y.data(), d_y, sizeof(float) * y.size(), cudaMemcpyDeviceToHost);
    }
    cudaFree(d_x);
    cudaFree(d_y);
    if (rc) return rc;
    if (e != cudaSuccess) return mcuda(e, "surrogate select");
    // The two halves run concurrently (Fig. 1): a candidate costs the larger of
    // its predicted GPU time and its host (harmonic) time.  Cheapest candidate
    // whose predicted error clears the bound by `margin` decades.
    double best_cost = 0.0;
    for (int i = 0; i < n; ++i) {
        if (y[2 * (size_t)i] > (float)(log10_bound - margin)) continue;
        double c = std::pow(10.0, (double)y[2 * (size_t)i + 1]);
        if (h_host_ms && h_host_ms[i] > c) c = h_host_ms[i];
        if (*best < 0 || c < best_cost) {
            *best = i;
            best_cost = c;
        }
    }
    if (h_pred) std::memcpy(h_pred, y.data(), sizeof(float) * y.size());
    return KSC_OK;
}

void ksc_mlp_free(ksc_mlp *m) { mlp_free(m); }

} // extern "C"
