// Schedule cost model: a small MLP (16 -> 64 -> 64 -> 1, ReLU) that predicts
// log2 of an out-of-core call's time from features of the problem and of a
// candidate plan.  Forward, backward (mean squared error) and Adam update are
// hand-written kernels; the planner evaluates all its candidates with one
// forward launch and keeps the one with the smallest prediction.
//
// Parameters are one FP32 vector, packed W1[64][16], b1[64], W2[64][64],
// b2[64], W3[64], b3 (5313 values).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ooc_internal.hpp"

namespace ooc {

namespace {

constexpr int IN = kMlpIn, H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == kMlpParams, "parameter packing");
constexpr int SB = 32;  // samples per block

// Forward pass of SB samples held in shared memory; fills z1/z2 (pre-activations) and y.
__device__ void forward_tile(const float* __restrict__ P, const float (*x)[IN], float (*z1)[H], float (*z2)[H],
                             float* y, int ns)
{
    const int j = threadIdx.x;  // 64 threads: one hidden unit each
    for (int s = 0; s < ns; ++s) {
        float a = P[OFF_B1 + j];
        for (int i = 0; i < IN; ++i) a = fmaf(x[s][i], P[OFF_W1 + j * IN + i], a);
        z1[s][j] = a;
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
        float a = P[OFF_B2 + j];
        for (int k = 0; k < H; ++k) a = fmaf(fmaxf(z1[s][k], 0.f), P[OFF_W2 + j * H + k], a);
        z2[s][j] = a;
    }
    __syncthreads();
    if (j < ns) {
        float a = P[OFF_B3];
        for (int k = 0; k < H; ++k) a = fmaf(fmaxf(z2[j][k], 0.f), P[OFF_W3 + k], a);
        y[j] = a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(H) mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                        int64_t n, float* __restrict__ Y)
{
    __shared__ float x[SB][IN], z1[SB][H], z2[SB][H], y[SB];
    const int64_t s0 = (int64_t)blockIdx.x * SB;
    const int ns = (int)(n - s0 < (int64_t)SB ? n - s0 : (int64_t)SB);
    for (int e = threadIdx.x; e < ns * IN; e += H) x[e / IN][e % IN] = X[(s0 + e / IN) * IN + e % IN];
    __syncthreads();
    forward_tile(P, x, z1, z2, y, ns);
    if (threadIdx.x < ns) Y[s0 + threadIdx.x] = y[threadIdx.x];
}

// Gradient of L = (1/n_total) * sum 0.5 (y - t)^2 for SB samples, added into G.
__global__ void __launch_bounds__(H) mlp_backward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                         const float* __restrict__ T, int64_t n, float inv_n,
                                                         float* __restrict__ G, float* __restrict__ loss)
{
    __shared__ float x[SB][IN], z1[SB][H], z2[SB][H], y[SB], dy[SB], d2[SB][H], d1[SB][H];
    const int64_t s0 = (int64_t)blockIdx.x * SB;
    const int ns = (int)(n - s0 < (int64_t)SB ? n - s0 : (int64_t)SB);
    const int j = threadIdx.x;
    for (int e = j; e < ns * IN; e += H) x[e / IN][e % IN] = X[(s0 + e / IN) * IN + e % IN];
    __syncthreads();
    forward_tile(P, x, z1, z2, y, ns);
    if (j < ns) {
        const float r = y[j] - T[s0 + j];
        dy[j] = r * inv_n;
        atomicAdd(loss, 0.5f * r * r * inv_n);
    }
    __syncthreads();
    // output layer
    {
        float gw = 0.f;
        for (int s = 0; s < ns; ++s) gw = fmaf(dy[s], fmaxf(z2[s][j], 0.f), gw);
        atomicAdd(&G[OFF_W3 + j], gw);
        if (j == 0) {
            float gb = 0.f;
            for (int s = 0; s < ns; ++s) gb += dy[s];
            atomicAdd(&G[OFF_B3], gb);
        }
        for (int s = 0; s < ns; ++s) d2[s][j] = z2[s][j] > 0.f ? dy[s] * P[OFF_W3 + j] : 0.f;
    }
    __syncthreads();
    // second hidden layer: row j of W2
    {
        float gb = 0.f;
        for (int s = 0; s < ns; ++s) gb += d2[s][j];
        atomicAdd(&G[OFF_B2 + j], gb);
        for (int k = 0; k < H; ++k) {
            float gw = 0.f;
            for (int s = 0; s < ns; ++s) gw = fmaf(d2[s][j], fmaxf(z1[s][k], 0.f), gw);
            atomicAdd(&G[OFF_W2 + j * H + k], gw);
        }
        // d1[s][j] = relu'(z1[s][j]) * sum_k d2[s][k] W2[k][j]
        for (int s = 0; s < ns; ++s) {
            float a = 0.f;
            for (int k = 0; k < H; ++k) a = fmaf(d2[s][k], P[OFF_W2 + k * H + j], a);
            d1[s][j] = z1[s][j] > 0.f ? a : 0.f;
        }
    }
    __syncthreads();
    // first hidden layer: row j of W1
    {
        float gb = 0.f;
        for (int s = 0; s < ns; ++s) gb += d1[s][j];
        atomicAdd(&G[OFF_B1 + j], gb);
        for (int i = 0; i < IN; ++i) {
            float gw = 0.f;
            for (int s = 0; s < ns; ++s) gw = fmaf(d1[s][j], x[s][i], gw);
            atomicAdd(&G[OFF_W1 + j * IN + i], gw);
        }
    }
}

// Adam (Kingma & Ba) on g = gradient + wd * p (L2 weight decay):
// m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                            float* __restrict__ v, int np, float lr, float wd, float b1, float b2, float c1, float c2,
                            float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float g = G[i] + wd * P[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// device buffers reused across calls (grown as needed); guarded by g_mu
std::mutex g_mu;
struct DevBufs {
    float *P = nullptr, *X = nullptr, *Y = nullptr, *G = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    int64_t cap = 0;
} g_buf;

int ensure_bufs(int64_t n, std::string& why)
{
    if (!g_buf.P) {
        if (cudaMalloc(&g_buf.P, kMlpParams * 4) || cudaMalloc(&g_buf.G, kMlpParams * 4) ||
            cudaMalloc(&g_buf.m, kMlpParams * 4) || cudaMalloc(&g_buf.v, kMlpParams * 4) ||
            cudaMalloc(&g_buf.loss, 4)) {
            cudaGetLastError();
            why = "cost-model parameter buffers";
            return OOC_ERR_ALLOC;
        }
    }
    if (n > g_buf.cap) {
        if (g_buf.X) cudaFree(g_buf.X);
        if (g_buf.Y) cudaFree(g_buf.Y);
        g_buf.X = g_buf.Y = nullptr;
        const int64_t cap = std::max<int64_t>(n, 1024);
        if (cudaMalloc(&g_buf.X, cap * IN * 4) || cudaMalloc(&g_buf.Y, cap * 4)) {
            cudaGetLastError();
            g_buf.cap = 0;
            why = "cost-model sample buffers";
            return OOC_ERR_ALLOC;
        }
        g_buf.cap = cap;
    }
    return OOC_OK;
}

}  // namespace

int mlp_forward_host(const float* params, const float* X, int64_t n, float* y, std::string& why)
{
    if (n <= 0) return OOC_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_bufs(n, why);
    if (rc) return rc;
    if (cudaMemcpy(g_buf.P, params, kMlpParams * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(g_buf.X, X, n * IN * 4, cudaMemcpyHostToDevice)) {
        why = "cost-model upload";
        return OOC_ERR_CUDA;
    }
    mlp_forward_kernel<<<(unsigned)((n + SB - 1) / SB), H>>>(g_buf.P, g_buf.X, n, g_buf.Y);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(y, g_buf.Y, n * 4, cudaMemcpyDeviceToHost)) {
        why = "cost-model forward";
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

int mlp_loss_grad_host(const float* params, const float* X, const float* t, int64_t n, float* grad, float* loss,
                       std::string& why)
{
    if (n <= 0) { why = "no samples"; return OOC_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_bufs(n, why);
    if (rc) return rc;
    if (cudaMemcpy(g_buf.P, params, kMlpParams * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(g_buf.X, X, n * IN * 4, cudaMemcpyHostToDevice) ||
        cudaMemcpy(g_buf.Y, t, n * 4, cudaMemcpyHostToDevice) || cudaMemset(g_buf.G, 0, kMlpParams * 4) ||
        cudaMemset(g_buf.loss, 0, 4)) {
        why = "cost-model upload";
        return OOC_ERR_CUDA;
    }
    mlp_backward_kernel<<<(unsigned)((n + SB - 1) / SB), H>>>(g_buf.P, g_buf.X, g_buf.Y, n, 1.f / (float)n, g_buf.G,
                                                             g_buf.loss);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(grad, g_buf.G, kMlpParams * 4, cudaMemcpyDeviceToHost) ||
        cudaMemcpy(loss, g_buf.loss, 4, cudaMemcpyDeviceToHost)) {
        why = "cost-model backward";
        return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

int mlp_train_host(float* params, const float* X, const float* t, int64_t n, int epochs, int batch, float lr,
                   float wd, uint64_t seed, float* final_loss, std::string& why)
{
    if (n <= 0 || epochs < 0 || batch <= 0) { why = "bad training arguments"; return OOC_ERR_INVALID_ARG; }
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_bufs(n, why);
    if (rc) return rc;
    // per-epoch shuffles of the samples (host permutation, xorshift64*), uploaded once
    std::vector<float> xs((size_t)n * IN), ts((size_t)n);
    std::vector<int64_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = i;
    uint64_t st = seed ? seed : 0x9E3779B97F4A7C15ull;
    auto rnd = [&st]() {
        st ^= st >> 12; st ^= st << 25; st ^= st >> 27;
        return st * 0x2545F4914F6CDD1Dull;
    };
    if (cudaMemcpy(g_buf.P, params, kMlpParams * 4, cudaMemcpyHostToDevice) || cudaMemset(g_buf.m, 0, kMlpParams * 4) ||
        cudaMemset(g_buf.v, 0, kMlpParams * 4)) {
        why = "cost-model upload";
        return OOC_ERR_CUDA;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    int64_t step = 0;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t i = n - 1; i > 0; --i) std::swap(perm[(size_t)i], perm[(size_t)(rnd() % (uint64_t)(i + 1))]);
        for (int64_t i = 0; i < n; ++i) {
            std::memcpy(&xs[(size_t)i * IN], &X[(size_t)perm[(size_t)i] * IN], IN * 4);
            ts[(size_t)i] = t[(size_t)perm[(size_t)i]];
        }
        if (cudaMemcpy(g_buf.X, xs.data(), n * IN * 4, cudaMemcpyHostToDevice) ||
            cudaMemcpy(g_buf.Y, ts.data(), n * 4, cudaMemcpyHostToDevice)) {
            why = "cost-model upload";
            return OOC_ERR_CUDA;
        }
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t nb = std::min<int64_t>(batch, n - b0);
            cudaMemsetAsync(g_buf.G, 0, kMlpParams * 4);
            cudaMemsetAsync(g_buf.loss, 0, 4);
            mlp_backward_kernel<<<(unsigned)((nb + SB - 1) / SB), H>>>(g_buf.P, g_buf.X + b0 * IN, g_buf.Y + b0, nb,
                                                                      1.f / (float)nb, g_buf.G, g_buf.loss);
            ++step;
            const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
            adam_kernel<<<(kMlpParams + 255) / 256, 256>>>(g_buf.P, g_buf.G, g_buf.m, g_buf.v, kMlpParams, lr, wd, b1,
                                                           b2, c1, c2, eps);
        }
    }
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(params, g_buf.P, kMlpParams * 4, cudaMemcpyDeviceToHost)) {
        why = "cost-model training";
        return OOC_ERR_CUDA;
    }
    if (final_loss) {
        // loss of the trained parameters over all samples
        if (cudaMemset(g_buf.G, 0, kMlpParams * 4) || cudaMemset(g_buf.loss, 0, 4)) return OOC_ERR_CUDA;
        mlp_backward_kernel<<<(unsigned)((n + SB - 1) / SB), H>>>(g_buf.P, g_buf.X, g_buf.Y, n, 1.f / (float)n, g_buf.G,
                                                                 g_buf.loss);
        if (cudaMemcpy(final_loss, g_buf.loss, 4, cudaMemcpyDeviceToHost)) return OOC_ERR_CUDA;
    }
    return OOC_OK;
}

}  // namespace ooc
