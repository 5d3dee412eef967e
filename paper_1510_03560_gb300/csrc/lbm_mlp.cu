// The activation proposer's network (include/lbm.h, lbm_mlp_*): a
// multilayer perceptron 34 -> 64 -> 64 -> 1 with ReLU hidden layers and a
// logistic output, its forward pass (FP32, or bfloat16 operands with FP32
// accumulation), the backward pass of the binary cross-entropy and Adam.
// One thread per sample for the per-sample passes, the weights staged in
// shared memory; one thread per parameter for the weight gradients, each
// summing over the samples in order, so that training is reproducible.
#include <cmath>
#include <cstdio>
#include <new>

#include <cuda_bf16.h>

#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int NI = LBM_MLP_IN;
constexpr int NH = LBM_MLP_HIDDEN;
constexpr int NP = LBM_MLP_NPARAM;
// parameter offsets
constexpr int OW1 = 0, OB1 = OW1 + NI * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH;
static_assert(OB3 + 1 == NP, "parameter packing");
constexpr int FWD_THREADS = 128;

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Forward pass, one thread per sample.  With `train`, the standardised
// inputs and hidden activations are kept for the backward pass and
// dz = (p - y) / n and the per-sample loss are written.
// The sample count is n, or *ndev when ndev is given (at most n).
template <bool BF16, bool TRAIN>
__global__ void __launch_bounds__(FWD_THREADS) k_fwd(const float *P, const float *mean, const float *scale,
                                                     const float *x, int n, const int *ndev, float *prob,
                                                     const float *y, float *Xn, float *H1, float *H2,
                                                     float *dz, double *lossv)
{
    __shared__ float w[NP];
    if (ndev) n = min(n, *ndev);
    if ((int)(blockIdx.x * blockDim.x) >= n) return;
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = BF16 ? bf16_round(P[i]) : P[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float xn[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const float v = (x[(size_t)s * NI + i] - mean[i]) * scale[i];
        xn[i] = BF16 ? bf16_round(v) : v;
        if (TRAIN) Xn[(size_t)s * NI + i] = xn[i];
    }
    float h1[NH];
#pragma unroll 4
    for (int k = 0; k < NH; ++k) {
        float acc = w[OB1 + k];
#pragma unroll
        for (int i = 0; i < NI; ++i) acc = fmaf(xn[i], w[OW1 + i * NH + k], acc);
        acc = fmaxf(acc, 0.f);
        h1[k] = BF16 ? bf16_round(acc) : acc;
        if (TRAIN) H1[(size_t)s * NH + k] = h1[k];
    }
    float z = w[OB3];
#pragma unroll 2
    for (int j = 0; j < NH; ++j) {
        float acc = w[OB2 + j];
#pragma unroll
        for (int k = 0; k < NH; ++k) acc = fmaf(h1[k], w[OW2 + k * NH + j], acc);
        acc = fmaxf(acc, 0.f);
        const float h2 = BF16 ? bf16_round(acc) : acc;
        if (TRAIN) H2[(size_t)s * NH + j] = h2;
        z = fmaf(h2, w[OW3 + j], z);
    }
    const float p = 1.f / (1.f + expf(-z));
    if (prob) prob[s] = p;
    if (TRAIN) {
        const float t = y[s];
        dz[s] = (p - t) / (float)n;
        // binary cross-entropy of the logit, in the stable form
        lossv[s] = (double)fmaxf(z, 0.f) - (double)z * (double)t + log1p(exp(-fabs((double)z)));
    }
}

// Backward pass through the hidden layers, one thread per sample.
__global__ void __launch_bounds__(FWD_THREADS) k_bwd(const float *P, int n, const float *dz,
                                                     const float *H1, const float *H2, float *dH1,
                                                     float *dH2)
{
    __shared__ float w2[NH * NH];
    __shared__ float w3[NH];
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) w2[i] = P[OW2 + i];
    for (int i = threadIdx.x; i < NH; i += blockDim.x) w3[i] = P[OW3 + i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float g2[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) {
        g2[j] = H2[(size_t)s * NH + j] > 0.f ? dz[s] * w3[j] : 0.f;
        dH2[(size_t)s * NH + j] = g2[j];
    }
#pragma unroll 4
    for (int k = 0; k < NH; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < NH; ++j) acc = fmaf(g2[j], w2[k * NH + j], acc);
        dH1[(size_t)s * NH + k] = H1[(size_t)s * NH + k] > 0.f ? acc : 0.f;
    }
}

// Weight gradients, one thread per parameter, each a sum over the samples
// in order.
__global__ void __launch_bounds__(256) k_wgrad(int n, const float *Xn, const float *H1, const float *H2,
                                               const float *dH1, const float *dH2, const float *dz,
                                               float *G)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    float acc = 0.f;
    if (p < OB1) {
        const int i = p / NH, k = p % NH;
        for (int s = 0; s < n; ++s) acc = fmaf(Xn[(size_t)s * NI + i], dH1[(size_t)s * NH + k], acc);
    } else if (p < OW2) {
        const int k = p - OB1;
        for (int s = 0; s < n; ++s) acc += dH1[(size_t)s * NH + k];
    } else if (p < OB2) {
        const int k = (p - OW2) / NH, j = (p - OW2) % NH;
        for (int s = 0; s < n; ++s) acc = fmaf(H1[(size_t)s * NH + k], dH2[(size_t)s * NH + j], acc);
    } else if (p < OW3) {
        const int j = p - OB2;
        for (int s = 0; s < n; ++s) acc += dH2[(size_t)s * NH + j];
    } else if (p < OB3) {
        const int j = p - OW3;
        for (int s = 0; s < n; ++s) acc = fmaf(H2[(size_t)s * NH + j], dz[s], acc);
    } else {
        for (int s = 0; s < n; ++s) acc += dz[s];
    }
    G[p] = acc;
}

// Mean of the per-sample losses, fixed order.
__global__ void __launch_bounds__(1024) k_loss_mean(const double *lossv, int n, double *out)
{
    __shared__ double red[1024];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) acc += lossv[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (double)(n > 0 ? n : 1);
}

__global__ void k_adam(float *P, const float *G, float *M, float *V, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float g = G[p];
    const float m = b1 * M[p] + (1.f - b1) * g;
    const float v = b2 * V[p] + (1.f - b2) * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_mlp {
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr, *mean = nullptr, *scale = nullptr;
    float *Xn = nullptr, *H1 = nullptr, *H2 = nullptr, *dH1 = nullptr, *dH2 = nullptr, *dz = nullptr;
    double *lossv = nullptr, *loss = nullptr;
};

namespace {

int mlp_fail(int code, const char *what, cudaError_t e = cudaSuccess)
{
    char msg[256];
    snprintf(msg, sizeof msg, "lbm_mlp: %s%s%s", what, e == cudaSuccess ? "" : ": ",
             e == cudaSuccess ? "" : cudaGetErrorString(e));
    set_global_error(msg);
    return code;
}

void mlp_free(lbm_mlp *m)
{
    void *ptrs[] = {m->P, m->G, m->M, m->V, m->mean, m->scale, m->Xn, m->H1,
                    m->H2, m->dH1, m->dH2, m->dz, m->lossv, m->loss};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

}  // namespace

cudaError_t lbm::mlp_forward_on(const lbm_mlp *m, const float *x, int n, const int *ndev, int bf16,
                                float *prob, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (n + FWD_THREADS - 1) / FWD_THREADS;
    if (bf16)
        k_fwd<true, false><<<grid, FWD_THREADS, 0, s>>>(m->P, m->mean, m->scale, x, n, ndev, prob, nullptr,
                                                        nullptr, nullptr, nullptr, nullptr, nullptr);
    else
        k_fwd<false, false><<<grid, FWD_THREADS, 0, s>>>(m->P, m->mean, m->scale, x, n, ndev, prob, nullptr,
                                                         nullptr, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

extern "C" {

int lbm_mlp_create(int max_batch, void *stream, lbm_mlp **out)
{
    if (!out) return mlp_fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_batch < 1) return mlp_fail(LBM_EINVAL, "max_batch must be >= 1");
    lbm_mlp *m = new (std::nothrow) lbm_mlp();
    if (!m) return mlp_fail(LBM_ENOMEM, "host allocation failed");
    m->max_batch = max_batch;
    m->stream = (cudaStream_t)stream;
    const size_t B = (size_t)max_batch;
    struct {
        void **dst;
        size_t bytes;
    } want[] = {
        {(void **)&m->P, NP * sizeof(float)},        {(void **)&m->G, NP * sizeof(float)},
        {(void **)&m->M, NP * sizeof(float)},        {(void **)&m->V, NP * sizeof(float)},
        {(void **)&m->mean, NI * sizeof(float)},     {(void **)&m->scale, NI * sizeof(float)},
        {(void **)&m->Xn, B * NI * sizeof(float)},   {(void **)&m->H1, B * NH * sizeof(float)},
        {(void **)&m->H2, B * NH * sizeof(float)},   {(void **)&m->dH1, B * NH * sizeof(float)},
        {(void **)&m->dH2, B * NH * sizeof(float)},  {(void **)&m->dz, B * sizeof(float)},
        {(void **)&m->lossv, B * sizeof(double)},    {(void **)&m->loss, sizeof(double)},
    };
    for (auto &w : want) {
        cudaError_t e = cudaMalloc(w.dst, w.bytes);
        if (e != cudaSuccess) {
            mlp_free(m);
            delete m;
            return mlp_fail(LBM_ENOMEM, "device allocation failed", e);
        }
    }
    cudaMemsetAsync(m->P, 0, NP * sizeof(float), m->stream);
    cudaMemsetAsync(m->M, 0, NP * sizeof(float), m->stream);
    cudaMemsetAsync(m->V, 0, NP * sizeof(float), m->stream);
    cudaMemsetAsync(m->mean, 0, NI * sizeof(float), m->stream);
    float ones[NI];
    for (float &v : ones) v = 1.f;
    cudaMemcpyAsync(m->scale, ones, sizeof ones, cudaMemcpyHostToDevice, m->stream);
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        mlp_free(m);
        delete m;
        return mlp_fail(LBM_ECUDA, "initialisation failed", e);
    }
    *out = m;
    return LBM_OK;
}

int lbm_mlp_destroy(lbm_mlp *m)
{
    if (!m) return LBM_OK;
    cudaStreamSynchronize(m->stream);
    mlp_free(m);
    delete m;
    return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp *m, const float *params)
{
    if (!m || !params) return mlp_fail(LBM_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(m->P, params, NP * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->M, 0, NP * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->V, 0, NP * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBM_OK : mlp_fail(LBM_ECUDA, "set_params", e);
}

int lbm_mlp_get_params(lbm_mlp *m, float *params)
{
    if (!m || !params) return mlp_fail(LBM_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(params, m->P, NP * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBM_OK : mlp_fail(LBM_ECUDA, "get_params", e);
}

int lbm_mlp_set_scaling(lbm_mlp *m, const float *mean, const float *scale)
{
    if (!m || !mean || !scale) return mlp_fail(LBM_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(m->mean, mean, NI * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->scale, scale, NI * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBM_OK : mlp_fail(LBM_ECUDA, "set_scaling", e);
}

int lbm_mlp_forward(lbm_mlp *m, const float *x, int n, int bf16, float *prob)
{
    if (!m || (n > 0 && (!x || !prob))) return mlp_fail(LBM_EINVAL, "NULL argument");
    if (n < 0) return mlp_fail(LBM_EINVAL, "n must be >= 0");
    cudaError_t e = mlp_forward_on(m, x, n, nullptr, bf16, prob, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBM_OK : mlp_fail(LBM_ECUDA, "forward", e);
}

int lbm_mlp_loss_grad(lbm_mlp *m, const float *x, const float *y, int n, double *loss, float *grad)
{
    if (!m || !x || !y || !loss) return mlp_fail(LBM_EINVAL, "NULL argument");
    if (n < 1 || n > m->max_batch) return mlp_fail(LBM_EINVAL, "n must be in 1..max_batch");
    const int grid = (n + FWD_THREADS - 1) / FWD_THREADS;
    cudaStream_t s = m->stream;
    k_fwd<false, true><<<grid, FWD_THREADS, 0, s>>>(m->P, m->mean, m->scale, x, n, nullptr, nullptr, y, m->Xn,
                                                    m->H1, m->H2, m->dz, m->lossv);
    k_bwd<<<grid, FWD_THREADS, 0, s>>>(m->P, n, m->dz, m->H1, m->H2, m->dH1, m->dH2);
    k_wgrad<<<(NP + 255) / 256, 256, 0, s>>>(n, m->Xn, m->H1, m->H2, m->dH1, m->dH2, m->dz, m->G);
    k_loss_mean<<<1, 1024, 0, s>>>(m->lossv, n, m->loss);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, m->G, NP * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? LBM_OK : mlp_fail(LBM_ECUDA, "loss_grad", e);
}

int lbm_mlp_adam(lbm_mlp *m, float lr, float beta1, float beta2, float eps, int t)
{
    if (!m || t < 1) return mlp_fail(LBM_EINVAL, "bad argument");
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<(NP + 255) / 256, 256, 0, m->stream>>>(m->P, m->G, m->M, m->V, lr, beta1, beta2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBM_OK : mlp_fail(LBM_ECUDA, "adam", e);
}

}  // extern "C"
