// mlp.cu -- learned bond-dimension scheduler (not in the paper): inference
// and training kernels of the 10 -> 64 -> 64 -> 1 MLP with exact-erf GELU,
// MSE loss and Adam, all FP32.  Parameter layout: W1[64][10], b1[64],
// W2[64][64], b2[64], W3[64], b3[1].
//
// Training step = forward with cached activations (thread per sample),
// back-propagation of the activations (thread per sample), parameter
// gradients as small reductions over the batch (thread per parameter, so
// the sum order is fixed and the gradient is deterministic) and the loss.
#include "common.cuh"
#include "ctrl.cuh"

namespace dmrg {
namespace {

constexpr int OFF_W1 = 0, OFF_B1 = MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    float Phi = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    float phi = expf(-0.5f * x * x) * 0.39894228040143268f;
    return Phi + x * phi;
}

// caches (B x 64 each): z1, h1, z2, h2; y (B)
__global__ void k_mlp_fwd(const float *__restrict__ P, int B, const float *__restrict__ X, float *__restrict__ y,
                          float *__restrict__ z1, float *__restrict__ h1, float *__restrict__ z2,
                          float *__restrict__ h2)
{
    __shared__ float sp[MLP_NPARAM];
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sp[i] = P[i];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float x[MLP_IN], a1[MLP_H];
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[(size_t)b * MLP_IN + i];
    for (int j = 0; j < MLP_H; ++j) {
        float acc = sp[OFF_B1 + j];
        for (int i = 0; i < MLP_IN; ++i) acc = fmaf(sp[OFF_W1 + j * MLP_IN + i], x[i], acc);
        if (z1) z1[(size_t)b * MLP_H + j] = acc;
        a1[j] = gelu(acc);
        if (h1) h1[(size_t)b * MLP_H + j] = a1[j];
    }
    float out = sp[OFF_B3];
    for (int j = 0; j < MLP_H; ++j) {
        float acc = sp[OFF_B2 + j];
        for (int i = 0; i < MLP_H; ++i) acc = fmaf(sp[OFF_W2 + j * MLP_H + i], a1[i], acc);
        float g = gelu(acc);
        if (z2) { z2[(size_t)b * MLP_H + j] = acc; h2[(size_t)b * MLP_H + j] = g; }
        out = fmaf(sp[OFF_W3 + j], g, out);
    }
    y[b] = out;
}

// dy_b = 2 (y_b - t_b) / B; dz2 = dy W3 gelu'(z2); dz1 = (W2^T dz2) gelu'(z1)
__global__ void k_mlp_bwd_act(const float *__restrict__ P, int B, const float *__restrict__ y,
                              const float *__restrict__ t, const float *__restrict__ z1, const float *__restrict__ z2,
                              float *__restrict__ dy, float *__restrict__ dz1, float *__restrict__ dz2)
{
    __shared__ float sp[MLP_NPARAM];
    for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) sp[i] = P[i];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float d = 2.0f * (y[b] - t[b]) / (float)B;
    dy[b] = d;
    float g2[MLP_H];
    for (int j = 0; j < MLP_H; ++j) {
        g2[j] = d * sp[OFF_W3 + j] * gelu_grad(z2[(size_t)b * MLP_H + j]);
        dz2[(size_t)b * MLP_H + j] = g2[j];
    }
    for (int i = 0; i < MLP_H; ++i) {
        float acc = 0.0f;
        for (int j = 0; j < MLP_H; ++j) acc = fmaf(sp[OFF_W2 + j * MLP_H + i], g2[j], acc);
        dz1[(size_t)b * MLP_H + i] = acc * gelu_grad(z1[(size_t)b * MLP_H + i]);
    }
}

// one thread per parameter: sum over the batch in sample order
__global__ void k_mlp_grad(int B, const float *__restrict__ X, const float *__restrict__ h1,
                           const float *__restrict__ h2, const float *__restrict__ dy, const float *__restrict__ dz1,
                           const float *__restrict__ dz2, float *__restrict__ grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPARAM) return;
    float acc = 0.0f;
    if (p < OFF_B1) {
        int j = p / MLP_IN, i = p % MLP_IN;
        for (int b = 0; b < B; ++b) acc = fmaf(dz1[(size_t)b * MLP_H + j], X[(size_t)b * MLP_IN + i], acc);
    } else if (p < OFF_W2) {
        int j = p - OFF_B1;
        for (int b = 0; b < B; ++b) acc += dz1[(size_t)b * MLP_H + j];
    } else if (p < OFF_B2) {
        int q = p - OFF_W2, j = q / MLP_H, i = q % MLP_H;
        for (int b = 0; b < B; ++b) acc = fmaf(dz2[(size_t)b * MLP_H + j], h1[(size_t)b * MLP_H + i], acc);
    } else if (p < OFF_W3) {
        int j = p - OFF_B2;
        for (int b = 0; b < B; ++b) acc += dz2[(size_t)b * MLP_H + j];
    } else if (p < OFF_B3) {
        int i = p - OFF_W3;
        for (int b = 0; b < B; ++b) acc = fmaf(dy[b], h2[(size_t)b * MLP_H + i], acc);
    } else {
        for (int b = 0; b < B; ++b) acc += dy[b];
    }
    grad[p] = acc;
}

__global__ void k_mlp_loss(int B, const float *__restrict__ y, const float *__restrict__ t, float *loss)
{
    __shared__ double sh[32];
    double a = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        double r = (double)y[b] - (double)t[b];
        a += r * r;
    }
    a = block_sum(a, sh);
    if (threadIdx.x == 0) loss[0] = (float)(a / B);
}

__global__ void k_adam(int n, float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

}  // namespace
}  // namespace dmrg

using namespace dmrg;

extern "C" {

dmrg_status dmrg_mlp_forward(dmrg_ctx *ctx, const float *params_dev, int B, const float *X_dev, float *y_dev)
{
    if (!ctx || !params_dev || !X_dev || !y_dev || B < 1) return DMRG_EINVAL;
    k_mlp_fwd<<<(B + 127) / 128, 128, 0, ctx->stream>>>(params_dev, B, X_dev, y_dev, nullptr, nullptr, nullptr,
                                                         nullptr); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status dmrg_mlp_loss_grad(dmrg_ctx *ctx, const float *params_dev, int B, const float *X_dev, const float *t_dev,
                               float *loss_dev, float *grad_dev)
{
    if (!ctx || !params_dev || !X_dev || !t_dev || !loss_dev || !grad_dev || B < 1) return DMRG_EINVAL;
    size_t per = (size_t)B * MLP_H;
    size_t need = sizeof(float) * (per * 6 + (size_t)B * 2 + 64);
    DMRG_TRY(ctx->work3.ensure(need));
    float *z1 = ctx->work3.as<float>(), *h1 = z1 + per, *z2 = h1 + per, *h2 = z2 + per, *dz1 = h2 + per,
          *dz2 = dz1 + per, *y = dz2 + per, *dy = y + B;
    cudaStream_t st = ctx->stream;
    k_mlp_fwd<<<(B + 127) / 128, 128, 0, st>>>(params_dev, B, X_dev, y, z1, h1, z2, h2); DMRG_COUNT_LAUNCH();
    k_mlp_bwd_act<<<(B + 127) / 128, 128, 0, st>>>(params_dev, B, y, t_dev, z1, z2, dy, dz1, dz2); DMRG_COUNT_LAUNCH();
    k_mlp_grad<<<(MLP_NPARAM + 127) / 128, 128, 0, st>>>(B, X_dev, h1, h2, dy, dz1, dz2, grad_dev); DMRG_COUNT_LAUNCH();
    k_mlp_loss<<<1, 256, 0, st>>>(B, y, t_dev, loss_dev); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

dmrg_status dmrg_mlp_train(dmrg_ctx *ctx, float *params_dev, int B, const float *X_dev, const float *t_dev,
                           float *m_dev, float *v_dev, int first_step, int steps, float lr, float *loss_host)
{
    if (!ctx || !params_dev || !X_dev || !t_dev || !m_dev || !v_dev || B < 1 || first_step < 1 || steps < 0)
        return DMRG_EINVAL;
    DMRG_TRY(ctx->work2.ensure(sizeof(float) * (MLP_NPARAM + 64)));
    float *grad = ctx->work2.as<float>();
    float *loss = grad + MLP_NPARAM;
    for (int i = 0; i < steps; ++i) {
        DMRG_TRY(dmrg_mlp_loss_grad(ctx, params_dev, B, X_dev, t_dev, loss, grad));
        DMRG_TRY(dmrg_mlp_adam(ctx, MLP_NPARAM, params_dev, grad, m_dev, v_dev, first_step + i, lr, 0.9f, 0.999f,
                               1e-8f));
    }
    if (loss_host) {
        DMRG_CUDA(cudaMemcpyAsync(loss_host, loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        DMRG_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return DMRG_OK;
}

dmrg_status dmrg_mlp_adam(dmrg_ctx *ctx, int n, float *params_dev, const float *grad_dev, float *m_dev, float *v_dev,
                          int step, float lr, float beta1, float beta2, float eps)
{
    if (!ctx || !params_dev || !grad_dev || !m_dev || !v_dev || n < 1 || step < 1) return DMRG_EINVAL;
    float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, params_dev, grad_dev, m_dev, v_dev, lr, beta1, beta2, eps, bc1,
                                                     bc2); DMRG_COUNT_LAUNCH();
    DMRG_CUDA(cudaGetLastError());
    return DMRG_OK;
}

}  // extern "C"
