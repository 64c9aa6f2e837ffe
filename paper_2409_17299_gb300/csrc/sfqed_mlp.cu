// K7 / K8: learned surrogate of the emission inverse CDF.
//
// A network 2 -> 64 -> 64 -> 64 -> 1 (SiLU hidden layers, BF16 weights,
// FP32 accumulation) maps (log10(chi)/3, logit(u)/16) to zeta/16 + 1/2, where
// zeta = ln y is what the emission table stores (y = 2 d / (3 chi (1-d))).
// It is trained on samples drawn from the table method itself; the table is
// kept as the fallback outside the trained range.  Training: one block per
// 128 samples, forward and backward through the 64 x 64 layers on the
// tensor cores (mma.sync BF16), gradients accumulated in FP32, then Adam.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"
#include "sfqed_mma.cuh"

namespace sfq {
namespace {

constexpr int TB = 128;                   // samples (threads) per training block
constexpr int TR_SMEM = 3 * TB * MLP_H * 4 + 4 * TB * MLP_H * 2 + MLP_NP * 2 + TB * 3 * 4 + 64;

struct TrainArgs {
    const __nv_bfloat16 *W16;
    float *grad;
    float *loss;                          // accumulated sum of squared errors
    const float *icdf_em32;               // target generator (the table method)
    const float *feat;                    // given features (n x 2), or null: draw them
    const float *target;                  // given targets, or null: from the table
    unsigned long long seed;
    unsigned long long sample0;
    long long n;                          // samples in this launch
    float inv_total;                      // 1 / samples per optimizer step
};

// table target for (log10 chi, logit u) in the FP32 table's own arithmetic
__device__ __forceinline__ float table_zeta(const float *tab, float lc, float s) {
    const float c = (lc + 3.0f) * 20.0f;
    const float t = (s + 16.0f) * 8.0f;
    return bilinear(tab, EM_NCHI, EM_NS, c, t);
}

__global__ void __launch_bounds__(TB) k_mlp_train(TrainArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    float *Z1 = reinterpret_cast<float *>(sm);
    float *Z2 = Z1 + TB * MLP_H;
    float *Z3 = Z2 + TB * MLP_H;
    __nv_bfloat16 *H1 = reinterpret_cast<__nv_bfloat16 *>(Z3 + TB * MLP_H);
    __nv_bfloat16 *H2 = H1 + TB * MLP_H;
    __nv_bfloat16 *H3 = H2 + TB * MLP_H;
    __nv_bfloat16 *D = H3 + TB * MLP_H;
    __nv_bfloat16 *W = D + TB * MLP_H;
    float *F = reinterpret_cast<float *>(W + MLP_NP + (MLP_NP & 1));
    float *DY = F + 2 * TB;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < MLP_NP; i += TB) W[i] = a.W16[i];
    const long long idx = (long long)blockIdx.x * TB + tid;
    const bool live = idx < a.n;
    float f0 = 0.f, f1 = 0.f, ty = 0.f;
    if (live) {
        if (a.feat) {
            f0 = a.feat[2 * idx];
            f1 = a.feat[2 * idx + 1];
            ty = a.target[idx];
        } else {
            const unsigned long long g = a.sample0 + (unsigned long long)idx;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0u, 0x4D4C5000u),
                                          make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32)));
            float u1, v1, u2, v2;
            Uniform<float>::draw(r.x, r.y, u1, v1);
            Uniform<float>::draw(r.z, r.w, u2, v2);
            const float lc = -3.0f + 6.0f * u1;
            float s = logit(u2, v2);
            s = fminf(fmaxf(s, -16.0f), 16.0f);
            f0 = lc / 3.0f;
            f1 = s / 16.0f;
            ty = table_zeta(a.icdf_em32, lc, s) / 16.0f + 0.5f;
        }
    }
    F[2 * tid] = f0;
    F[2 * tid + 1] = f1;
    __syncthreads();
    // layer 1 (FP32)
    for (int o = 0; o < MLP_H; ++o) {
        const float z = __bfloat162float(W[MLP_W1 + 2 * o]) * f0 + __bfloat162float(W[MLP_W1 + 2 * o + 1]) * f1 +
                        __bfloat162float(W[MLP_B1 + o]);
        Z1[tid * MLP_H + o] = z;
        H1[tid * MLP_H + o] = __float2bfloat16_rn(silu_f(z));
    }
    __syncthreads();
    // layers 2 and 3 on the tensor cores: Z = H W^T + b, each warp its 32 rows
    for (int layer = 0; layer < 2; ++layer) {
        const __nv_bfloat16 *Hin = layer == 0 ? H1 : H2;
        __nv_bfloat16 *Hout = layer == 0 ? H2 : H3;
        float *Zout = layer == 0 ? Z2 : Z3;
        const __nv_bfloat16 *Wl = W + (layer == 0 ? MLP_W2 : MLP_W3);
        const __nv_bfloat16 *bl = W + (layer == 0 ? MLP_B2 : MLP_B3);
        auto A = [&](int i, int k) { return Hin[i * MLP_H + k]; };
        auto B = [&](int k, int j) { return Wl[j * MLP_H + k]; };
        for (int mt = 0; mt < 2; ++mt)
            for (int nt = 0; nt < 8; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                const int r0 = warp * 32 + mt * 16;
                mma_tile(r0, nt * 8, MLP_H, A, B, c);
                for (int q = 0; q < 4; ++q) {
                    int r, col;
                    tile_coords(r0, nt * 8, q, r, col);
                    const float z = c[q] + __bfloat162float(bl[col]);
                    Zout[r * MLP_H + col] = z;
                    Hout[r * MLP_H + col] = __float2bfloat16_rn(silu_f(z));
                }
            }
        __syncthreads();
    }
    // layer 4 and the loss
    float y = __bfloat162float(W[MLP_B4]);
    for (int i = 0; i < MLP_H; ++i) y += __bfloat162float(W[MLP_W4 + i]) * __bfloat162float(H3[tid * MLP_H + i]);
    const float res = live ? y - ty : 0.f;
    DY[tid] = 2.0f * res * a.inv_total;
    __syncthreads();
    // gradients of layer 4
    if (tid < MLP_H) {
        float g = 0.f;
        for (int k = 0; k < TB; ++k) g += DY[k] * __bfloat162float(H3[k * MLP_H + tid]);
        atomicAdd(&a.grad[MLP_W4 + tid], g);
    } else if (tid == MLP_H) {
        float g = 0.f;
        for (int k = 0; k < TB; ++k) g += DY[k];
        atomicAdd(&a.grad[MLP_B4], g);
    }
    // D3 = dy W4 * silu'(Z3)
    for (int o = 0; o < MLP_H; ++o)
        D[tid * MLP_H + o] = __float2bfloat16_rn(DY[tid] * __bfloat162float(W[MLP_W4 + o]) * dsilu_f(Z3[tid * MLP_H + o]));
    __syncthreads();
    // layers 3 and 2 backward: dW = D^T H_in, db = sum D, D_in = (D W) * silu'(Z_in)
    for (int layer = 1; layer >= 0; --layer) {
        const __nv_bfloat16 *Hin = layer == 1 ? H2 : H1;
        const float *Zin = layer == 1 ? Z2 : Z1;
        const __nv_bfloat16 *Wl = W + (layer == 1 ? MLP_W3 : MLP_W2);
        float *gW = a.grad + (layer == 1 ? MLP_W3 : MLP_W2);
        float *gb = a.grad + (layer == 1 ? MLP_B3 : MLP_B2);
        {   // dW (64 x 64) over the block's 128 samples: 32 tiles, 8 per warp
            auto A = [&](int o, int k) { return D[k * MLP_H + o]; };
            auto B = [&](int k, int i) { return Hin[k * MLP_H + i]; };
            for (int tt = warp; tt < 32; tt += TB / 32) {
                const int mt = tt >> 3, nt = tt & 7;
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_tile(mt * 16, nt * 8, TB, A, B, c);
                for (int q = 0; q < 4; ++q) {
                    int r, col;
                    tile_coords(mt * 16, nt * 8, q, r, col);
                    atomicAdd(&gW[r * MLP_H + col], c[q]);
                }
            }
        }
        if (tid < MLP_H) {
            float g = 0.f;
            for (int k = 0; k < TB; ++k) g += __bfloat162float(D[k * MLP_H + tid]);
            atomicAdd(&gb[tid], g);
        }
        // D_in into H3's buffer (H3 is dead after layer 4's gradients), then back to D
        __nv_bfloat16 *Dn = H3;
        {
            auto A = [&](int k, int o) { return D[k * MLP_H + o]; };
            auto B = [&](int o, int i) { return Wl[o * MLP_H + i]; };
            for (int mt = 0; mt < 2; ++mt)
                for (int nt = 0; nt < 8; ++nt) {
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
                    const int r0 = warp * 32 + mt * 16;
                    mma_tile(r0, nt * 8, MLP_H, A, B, c);
                    for (int q = 0; q < 4; ++q) {
                        int r, col;
                        tile_coords(r0, nt * 8, q, r, col);
                        Dn[r * MLP_H + col] = __float2bfloat16_rn(c[q] * dsilu_f(Zin[r * MLP_H + col]));
                    }
                }
        }
        __syncthreads();
        for (int o = 0; o < MLP_H; ++o) D[tid * MLP_H + o] = Dn[tid * MLP_H + o];
        __syncthreads();
    }
    // layer 1 gradients
    if (tid < MLP_H) {
        float g0 = 0.f, g1 = 0.f, gbv = 0.f;
        for (int k = 0; k < TB; ++k) {
            const float d = __bfloat162float(D[k * MLP_H + tid]);
            g0 += d * F[2 * k];
            g1 += d * F[2 * k + 1];
            gbv += d;
        }
        atomicAdd(&a.grad[MLP_W1 + 2 * tid], g0);
        atomicAdd(&a.grad[MLP_W1 + 2 * tid + 1], g1);
        atomicAdd(&a.grad[MLP_B1 + tid], gbv);
    }
    float l = res * res;
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) atomicAdd(a.loss, l);
}

__global__ void k_mlp_adam(float *P, float *M, float *V, float *G, __nv_bfloat16 *W16, float lr, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = G[i];
    G[i] = 0.f;
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    const float p = P[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    P[i] = p;
    W16[i] = __float2bfloat16_rn(p);
}

// He-style initialisation from Philox normals (Box-Muller); biases zero
__global__ void k_mlp_init(float *P, float *M, float *V, float *G, __nv_bfloat16 *W16, unsigned long long seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NP) return;
    float fan = 0.f;
    if (i < MLP_B1) fan = 2.f;
    else if (i >= MLP_W2 && i < MLP_B2) fan = 64.f;
    else if (i >= MLP_W3 && i < MLP_B3) fan = 64.f;
    else if (i >= MLP_W4 && i < MLP_B4) fan = 64.f;
    float p = 0.f;
    if (fan > 0.f) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, 0u, 0u, 0x494E4954u),
                                      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
        float u1, v1, u2, v2;
        Uniform<float>::draw(r.x, r.y, u1, v1);
        Uniform<float>::draw(r.z, r.w, u2, v2);
        const float nrm = sqrtf(-2.f * logf(u1)) * cosf(6.2831853f * u2);
        p = nrm * sqrtf(2.f / fan) * (i >= MLP_W4 ? 0.5f : 1.f);
    }
    P[i] = p;
    M[i] = 0.f;
    V[i] = 0.f;
    G[i] = 0.f;
    W16[i] = __float2bfloat16_rn(p);
}

// forward of n feature pairs, one warp per 32 samples (component check)
constexpr int EVAL_T = 128;
__global__ void __launch_bounds__(EVAL_T) k_mlp_eval(const __nv_bfloat16 *W16, const float *feat, long long n,
                                                     float *y) {
    __shared__ __align__(16) unsigned char sm[MLP_INF_BYTES];
    const MlpInf m = mlp_stage(sm, W16);
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float f0 = i < n ? feat[2 * i] : 0.f, f1 = i < n ? feat[2 * i + 1] : 0.f;
    const float out = mlp_forward_warp(f0, f1, m);
    if (i < n) y[i] = out;
}

}  // namespace
}  // namespace sfq

using namespace sfq;

static qed_status mlp_alloc(qed_ctx *ctx) {
    if (ctx->mlp_p) return QED_OK;
    if (cudaMalloc(&ctx->mlp_p, sizeof(float) * MLP_NP * 4) != cudaSuccess ||
        cudaMalloc(&ctx->mlp_w16, sizeof(__nv_bfloat16) * (MLP_NP + 1)) != cudaSuccess ||
        cudaMalloc(&ctx->mlp_loss, sizeof(float) * 2) != cudaSuccess)
        return QED_ERR_NOMEM;
    if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_SMEM) != cudaSuccess)
        return QED_ERR_CUDA;
    return QED_OK;
}

qed_status sfq_mlp_set_params(qed_ctx *ctx, const float *params) {
    if (!ctx || !params) return QED_ERR_INVALID;
    qed_status e = mlp_alloc(ctx);
    if (e != QED_OK) return e;
    cudaStream_t st = ctx->stream;
    float *P = ctx->mlp_p;
    SFQ_CUDA(cudaMemcpyAsync(P, params, sizeof(float) * MLP_NP, cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemsetAsync(P + MLP_NP, 0, sizeof(float) * MLP_NP * 3, st));
    // BF16 copy through the Adam kernel with a zero step (P unchanged)
    k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, st>>>(P, P + MLP_NP, P + 2 * MLP_NP, P + 3 * MLP_NP,
                                                      ctx->mlp_w16, 0.f, 1.f, 1.f);
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaStreamSynchronize(st));
    ctx->mlp_ready = 1;
    return QED_OK;
}

qed_status sfq_mlp_get_params(qed_ctx *ctx, float *params) {
    if (!ctx || !params || !ctx->mlp_p) return QED_ERR_STATE;
    SFQ_CUDA(cudaMemcpyAsync(params, ctx->mlp_p, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost, ctx->stream));
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

qed_status sfq_mlp_eval(qed_ctx *ctx, const float *feat, int64_t n, float *y) {
    if (!ctx || n < 0 || (n > 0 && (!feat || !y))) return QED_ERR_INVALID;
    if (!ctx->mlp_p) return QED_ERR_STATE;
    if (n == 0) return QED_OK;
    k_mlp_eval<<<(unsigned)((n + EVAL_T - 1) / EVAL_T), EVAL_T, 0, ctx->stream>>>(ctx->mlp_w16, feat, n, y);
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

// one gradient of the mean squared error over n given samples (no update)
qed_status sfq_mlp_grad(qed_ctx *ctx, const float *feat, const float *target, int64_t n, float *grad_host,
                        double *loss) {
    if (!ctx || n <= 0 || !feat || !target || !grad_host) return QED_ERR_INVALID;
    if (!ctx->mlp_p) return QED_ERR_STATE;
    cudaStream_t st = ctx->stream;
    float *G = ctx->mlp_p + 3 * MLP_NP;
    SFQ_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * MLP_NP, st));
    SFQ_CUDA(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(float), st));
    TrainArgs a{ctx->mlp_w16, G, ctx->mlp_loss, ctx->icdf_em32, feat, target, 0ull, 0ull, (long long)n,
                1.0f / (float)n};
    k_mlp_train<<<(unsigned)((n + TB - 1) / TB), TB, TR_SMEM, st>>>(a);
    SFQ_CUDA(cudaGetLastError());
    float l = 0.f;
    SFQ_CUDA(cudaMemcpyAsync(grad_host, G, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaMemcpyAsync(&l, ctx->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    SFQ_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * MLP_NP, st));
    if (loss) *loss = l / (double)n;
    return QED_OK;
}

// Train on n_samples table draws: batches of `batch`, Adam with a cosine
// learning-rate decay from lr to lr/100.
qed_status sfq_mlp_train(qed_ctx *ctx, int64_t n_samples, int batch, double lr, uint64_t seed, double *final_loss) {
    if (!ctx || n_samples <= 0 || batch <= 0 || batch % TB || !(lr > 0.0)) return QED_ERR_INVALID;
    qed_status e = mlp_alloc(ctx);
    if (e != QED_OK) return e;
    cudaStream_t st = ctx->stream;
    float *P = ctx->mlp_p, *M = P + MLP_NP, *V = P + 2 * MLP_NP, *G = P + 3 * MLP_NP;
    k_mlp_init<<<(MLP_NP + 255) / 256, 256, 0, st>>>(P, M, V, G, ctx->mlp_w16, seed);
    const int64_t steps = (n_samples + batch - 1) / batch;
    double last = 0.0;
    int64_t last_n = 0;
    for (int64_t s = 0; s < steps; ++s) {
        const bool tail = s >= steps - 16;        // loss of the last steps
        if (tail && s == steps - 16) SFQ_CUDA(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(float), st));
        TrainArgs a{ctx->mlp_w16, G, ctx->mlp_loss, ctx->icdf_em32, nullptr, nullptr, seed,
                    (unsigned long long)(s * batch), (long long)batch, 1.0f / (float)batch};
        k_mlp_train<<<(unsigned)(batch / TB), TB, TR_SMEM, st>>>(a);
        const double frac = (double)s / (double)(steps > 1 ? steps - 1 : 1);
        const double lr_t = lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(3.14159265358979323846 * frac)));
        const double bc1 = 1.0 - pow(0.9, (double)(s + 1)), bc2 = 1.0 - pow(0.999, (double)(s + 1));
        k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, st>>>(P, M, V, G, ctx->mlp_w16, (float)lr_t, (float)bc1,
                                                          (float)bc2);
        SFQ_LAUNCHED(ctx, 2);
        if (tail) last_n += batch;
    }
    SFQ_CUDA(cudaGetLastError());
    float l = 0.f;
    SFQ_CUDA(cudaMemcpyAsync(&l, ctx->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    last = last_n ? (double)l / (double)last_n : 0.0;
    if (final_loss) *final_loss = last;
    ctx->mlp_ready = 1;
    return QED_OK;
}
