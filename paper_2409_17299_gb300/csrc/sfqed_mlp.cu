// K7 / K8: learned surrogate of the emission inverse CDF.
//
// A network 2 -> 64 -> 64 -> 64 -> 1 (SiLU hidden layers, BF16 weights,
// FP32 accumulation) maps (log10(chi)/3, logit(u)/16) to zeta/16 + 1/2, where
// zeta = ln y is what the emission table stores (y = 2 d / (3 chi (1-d))).
// It is trained on samples drawn from the table method itself; the table is
// kept as the fallback outside the trained range.  Training (k_mlp_train
// below): forward and backward products of 128-sample tiles on the tcgen05
// tensor cores with accumulators in tensor memory, gradients summed in FP32,
// Adam, all steps in one cooperative launch.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"
#include "sfqed_mma.cuh"
#include "sfqed_tc.cuh"

namespace sfq {
namespace {

// ---- training on the tensor cores (tcgen05, accumulators in tensor memory)
//
// One persistent cooperative kernel runs every optimizer step.  A CTA holds
// 128 samples at a time (one per tensor-memory lane) and keeps, in shared
// memory, its own copy of the FP32 parameters and Adam moments: every CTA
// applies the same Adam update to the same summed gradient, so the copies
// stay identical and one grid barrier per step suffices.  512 threads: the
// four warps that share a lane quadrant split the 64 columns of their 32
// samples, 16 each.
//
// Per tile of 128 samples (B = BF16 storage, as in the network the oracle
// defines; Z and dy stay FP32):
//   Z2 = H1 W2^T, Z3 = H2 W3^T           M=128 N=64 K=64   (tensor memory)
//   P3 = D3 W3,   P2 = D2 W2             M=128 N=64 K=64
//   G1 = [D3;D2] x [H2;H1;1]             M=128 N=144 K=128: dW3, dW2, db3, db2
//   G2 = [D1;H3] x [f0 hi/lo, f1 hi/lo, 1, dy hi/lo]
//                                        M=128 N=16 K=128: dW1, db1, dW4
// (the first factor MN-major: rows are units, K runs over the samples).
// Layer 1 (2 -> 64) and layer 4 (64 -> 1) run on the CUDA cores.  The SiLU
// derivatives are computed in the forward pass and kept in tensor memory
// until the backward pass multiplies them in.  G1 and G2 accumulate over
// the CTA's tiles of a step and are added to the step's gradient sum with
// vector atomics.  Features and dy enter G2 as BF16 hi + lo pairs, so the
// BF16 operand rounding leaves them exact to about 2^-17.
constexpr int TT = 512;                       // threads
constexpr int TS = 128;                       // samples per tile = tensor-memory lanes
constexpr int GSTRIDE = 8580;                 // MLP_NP rounded up to whole float4s
// shared memory (bytes).  Activation / delta tiles: 128 samples x 64 units
// in core matrices of 8 samples x 8 units; unit block j at j x 2048, sample
// r at r x 16.  Weight tiles W[o][i]: (o/8) x 1024 + (i/8) x 128.
constexpr int SM_W2 = 0, SM_W3 = 8192;
constexpr int SM_D3 = 16384, SM_D2 = SM_D3 + 16384;                       // [D3; D2]
constexpr int SM_H2 = SM_D2 + 16384, SM_H1 = SM_H2 + 16384;               // [H2; H1; ones; zero]
constexpr int SM_ONES = SM_H1 + 16384, SM_ZERO = SM_ONES + 2048;
constexpr int SM_FB = SM_ZERO + 2048, SM_D1 = SM_FB + 2048, SM_H3 = SM_D1 + 16384;   // [FB; D1], [D1; H3]
constexpr int SM_P = SM_H3 + 16384, SM_M = SM_P + GSTRIDE * 4, SM_V = SM_M + GSTRIDE * 4;
constexpr int SM_WQ = SM_V + GSTRIDE * 4;                                 // BF16-rounded W1, biases, W4 (MLP_F_*)
constexpr int SM_YP = SM_WQ + 388 * 4;                                    // partial outputs [4][128]
constexpr int SM_SF = SM_YP + 4 * TS * 4;                                 // sample: f0, f1, target, live [128]
constexpr int SM_MISC = SM_SF + TS * 16;
constexpr int TR_SMEM = SM_MISC + 64;
static_assert(SM_P % 16 == 0 && SM_WQ % 16 == 0 && SM_MISC % 8 == 0 && GSTRIDE % 4 == 0, "alignment");
static_assert(MLP_B1 % 4 == 0 && MLP_W2 % 4 == 0 && MLP_B2 % 4 == 0 && MLP_W3 % 4 == 0 && MLP_B3 % 4 == 0 &&
                  MLP_W4 % 4 == 0 && MLP_B4 % 4 == 0 && GSTRIDE - MLP_B4 <= 4,
              "the Adam update takes the parameters in groups of four that never straddle two regions");
static_assert(TR_SMEM <= 227 * 1024, "shared memory");
// tensor-memory columns: products, SiLU derivatives of layers 1 and 2, gradients
constexpr uint32_t TM_COLS = 512, TZ = 0, TD1 = 64, TD2 = 128, TG1 = 256, TG2 = 416;
constexpr uint32_t WAIT_POLLS = 1u << 22, BAR_POLLS = 1u << 24;      // defaults of the bounded waits
// instruction descriptors: forward (A, B K-major), backward (B MN-major), gradients
constexpr uint32_t ID_FWD = tc::idesc_bf16(128, 64, 0, 0), ID_BWD = tc::idesc_bf16(128, 64, 0, 1);
constexpr uint32_t ID_G1 = tc::idesc_bf16(128, 144, 1, 1), ID_G2 = tc::idesc_bf16(128, 16, 1, 1);

struct TrainArgs {
    float *P, *M, *V;                         // parameters and moments (read at start, written back at the end)
    float *gbuf;                              // three gradient sums of GSTRIDE floats (zero at launch); the gradient
    __nv_bfloat16 *W16;
    float *loss;                              // sum of squared errors of the counted steps
    const float *icdf_em32;                   // target generator (the table method)
    const float *feat, *target;               // given samples, or null: draw them
    const float *sched;                       // per step: lr / bias correction 1, 1 / bias correction 2
    unsigned long long seed;
    long long per_step;                       // samples per step (the batch), or the given samples
    long long steps;                          // optimizer steps; 0: one gradient, no update
    long long tail_from;                      // steps from here on add to *loss
    float inv_total;                          // 1 / per_step
    unsigned *bar;                            // grid-barrier arrivals (zero at launch)
    uint32_t bar_polls;                       // polls of a grid barrier before the launch gives up
    int *status;                              // 0 ok, 1 a barrier wait ran out, 2 an MMA wait ran out
};

// table target for (log10 chi, logit u) in the FP32 table's own arithmetic
__device__ __forceinline__ float table_zeta(const float *tab, float lc, float s) {
    const float c = (lc + 3.0f) * 20.0f;
    const float t = (s + 16.0f) * 8.0f;
    return bilinear(tab, EM_NCHI, EM_NS, c, t);
}

__device__ __forceinline__ uint32_t wtile_off(int o, int i) {
    return (uint32_t)((o >> 3) * 1024 + (i >> 3) * 128 + (o & 7) * 16 + (i & 7) * 2);
}

// parameter p's BF16 value where the forward and backward passes read it
__device__ __forceinline__ void put_weight(unsigned char *sm, float *wq, int p, float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    if (p >= MLP_W2 && p < MLP_B2) {
        const int q = p - MLP_W2;
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_W2 + wtile_off(q >> 6, q & 63)) = b;
    } else if (p >= MLP_W3 && p < MLP_B3) {
        const int q = p - MLP_W3;
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_W3 + wtile_off(q >> 6, q & 63)) = b;
    } else {
        int d;
        if (p < MLP_B1) d = MLP_F_W1 + p;
        else if (p < MLP_W2) d = MLP_F_B1 + (p - MLP_B1);
        else if (p < MLP_W3) d = MLP_F_B2 + (p - MLP_B2);
        else if (p < MLP_W4) d = MLP_F_B3 + (p - MLP_B3);
        else if (p < MLP_B4) d = MLP_F_W4 + (p - MLP_W4);
        else d = MLP_F_B4;
        wq[d] = __bfloat162float(b);
    }
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);     // a in the low half
    return *reinterpret_cast<const uint32_t *>(&h);
}

// fire-and-forget additions to global memory (no value returned)
__device__ __forceinline__ void red_add(float *p, float a) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(a) : "memory");
}
__device__ __forceinline__ void red_add2(float *p, float a, float b) {
    asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add4(float *p, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// all CTAs arrive; false when a wait ran out (the status word says which)
__device__ bool grid_sync(unsigned *bar, unsigned target, uint32_t polls, int *status, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned v = 0;
        for (uint32_t it = 0; it < polls; ++it) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target || *reinterpret_cast<volatile int *>(status)) break;
        }
        if (v < target) {
            atomicCAS(status, 0, 1);
            *s_flag = 1;
        }
        __threadfence();
    }
    __syncthreads();
    return *reinterpret_cast<volatile int *>(s_flag) == 0;
}

// 16 activations of one sample row (units u0..u0+15): pre-activation z (with
// bias) -> BF16 SiLU into two unit blocks of `tile`, SiLU derivative into d
__device__ __forceinline__ void silu_row(unsigned char *tile, int u0, int r, const float z[16], float d[16],
                                         float h[16]) {
    uint32_t pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float s0 = sigmoid_f(z[2 * q]), s1 = sigmoid_f(z[2 * q + 1]);
        pk[q] = pack2(z[2 * q] * s0, z[2 * q + 1] * s1);
        d[2 * q] = s0 * (1.0f + z[2 * q] * (1.0f - s0));
        d[2 * q + 1] = s1 * (1.0f + z[2 * q + 1] * (1.0f - s1));
        h[2 * q] = bf16_lo(pk[q]);
        h[2 * q + 1] = bf16_hi(pk[q]);
    }
    *reinterpret_cast<uint4 *>(tile + (u0 / 8) * 2048 + r * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4 *>(tile + (u0 / 8 + 1) * 2048 + r * 16) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

__device__ __forceinline__ void store_row(unsigned char *tile, int u0, int r, const float v[16]) {
    uint32_t pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pk[q] = pack2(v[2 * q], v[2 * q + 1]);
    *reinterpret_cast<uint4 *>(tile + (u0 / 8) * 2048 + r * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4 *>(tile + (u0 / 8 + 1) * 2048 + r * 16) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

__global__ void __launch_bounds__(TT, 1) k_mlp_train(TrainArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    float *sP = reinterpret_cast<float *>(sm + SM_P), *sM = reinterpret_cast<float *>(sm + SM_M);
    float *sV = reinterpret_cast<float *>(sm + SM_V), *wq = reinterpret_cast<float *>(sm + SM_WQ);
    float *yp = reinterpret_cast<float *>(sm + SM_YP);
    float4 *sf = reinterpret_cast<float4 *>(sm + SM_SF);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + SM_MISC);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + SM_MISC + 8);
    int *s_flag = reinterpret_cast<int *>(sm + SM_MISC + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, cq = warp >> 2;       // lane quadrant; column quarter
    const int r = quad * 32 + lane, u0 = cq * 16;    // sample row; first unit of this thread
    const bool train = a.steps > 0;
    const uint32_t base = tc::smem_u32(sm);

    for (int p = tid; p < GSTRIDE; p += TT) {
        const bool in = p < MLP_NP;                  // the last three entries pad to a whole float4
        sP[p] = in ? a.P[p] : 0.f;
        sM[p] = in && train ? a.M[p] : 0.f;
        sV[p] = in && train ? a.V[p] : 0.f;
        if (in) put_weight(sm, wq, p, sP[p]);
    }
    // constant blocks: a BF16 one in unit 0 of every sample row; zeros
    if (tid < TS) {
        *reinterpret_cast<uint4 *>(sm + SM_ONES + tid * 16) = make_uint4(0x3F80u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(sm + SM_ZERO + tid * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) tc::alloc(tslot, TM_COLS);
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        *s_flag = 0;
    }
    tc::fence_proxy_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot, tl = tmem + ((uint32_t)(quad * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;

    // shared-memory writes done: hand the tiles to the tensor cores, one
    // thread issues `fn`, everyone waits for its completion
    auto run_mma = [&](auto fn) -> bool {
        tc::fence_proxy_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            fn();
            tc::commit(mbar);
        }
        bool done = tc::mbar_wait(mbar, phase, WAIT_POLLS);
        phase ^= 1u;
        tc::fence_after_sync();
        done = __syncthreads_and(done);
        if (!done && tid == 0) atomicCAS(a.status, 0, 2);
        return done;
    };
    auto k_steps = [&](uint32_t d, uint32_t aa, uint32_t alb, uint32_t asb, uint32_t ast, uint32_t bb,
                       uint32_t blb, uint32_t bsb, uint32_t bst, uint32_t id, int n, bool acc) {
        for (int kk = 0; kk < n; ++kk)
            tc::mma(d, tc::sdesc(aa + kk * ast, alb, asb), tc::sdesc(bb + kk * bst, blb, bsb), id, acc || kk > 0);
    };
    auto bias16 = [&](int off, float z[16]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 b = *reinterpret_cast<const float4 *>(wq + off + u0 + 4 * q);
            z[4 * q] += b.x;
            z[4 * q + 1] += b.y;
            z[4 * q + 2] += b.z;
            z[4 * q + 3] += b.w;
        }
    };

    // the samples of tile t of step s: drawn (or read) by the first 128
    // threads into sf; the caller synchronises the block before use
    auto draw = [&](long long s_, long long t) {
        if (tid < TS) {
            const long long idx = t * TS + tid;
            float f0 = 0.f, f1 = 0.f, ty = 0.f;
            const bool live = idx < a.per_step;
            if (live) {
                if (a.feat) {
                    f0 = a.feat[2 * idx];
                    f1 = a.feat[2 * idx + 1];
                    ty = a.target[idx];
                } else {
                    const unsigned long long gi = (unsigned long long)s_ * a.per_step + (unsigned long long)idx;
                    const uint4 q = philox4x32_10(make_uint4((uint32_t)gi, (uint32_t)(gi >> 32), 0u, 0x4D4C5000u),
                                                  make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32)));
                    float u1, v1, u2, v2;
                    Uniform<float>::draw(q.x, q.y, u1, v1);
                    Uniform<float>::draw(q.z, q.w, u2, v2);
                    const float lc = -3.0f + 6.0f * u1;
                    float sv = logit(u2, v2);
                    sv = fminf(fmaxf(sv, -16.0f), 16.0f);
                    f0 = lc / 3.0f;
                    f1 = sv / 16.0f;
                    ty = table_zeta(a.icdf_em32, lc, sv) / 16.0f + 0.5f;
                }
            }
            sf[tid] = make_float4(f0, f1, ty, live ? 1.f : 0.f);
        }
    };

    const long long tiles = (a.per_step + TS - 1) / TS;
    const long long nsteps = train ? a.steps : 1;
    bool drawn = false;                              // sf already holds the next tile's samples
    for (long long s = 0; s < nsteps && ok; ++s) {
        float *g = a.gbuf + (train ? (s % 3) * GSTRIDE : 0);
        float dysum = 0.f, sq = 0.f;
        bool first = true;
        for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
            if (!drawn) draw(s, t);
            drawn = false;
            __syncthreads();
            const float4 smp = sf[r];
            const float f0 = smp.x, f1 = smp.y;
            // layer 1 on the CUDA cores: H1, SiLU' into tensor memory
            {
                float z[16], d[16], h[16];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float4 w = *reinterpret_cast<const float4 *>(wq + MLP_F_W1 + 2 * (u0 + 2 * q));
                    z[2 * q] = w.x * f0 + w.y * f1;
                    z[2 * q + 1] = w.z * f0 + w.w * f1;
                }
                bias16(MLP_F_B1, z);
                silu_row(sm + SM_H1, u0, r, z, d, h);
                tc::st16(tl + TD1 + u0, d);
            }
            // Z2 = H1 W2^T -> H2, SiLU'
            ok = run_mma([&] { k_steps(tmem + TZ, base + SM_H1, 2048, 128, 4096, base + SM_W2, 128, 1024, 256, ID_FWD, 4, false); });
            if (!ok) break;
            {
                float z[16], d[16], h[16];
                tc::ld16(tl + TZ + u0, z);
                bias16(MLP_F_B2, z);
                silu_row(sm + SM_H2, u0, r, z, d, h);
                tc::st16(tl + TD2 + u0, d);
            }
            // Z3 = H2 W3^T -> H3, the output y (layer 4), D3 = dy W4 SiLU'(Z3)
            ok = run_mma([&] { k_steps(tmem + TZ, base + SM_H2, 2048, 128, 4096, base + SM_W3, 128, 1024, 256, ID_FWD, 4, false); });
            if (!ok) break;
            {
                float z[16], d[16], h[16];
                tc::ld16(tl + TZ + u0, z);
                bias16(MLP_F_B3, z);
                silu_row(sm + SM_H3, u0, r, z, d, h);
                float yq = 0.f;
#pragma unroll
                for (int q = 0; q < 16; ++q) yq += wq[MLP_F_W4 + u0 + q] * h[q];
                yp[cq * TS + r] = yq;
                __syncthreads();
                const float y = wq[MLP_F_B4] + ((yp[r] + yp[TS + r]) + yp[2 * TS + r]) + yp[3 * TS + r];
                const float res = smp.w != 0.f ? y - smp.z : 0.f;
                const float dy = 2.0f * res * a.inv_total;
                if (cq == 0) {
                    dysum += dy;
                    sq += res * res;
                    // G2's B row: f0, f1 and dy as BF16 hi + lo, and a one
                    const __nv_bfloat16 f0h = __float2bfloat16_rn(f0), f1h = __float2bfloat16_rn(f1);
                    const __nv_bfloat16 dyh = __float2bfloat16_rn(dy);
                    const __nv_bfloat16 f0l = __float2bfloat16_rn(f0 - __bfloat162float(f0h));
                    const __nv_bfloat16 f1l = __float2bfloat16_rn(f1 - __bfloat162float(f1h));
                    const __nv_bfloat16 dyl = __float2bfloat16_rn(dy - __bfloat162float(dyh));
                    *reinterpret_cast<uint4 *>(sm + SM_FB + r * 16) =
                        make_uint4(pack_bf16(f0h, f0l), pack_bf16(f1h, f1l), pack_bf16(__float2bfloat16_rn(1.0f), dyh),
                                   pack_bf16(dyl, __float2bfloat16_rn(0.0f)));
                }
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = dy * wq[MLP_F_W4 + u0 + q] * d[q];
                store_row(sm + SM_D3, u0, r, v);
            }
            // P3 = D3 W3; D2 = P3 SiLU'(Z2)
            ok = run_mma([&] { k_steps(tmem + TZ, base + SM_D3, 2048, 128, 4096, base + SM_W3, 1024, 128, 2048, ID_BWD, 4, false); });
            if (!ok) break;
            {
                float pv[16], d[16];
                tc::ld16(tl + TZ + u0, pv);
                tc::ld16(tl + TD2 + u0, d);
#pragma unroll
                for (int q = 0; q < 16; ++q) pv[q] *= d[q];
                store_row(sm + SM_D2, u0, r, pv);
            }
            // P2 = D2 W2; D1 = P2 SiLU'(Z1)
            ok = run_mma([&] { k_steps(tmem + TZ, base + SM_D2, 2048, 128, 4096, base + SM_W2, 1024, 128, 2048, ID_BWD, 4, false); });
            if (!ok) break;
            {
                float pv[16], d[16];
                tc::ld16(tl + TZ + u0, pv);
                tc::ld16(tl + TD1 + u0, d);
#pragma unroll
                for (int q = 0; q < 16; ++q) pv[q] *= d[q];
                store_row(sm + SM_D1, u0, r, pv);
            }
            // weight and bias gradients of the tile, accumulated over the CTA's tiles of the step
            const bool acc = !first;
            ok = run_mma([&] {
                k_steps(tmem + TG1, base + SM_D3, 128, 2048, 256, base + SM_H2, 128, 2048, 256, ID_G1, 8, acc);
                k_steps(tmem + TG2, base + SM_D1, 128, 2048, 256, base + SM_FB, 128, 2048, 256, ID_G2, 8, acc);
            });
            first = false;
        }
        if (!ok) break;
        if (!first) {
            // row r of G1: dW3 row r and db3 (r < 64), or dW2 row r - 64 and db2;
            // this thread's 16 columns of it
            const bool lo = r < 64;
            float *gw = g + (lo ? MLP_W3 + r * 64 : MLP_W2 + (r - 64) * 64) + u0;
            float v[16];
            tc::ld16(tl + TG1 + (lo ? 0u : 64u) + u0, v);
#pragma unroll
            for (int q = 0; q < 16; q += 4)
                red_add4(gw + q, v[q], v[q + 1], v[q + 2], v[q + 3]);
            if (cq == 0) {
                float v8[8];
                tc::ld8(tl + TG1 + 128, v8);
                red_add(g + (lo ? MLP_B3 + r : MLP_B2 + (r - 64)), v8[0]);
                tc::ld8(tl + TG2, v8);
                if (lo) {
                    red_add2(g + MLP_W1 + 2 * r, v8[0] + v8[1], v8[2] + v8[3]);
                    red_add(g + MLP_B1 + r, v8[4]);
                } else {
                    red_add(g + MLP_W4 + (r - 64), v8[5] + v8[6]);
                }
            }
        }
        if (cq == 0) {
            for (int o = 16; o > 0; o >>= 1) {
                dysum += __shfl_down_sync(0xffffffffu, dysum, o);
                sq += __shfl_down_sync(0xffffffffu, sq, o);
            }
            if (lane == 0) {
                if (dysum != 0.f) red_add(g + MLP_B4, dysum);
                if (!train || s >= a.tail_from) red_add(a.loss, sq);
            }
        }
        if (!train) break;
        // the next step's first samples do not depend on the update: drawn
        // while the other CTAs arrive
        if (s + 1 < nsteps && blockIdx.x < tiles) {
            draw(s + 1, blockIdx.x);
            drawn = true;
        }
        // every CTA's sums are in: the same Adam update in every CTA
        if (!grid_sync(a.bar, (unsigned)(gridDim.x * (s + 1)), a.bar_polls, a.status, s_flag)) {
            ok = false;
            break;
        }
        const float lr_c = a.sched[2 * s], ibc2 = a.sched[2 * s + 1];
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        // four consecutive parameters per thread and group (every region of
        // the layout starts at a multiple of four, so a group never straddles
        // two), all gradient loads in flight before the first use
        constexpr int NG = GSTRIDE / 4, AG = (NG + TT - 1) / TT;
        float4 gv[AG];
#pragma unroll
        for (int k = 0; k < AG; ++k) {
            const int gi = tid + k * TT;
            gv[k] = gi < NG ? __ldcg(reinterpret_cast<const float4 *>(g) + gi) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        auto adam = [&](float gr, float &m, float &v, float &pp) {
            m = b1 * m + (1.f - b1) * gr;
            v = b2 * v + (1.f - b2) * gr * gr;
            pp = pp - __fdividef(lr_c * m, sqrt_approx(v * ibc2) + eps);
        };
#pragma unroll
        for (int k = 0; k < AG; ++k) {
            const int gi = tid + k * TT, p = 4 * gi;
            if (gi >= NG) break;
            float4 m4 = reinterpret_cast<float4 *>(sM)[gi], v4 = reinterpret_cast<float4 *>(sV)[gi];
            float4 p4 = reinterpret_cast<float4 *>(sP)[gi];
            adam(gv[k].x, m4.x, v4.x, p4.x);
            adam(gv[k].y, m4.y, v4.y, p4.y);
            adam(gv[k].z, m4.z, v4.z, p4.z);
            adam(gv[k].w, m4.w, v4.w, p4.w);
            reinterpret_cast<float4 *>(sM)[gi] = m4;
            reinterpret_cast<float4 *>(sV)[gi] = v4;
            reinterpret_cast<float4 *>(sP)[gi] = p4;
            // the BF16 values where the passes read them
            const uint2 b = make_uint2(pack2(p4.x, p4.y), pack2(p4.z, p4.w));
            if (p >= MLP_W2 && p < MLP_B2) {
                const int q = p - MLP_W2;
                *reinterpret_cast<uint2 *>(sm + SM_W2 + wtile_off(q >> 6, q & 63)) = b;
            } else if (p >= MLP_W3 && p < MLP_B3) {
                const int q = p - MLP_W3;
                *reinterpret_cast<uint2 *>(sm + SM_W3 + wtile_off(q >> 6, q & 63)) = b;
            } else {
                // W1, b1 at MLP_F_W1 = 0.., b2 at MLP_F_B2, b3, W4, b4 (and the
                // group's padding) at MLP_F_B3..: offsets p, p - 4096, p - 8192
                const int d = p < MLP_W2 ? p : (p < MLP_W3 ? p - (MLP_B2 - MLP_F_B2) : p - (MLP_B3 - MLP_F_B3));
                *reinterpret_cast<float4 *>(wq + d) = make_float4(bf16_lo(b.x), bf16_hi(b.x), bf16_lo(b.y), bf16_hi(b.y));
            }
        }
        // the sum two steps ahead was last read before this step's barrier
        float *gz = a.gbuf + ((s + 2) % 3) * GSTRIDE;
        for (int p = blockIdx.x * TT + tid; p < GSTRIDE; p += gridDim.x * TT) __stcg(gz + p, 0.f);
        __syncthreads();
    }
    if (train && ok && blockIdx.x == 0) {
        for (int p = tid; p < MLP_NP; p += TT) {
            a.P[p] = sP[p];
            a.M[p] = sM[p];
            a.V[p] = sV[p];
            a.W16[p] = __float2bfloat16_rn(sP[p]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, TM_COLS);
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

// scratch of one training or gradient call: three gradient sums (the
// gradient call uses the context's gradient buffer instead), the step
// schedule, the barrier counter and the status word
struct TrainScratch {
    void *mem = nullptr;
    float *gbuf = nullptr, *sched = nullptr;
    unsigned *bar = nullptr;
    int *status = nullptr;
    ~TrainScratch() {
        if (mem) cudaFree(mem);
    }
};

static qed_status train_scratch(TrainScratch &t, int64_t steps, cudaStream_t st) {
    const size_t g = sizeof(float) * 3 * GSTRIDE, sc = sizeof(float) * 2 * (size_t)(steps > 0 ? steps : 1);
    const size_t bytes = g + ((sc + 255) / 256) * 256 + 256;
    if (cudaMalloc(&t.mem, bytes) != cudaSuccess) return QED_ERR_NOMEM;
    t.gbuf = static_cast<float *>(t.mem);
    t.sched = reinterpret_cast<float *>(static_cast<char *>(t.mem) + g);
    t.bar = reinterpret_cast<unsigned *>(static_cast<char *>(t.mem) + g + ((sc + 255) / 256) * 256);
    t.status = reinterpret_cast<int *>(t.bar + 1);
    SFQ_CUDA(cudaMemsetAsync(t.gbuf, 0, g, st));
    SFQ_CUDA(cudaMemsetAsync(t.bar, 0, 256, st));
    return QED_OK;
}

// CTAs of the training kernel: one per SM at most (its shared memory and
// tensor-memory columns take a whole SM), no more than there are tiles
static qed_status train_grid(long long tiles, int *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    SFQ_CUDA(cudaGetDevice(&dev));
    SFQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SFQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_train, TT, TR_SMEM));
    if (per_sm < 1) return QED_ERR_CUDA;
    const long long cap = (long long)sms * per_sm;
    *grid = (int)(tiles < cap ? tiles : cap);
    return QED_OK;
}

// one gradient of the mean squared error over n given samples (no update)
qed_status sfq_mlp_grad(qed_ctx *ctx, const float *feat, const float *target, int64_t n, float *grad_host,
                        double *loss) {
    if (!ctx || n <= 0 || !feat || !target || !grad_host) return QED_ERR_INVALID;
    if (!ctx->mlp_p) return QED_ERR_STATE;
    cudaStream_t st = ctx->stream;
    float *P = ctx->mlp_p;
    TrainScratch t;
    qed_status e = train_scratch(t, 0, st);
    if (e != QED_OK) return e;
    SFQ_CUDA(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(float), st));
    int grid = 0;
    if ((e = train_grid((n + TS - 1) / TS, &grid)) != QED_OK) return e;
    TrainArgs a{P, P + MLP_NP, P + 2 * MLP_NP, t.gbuf, ctx->mlp_w16, ctx->mlp_loss, ctx->icdf_em32, feat, target,
                t.sched, 0ull, (long long)n, 0ll, 0ll, 1.0f / (float)n, t.bar, BAR_POLLS, t.status};
    k_mlp_train<<<grid, TT, TR_SMEM, st>>>(a);
    SFQ_CUDA(cudaGetLastError());
    SFQ_LAUNCHED(ctx, 1);
    float l = 0.f;
    int status = 0;
    SFQ_CUDA(cudaMemcpyAsync(grad_host, t.gbuf, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaMemcpyAsync(&l, ctx->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaMemcpyAsync(&status, t.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    if (status) return QED_ERR_TIMEOUT;
    if (loss) *loss = l / (double)n;
    return QED_OK;
}

// Train on n_samples table draws: batches of `batch`, Adam with a cosine
// learning-rate decay from lr to lr/100.  All steps run in one cooperative
// launch of k_mlp_train; the step schedule is computed here in FP64 and
// rounded to FP32 once.
qed_status sfq_mlp_train(qed_ctx *ctx, int64_t n_samples, int batch, double lr, uint64_t seed, double *final_loss) {
    if (!ctx || n_samples <= 0 || batch <= 0 || batch % TS || !(lr > 0.0)) return QED_ERR_INVALID;
    qed_status e = mlp_alloc(ctx);
    if (e != QED_OK) return e;
    cudaStream_t st = ctx->stream;
    float *P = ctx->mlp_p, *M = P + MLP_NP, *V = P + 2 * MLP_NP, *G = P + 3 * MLP_NP;
    k_mlp_init<<<(MLP_NP + 255) / 256, 256, 0, st>>>(P, M, V, G, ctx->mlp_w16, seed);
    SFQ_CUDA(cudaGetLastError());
    const int64_t steps = (n_samples + batch - 1) / batch;
    std::vector<float> sched((size_t)steps * 2);
    for (int64_t s = 0; s < steps; ++s) {
        const double frac = (double)s / (double)(steps > 1 ? steps - 1 : 1);
        const double lr_t = lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(3.14159265358979323846 * frac)));
        const double bc1 = 1.0 - pow(0.9, (double)(s + 1)), bc2 = 1.0 - pow(0.999, (double)(s + 1));
        sched[2 * s] = (float)(lr_t / bc1);
        sched[2 * s + 1] = (float)(1.0 / bc2);
    }
    TrainScratch t;
    if ((e = train_scratch(t, steps, st)) != QED_OK) return e;
    SFQ_CUDA(cudaMemcpyAsync(t.sched, sched.data(), sizeof(float) * sched.size(), cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(float), st));
    int grid = 0;
    if ((e = train_grid(batch / TS, &grid)) != QED_OK) return e;
    const int64_t tail = steps < 16 ? steps : 16;     // the loss is averaged over the last 16 steps
    TrainArgs a{P, M, V, t.gbuf, ctx->mlp_w16, ctx->mlp_loss, ctx->icdf_em32, nullptr, nullptr, t.sched, seed,
                (long long)batch, (long long)steps, (long long)(steps - tail), 1.0f / (float)batch, t.bar,
                ctx->cfg.wait_polls > 0 ? (uint32_t)ctx->cfg.wait_polls : BAR_POLLS, t.status};
    void *args[] = {&a};
    SFQ_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_mlp_train), dim3(grid), dim3(TT), args,
                                         (size_t)TR_SMEM, st));
    SFQ_LAUNCHED(ctx, 2);
    float l = 0.f;
    int status = 0;
    SFQ_CUDA(cudaMemcpyAsync(&l, ctx->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaMemcpyAsync(&status, t.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    if (status) return QED_ERR_TIMEOUT;
    if (final_loss) *final_loss = (double)l / (double)(tail * batch);
    ctx->mlp_ready = 1;
    return QED_OK;
}
