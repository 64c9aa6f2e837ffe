// Warp-level BF16 tensor-core tiles (mma.sync m16n8k16, FP32 accumulation)
// for inference of the 2 -> 64 -> 64 -> 64 -> 1 surrogate network inside the
// lepton pass, where each warp evaluates its own 32 samples; the parameter
// layout and the activation functions are shared with the training kernel.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace sfq {

constexpr int MLP_H = 64;
constexpr int MLP_NP = MLP_H * 2 + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_H + 1;   // 8577
// parameter offsets (W[out][in] row-major)
constexpr int MLP_W1 = 0, MLP_B1 = 128, MLP_W2 = 192, MLP_B2 = 192 + 4096, MLP_W3 = MLP_B2 + 64,
              MLP_B3 = MLP_W3 + 4096, MLP_W4 = MLP_B3 + 64, MLP_B4 = MLP_W4 + 64;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// SiLU z * sigmoid(z) with the fast exponential and division (the exponent
// is clamped so that 1 + e^-z stays finite)
__device__ __forceinline__ float sigmoid_f(float z) { return __fdividef(1.0f, 1.0f + __expf(-fmaxf(z, -80.0f))); }
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = sigmoid_f(z);
    return s * (1.0f + z * (1.0f - s));
}

// ---- inference: weights staged in shared memory, activations in registers
// The two 64 x 64 layers are kept in BF16 with rows padded to 72 elements
// (fragment loads hit 32 distinct banks); the 2 -> 64 layer, the biases and
// the 64 -> 1 layer are kept in FP32 (converted from BF16 once).
constexpr int MLP_LD = 72;
constexpr int MLP_F_W1 = 0, MLP_F_B1 = 128, MLP_F_B2 = 192, MLP_F_B3 = 256, MLP_F_W4 = 320, MLP_F_B4 = 384;
constexpr int MLP_INF_BYTES = 2 * MLP_H * MLP_LD * 2 + 388 * 4;     // 19984

struct MlpInf {
    const __nv_bfloat16 *W2, *W3;   // [64][MLP_LD]
    const float *f;                 // MLP_F_* offsets
};

// Stage the network (BF16 parameters in global memory, MLP_W*/MLP_B*
// layout) into `smem` (MLP_INF_BYTES, 16-byte aligned).  Every thread of the
// block calls it; the caller synchronises the block before use.
__device__ __forceinline__ MlpInf mlp_stage(unsigned char *smem, const __nv_bfloat16 *W16) {
    __nv_bfloat16 *w2 = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *w3 = w2 + MLP_H * MLP_LD;
    float *f = reinterpret_cast<float *>(w3 + MLP_H * MLP_LD);
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) {
        const int r = i >> 6, c = i & 63;
        w2[r * MLP_LD + c] = W16[MLP_W2 + i];
        w3[r * MLP_LD + c] = W16[MLP_W3 + i];
    }
    for (int i = threadIdx.x; i <= MLP_F_B4; i += blockDim.x) {
        int src;
        if (i < MLP_F_B1) src = MLP_W1 + i;
        else if (i < MLP_F_B2) src = MLP_B1 + (i - MLP_F_B1);
        else if (i < MLP_F_B3) src = MLP_B2 + (i - MLP_F_B2);
        else if (i < MLP_F_W4) src = MLP_B3 + (i - MLP_F_B3);
        else if (i < MLP_F_B4) src = MLP_W4 + (i - MLP_F_W4);
        else src = MLP_B4;
        f[i] = __bfloat162float(W16[src]);
    }
    return MlpInf{w2, w3, f};
}

__device__ __forceinline__ uint32_t silu_pack(float z0, float z1) {
    return pack_bf16(__float2bfloat16_rn(silu_f(z0)), __float2bfloat16_rn(silu_f(z1)));
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// Forward pass of one warp over 32 samples, sample r in lane r (features f0,
// f1).  All 32 lanes must call it.  The warp works on two 16-row tiles; the
// accumulator fragment of one layer's m16n8k16 products is, after bias, SiLU
// and BF16 rounding, exactly the A fragment of the next layer's, so the
// activations stay in registers.  Returns this lane's output.
__device__ __forceinline__ float mlp_forward_warp(float f0, float f1, const MlpInf &m) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int src = 4 * (lane & 7);                 // lane holding row (lane mod 16) of a tile's output
    const bool upper = (lane >> 3) & 1;
    float y = 0.f;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int ra = mt * 16 + g, rb = ra + 8;
        const float a0 = __shfl_sync(0xffffffffu, f0, ra), a1 = __shfl_sync(0xffffffffu, f1, ra);
        const float b0 = __shfl_sync(0xffffffffu, f0, rb), b1 = __shfl_sync(0xffffffffu, f1, rb);
        uint32_t A[4][4];
        // 2 -> 64 on the CUDA cores, written straight into the A fragments
#pragma unroll
        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = 16 * kb + 8 * h + 2 * t;
                const float w00 = m.f[MLP_F_W1 + 2 * col], w01 = m.f[MLP_F_W1 + 2 * col + 1];
                const float w10 = m.f[MLP_F_W1 + 2 * col + 2], w11 = m.f[MLP_F_W1 + 2 * col + 3];
                const float c0 = m.f[MLP_F_B1 + col], c1 = m.f[MLP_F_B1 + col + 1];
                A[kb][2 * h] = silu_pack(w00 * a0 + w01 * a1 + c0, w10 * a0 + w11 * a1 + c1);
                A[kb][2 * h + 1] = silu_pack(w00 * b0 + w01 * b1 + c0, w10 * b0 + w11 * b1 + c1);
            }
        // 64 -> 64 twice on the tensor cores
#pragma unroll 1
        for (int layer = 0; layer < 2; ++layer) {
            const __nv_bfloat16 *Wl = layer == 0 ? m.W2 : m.W3;
            const float *bl = m.f + (layer == 0 ? MLP_F_B2 : MLP_F_B3);
            uint32_t An[4][4];
#pragma unroll
            for (int kn = 0; kn < 4; ++kn)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int nt = 2 * kn + h;
                    const __nv_bfloat16 *wr = Wl + (nt * 8 + g) * MLP_LD + 2 * t;   // B(k, j) = W[j][k]
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int kb = 0; kb < 4; ++kb) {
                        uint32_t bfr[2];
                        bfr[0] = *reinterpret_cast<const uint32_t *>(wr + 16 * kb);
                        bfr[1] = *reinterpret_cast<const uint32_t *>(wr + 16 * kb + 8);
                        mma_bf16_16816(c, A[kb], bfr);
                    }
                    const int col = nt * 8 + 2 * t;
                    const float bc0 = bl[col], bc1 = bl[col + 1];
                    An[kn][2 * h] = silu_pack(c[0] + bc0, c[1] + bc1);       // row g
                    An[kn][2 * h + 1] = silu_pack(c[2] + bc0, c[3] + bc1);   // row g + 8
                }
#pragma unroll
            for (int kb = 0; kb < 4; ++kb)
#pragma unroll
                for (int r = 0; r < 4; ++r) A[kb][r] = An[kb][r];
        }
        // 64 -> 1: partial dot products over this lane's columns, then over t
        float ya = 0.f, yb = 0.f;
#pragma unroll
        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = 16 * kb + 8 * h + 2 * t;
                const float w0 = m.f[MLP_F_W4 + col], w1 = m.f[MLP_F_W4 + col + 1];
                ya += w0 * bf16_lo(A[kb][2 * h]) + w1 * bf16_hi(A[kb][2 * h]);
                yb += w0 * bf16_lo(A[kb][2 * h + 1]) + w1 * bf16_hi(A[kb][2 * h + 1]);
            }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        // lane r takes row r: tile r / 16, row (r mod 16) = g' or g' + 8 of lane 4 g'
        const float ta = __shfl_sync(0xffffffffu, ya, src), tb = __shfl_sync(0xffffffffu, yb, src);
        if ((lane >> 4) == mt) y = upper ? tb : ta;
    }
    return y + m.f[MLP_F_B4];
}

}  // namespace sfq
