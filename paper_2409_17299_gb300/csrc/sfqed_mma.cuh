// Warp-level BF16 tensor-core tiles (mma.sync m16n8k16, FP32 accumulation)
// for the 2 -> 64 -> 64 -> 64 -> 1 surrogate network.  Operands are read
// through index functors so one routine serves the forward product H W^T,
// the input-gradient product D W and the weight-gradient product D^T H.
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

// One 16 x 8 tile of C = A B (rows row0.., columns col0..) accumulated over
// K (a multiple of 16).  a(i, k) and b(k, j) return bf16 elements.  The
// fragment layout is that of mma.m16n8k16: lane = 4 g + t holds
// A rows g, g+8 / columns 2t, 2t+1, 2t+8, 2t+9; B rows 2t, 2t+1, 2t+8, 2t+9 /
// column g; C rows g, g+8 / columns 2t, 2t+1.
template <class FA, class FB>
__device__ __forceinline__ void mma_tile(int row0, int col0, int K, FA a, FB b, float c[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t af[4], bf[2];
        af[0] = pack_bf16(a(row0 + g, k0 + 2 * t), a(row0 + g, k0 + 2 * t + 1));
        af[1] = pack_bf16(a(row0 + g + 8, k0 + 2 * t), a(row0 + g + 8, k0 + 2 * t + 1));
        af[2] = pack_bf16(a(row0 + g, k0 + 2 * t + 8), a(row0 + g, k0 + 2 * t + 9));
        af[3] = pack_bf16(a(row0 + g + 8, k0 + 2 * t + 8), a(row0 + g + 8, k0 + 2 * t + 9));
        bf[0] = pack_bf16(b(k0 + 2 * t, col0 + g), b(k0 + 2 * t + 1, col0 + g));
        bf[1] = pack_bf16(b(k0 + 2 * t + 8, col0 + g), b(k0 + 2 * t + 9, col0 + g));
        mma_bf16_16816(c, af, bf);
    }
}

// where the four accumulators of a tile live in C
__device__ __forceinline__ void tile_coords(int row0, int col0, int q, int &r, int &col) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    r = row0 + g + ((q & 2) ? 8 : 0);
    col = col0 + 2 * t + (q & 1);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// Forward pass of one warp over 32 samples held one per lane.  f0, f1: this
// lane's features.  W: bf16 parameters (shared or global memory), bufA and
// bufB: per-warp scratch of 32 x 64 bf16 each.  Returns this lane's output.
__device__ __forceinline__ float mlp_forward_warp(float f0, float f1, const __nv_bfloat16 *W, __nv_bfloat16 *bufA,
                                                  __nv_bfloat16 *bufB) {
    const int lane = threadIdx.x & 31;
    for (int o = 0; o < MLP_H; ++o) {
        const float z = __bfloat162float(W[MLP_W1 + 2 * o]) * f0 + __bfloat162float(W[MLP_W1 + 2 * o + 1]) * f1 +
                        __bfloat162float(W[MLP_B1 + o]);
        bufA[lane * MLP_H + o] = __float2bfloat16_rn(silu_f(z));
    }
    __syncwarp();
    __nv_bfloat16 *in = bufA, *out = bufB;
    for (int layer = 0; layer < 2; ++layer) {
        const __nv_bfloat16 *Wl = W + (layer == 0 ? MLP_W2 : MLP_W3);
        const __nv_bfloat16 *bl = W + (layer == 0 ? MLP_B2 : MLP_B3);
        auto a = [&](int i, int k) { return in[i * MLP_H + k]; };
        auto b = [&](int k, int j) { return Wl[j * MLP_H + k]; };     // (H W^T)(i, j)
        for (int mt = 0; mt < 2; ++mt)
            for (int nt = 0; nt < 8; ++nt) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_tile(mt * 16, nt * 8, MLP_H, a, b, c);
                for (int q = 0; q < 4; ++q) {
                    int r, col;
                    tile_coords(mt * 16, nt * 8, q, r, col);
                    out[r * MLP_H + col] = __float2bfloat16_rn(silu_f(c[q] + __bfloat162float(bl[col])));
                }
            }
        __syncwarp();
        __nv_bfloat16 *tmp = in;
        in = out;
        out = tmp;
    }
    float y = __bfloat162float(W[MLP_B4]);
    for (int i = 0; i < MLP_H; ++i) y += __bfloat162float(W[MLP_W4 + i]) * __bfloat162float(in[lane * MLP_H + i]);
    __syncwarp();
    return y;
}

}  // namespace sfq
