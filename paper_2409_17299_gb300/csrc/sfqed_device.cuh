// Device building blocks of the QED step (arXiv:2409.17299, Sec. 3).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sfqed_internal.h"

namespace sfq {

// CODATA 2018, wavelength 0.8 um: R = m c^2 / (hbar omega).
constexpr double ALPHA = 7.2973525693e-3;
constexpr double RS = 329718.75885517005;
constexpr double PAIR_CHI_MIN = 0.01;   // pair rate taken as zero below
constexpr uint64_t CHILD_KEY_XOR = 0xC0FFEEull;

// ---------------------------------------------------------------------------
// Precision-generic math (T = double: FP64 mode; T = float: FP32 mode).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double m_exp(double a) { return exp(a); }
__device__ __forceinline__ float m_exp(float a) { return expf(a); }
__device__ __forceinline__ double m_log(double a) { return log(a); }
__device__ __forceinline__ float m_log(float a) { return logf(a); }
__device__ __forceinline__ double m_log1p(double a) { return log1p(a); }
__device__ __forceinline__ float m_log1p(float a) { return log1pf(a); }
__device__ __forceinline__ double m_log10(double a) { return log10(a); }
__device__ __forceinline__ float m_log10(float a) { return log10f(a); }
__device__ __forceinline__ double m_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float m_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double m_floor(double a) { return floor(a); }
__device__ __forceinline__ float m_floor(float a) { return floorf(a); }
__device__ __forceinline__ double m_cbrt2(double a) { double c = cbrt(a); return c * c; }  // a^(2/3)
__device__ __forceinline__ float m_cbrt2(float a) { float c = cbrtf(a); return c * c; }
__device__ __forceinline__ void m_sincos(double a, double *s, double *c) { sincos(a, s, c); }
__device__ __forceinline__ void m_sincos(float a, float *s, float *c) { sincosf(a, s, c); }
// Rate and waiting-time arithmetic: IEEE in FP64 mode; in FP32 mode the
// hardware approximations (a few ulp, far below the approximant's own 1e-6
// error and the statistics of the draws)
__device__ __forceinline__ double f_log10(double a) { return log10(a); }
__device__ __forceinline__ float f_log10(float a) { return __log10f(a); }
__device__ __forceinline__ double f_exp(double a) { return exp(a); }
__device__ __forceinline__ float f_exp(float a) { return __expf(a); }
__device__ __forceinline__ double f_div(double a, double b) { return a / b; }
__device__ __forceinline__ float f_div(float a, float b) { return __fdividef(a, b); }
// 1 / sqrt and sqrt: IEEE in FP64 mode; in FP32 mode from the hardware
// reciprocal square root (2 ulp), sqrt(v) = v / sqrt(v) with 0 kept exact
__device__ __forceinline__ double f_rsqrt(double a) { return 1.0 / sqrt(a); }
__device__ __forceinline__ float f_rsqrt(float a) { return rsqrtf(a); }
__device__ __forceinline__ double f_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float f_sqrt(float a) { return a > 0.f ? a * rsqrtf(a) : 0.f; }

// Per-thread asynchronous copies global -> shared (cp.async): a thread
// stages the next particle while it computes on the current one; the
// hardware wait (wait_group) needs no spinning.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// particle arrays are read and written by the same kernels: plain loads
template <class T> __device__ __forceinline__ T ld(const void *p, size_t i) {
    return reinterpret_cast<const T *>(p)[i];
}
template <class T> __device__ __forceinline__ void st(void *p, size_t i, T v) {
    reinterpret_cast<T *>(p)[i] = v;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): counter (c0..c3), key (k0, k1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product gives both halves
        const uint64_t m0 = (uint64_t)0xD2511F53u * c.x, m1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(m0 >> 32), lo0 = (uint32_t)m0;
        const uint32_t hi1 = (uint32_t)(m1 >> 32), lo1 = (uint32_t)m1;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// The key of round r is (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85).  Kernels
// that draw with one key for every particle take the ten round keys
// precomputed in their arguments, so each round's key is an operand read
// from the argument space rather than two additions per draw.
__host__ __device__ __forceinline__ PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k[2 * r] = k0;
        K.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = (uint64_t)0xD2511F53u * c.x, m1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(m1 >> 32) ^ c.y ^ K.k[2 * r], (uint32_t)m1,
                       (uint32_t)(m0 >> 32) ^ c.w ^ K.k[2 * r + 1], (uint32_t)m0);
    }
    return c;
}
__device__ __forceinline__ uint4 event_draw(const PhiloxKeys &K, uint64_t id, unsigned step, unsigned k) {
    return philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, k), K);
}

__device__ __forceinline__ uint4 event_draw(uint64_t seed, uint64_t id, unsigned step, unsigned k) {
    return philox4x32_10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, k),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Uniform draws from two Philox words (a, b): u = (m + 1/2) 2^-52 with
// m = a 2^20 + (b >> 12), in (0, 1) and never 0 or 1.  FP64 mode uses u
// itself and v = 1 - u (exact in double).  FP32 mode builds u and 1 - u
// separately from the bits, (m + 1/2) 2^-52 and (m' + 1/2) 2^-52 with
// m' = ~a 2^20 + (~b >> 12) = 2^52 - 1 - m, each to FP32 relative precision,
// so that log u and log(1 - u) stay accurate at both ends without FP64.
template <class T> struct Uniform;
template <> struct Uniform<double> {
    static __device__ __forceinline__ void draw(uint32_t a, uint32_t b, double &u, double &v) {
        const uint64_t m = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
        u = ((double)m + 0.5) * 0x1p-52;
        v = 1.0 - u;
    }
    static __device__ __forceinline__ double neglog(double u, double) { return -log(u); }
};
template <> struct Uniform<float> {
    static __device__ __forceinline__ void draw(uint32_t a, uint32_t b, float &u, float &v) {
        u = fmaf(__uint2float_rn(a), 0x1p-32f, fmaf(__uint2float_rn(b >> 12), 0x1p-52f, 0x1p-53f));
        v = fmaf(__uint2float_rn(~a), 0x1p-32f, fmaf(__uint2float_rn((~b) >> 12), 0x1p-52f, 0x1p-53f));
    }
    // -ln u.  Below 1/2 the hardware logarithm (within 3 ulp).  Above, from
    // v = 1 - u (held to full relative precision): -ln(1 - v) = 2 atanh(z)
    // with z = v / (2 - v) in (0, 1/3], summed as the odd series
    // 2 (z + z^3/3 + ... + z^13/13); the first omitted term is below 1e-8
    // of the sum.
    static __device__ __forceinline__ float neglog(float u, float v) {
        if (u < 0.5f) return -__logf(u);
        const float z = __fdividef(v, 2.0f - v), z2 = z * z;
        float t = 1.0f / 13.0f;
        t = fmaf(t, z2, 1.0f / 11.0f);
        t = fmaf(t, z2, 1.0f / 9.0f);
        t = fmaf(t, z2, 1.0f / 7.0f);
        t = fmaf(t, z2, 1.0f / 5.0f);
        t = fmaf(t, z2, 1.0f / 3.0f);
        t = fmaf(t, z2, 1.0f);
        return 2.0f * z * t;
    }
};

// ---------------------------------------------------------------------------
// Fields (analytic descriptors).  FP64 mode: phase t = t_n + tau, as given.
// FP32 mode: phase from t_n reduced modulo 2 pi plus tau.
// ---------------------------------------------------------------------------
// A: any argument block with field_kind, prm[6], prm_f[6], t_n (FP64 phase
// of the step start) and t_n_red_f (the same reduced mod 2 pi, FP32).
template <class T, class A> __device__ __forceinline__ T prm_of(const A &a, int i) {
    if constexpr (sizeof(T) == 8) return a.prm[i];
    else return a.prm_f[i];      // no double-to-float conversion in FP32 mode
}

// sine and cosine of the time phase at t_n + tau (shared by all particles
// evaluated at the same tau, e.g. every particle at the start of a step)
template <class T> struct Phase { T s, c; };
template <class T, class A> __device__ __forceinline__ Phase<T> time_phase(const A &a, double tau) {
    Phase<T> q{(T)0, (T)1};
    if (a.field_kind == QED_FIELD_UNIFORM) return q;
    if constexpr (sizeof(T) == 8) {
        m_sincos(a.t_n + tau, &q.s, &q.c);
    } else {
        // the phase reduced mod 2 pi plus the clock inside the step: an
        // argument in [0, 2 pi + dt], where the hardware sine and cosine are
        // within 1e-6 absolute
        __sincosf(a.t_n_red_f + (float)tau, &q.s, &q.c);
    }
    return q;
}

// Gridded field: trilinear interpolation on the periodic node grid (lerp
// a + f (b - a) as one fused multiply-add: in x along the four x-edges of
// the cell, then y, then z).  The scaled coordinate is rounded on its own
// (no contraction with the fraction), as in the oracle.
template <class T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }

template <class T>
__device__ __forceinline__ void grid_axis(T x, int n, T inv_h, int &i0, int &i1, T &f) {
    const T u = mul_rn<T>(x, inv_h);
    const T fl = floor(u);
    long long i = (long long)fl % n;
    if (i < 0) i += n;
    i0 = (int)i;
    i1 = i0 + 1 == n ? 0 : i0 + 1;
    f = u - fl;
}

// The kernels read the grid interleaved, eight values per node (the six
// components and two pads), so a node is one 32-byte (FP32) or three
// 16-byte (FP64) vector loads.
template <class T> __device__ __forceinline__ void load_node(const T *g, long long node, T v[6]);
template <> __device__ __forceinline__ void load_node<float>(const float *g, long long node, float v[6]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(g + 8 * node));
    const float2 b = __ldg(reinterpret_cast<const float2 *>(g + 8 * node + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y;
}
template <> __device__ __forceinline__ void load_node<double>(const double *g, long long node, double v[6]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(g + 8 * node));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(g + 8 * node + 2));
    const double2 c = __ldg(reinterpret_cast<const double2 *>(g + 8 * node + 4));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

// lerp in x along the cell edge at row (j, k), then into acc with weight fy
// (first edge of a y pair: acc = the x-lerp itself)
template <class T>
__device__ __forceinline__ void edge_x(const T *g, long long row, int i0, int i1, T fx, T out[6]) {
    T v0[6], v1[6];
    load_node<T>(g, row + i0, v0);
    load_node<T>(g, row + i1, v1);
#pragma unroll
    for (int c = 0; c < 6; ++c) out[c] = fma(fx, v1[c] - v0[c], v0[c]);
}

template <class T, class A>
__device__ __forceinline__ void eval_grid(const A &a, const T x[3], T E[3], T B[3]) {
    const int nx = a.gn[0], ny = a.gn[1], nz = a.gn[2];
    int i0, i1, j0, j1, k0, k1;
    T fx, fy, fz;
    if constexpr (sizeof(T) == 8) {
        grid_axis<T>(x[0], nx, a.ginv[0], i0, i1, fx);
        grid_axis<T>(x[1], ny, a.ginv[1], j0, j1, fy);
        grid_axis<T>(x[2], nz, a.ginv[2], k0, k1, fz);
    } else {
        grid_axis<T>(x[0], nx, a.ginv_f[0], i0, i1, fx);
        grid_axis<T>(x[1], ny, a.ginv_f[1], j0, j1, fy);
        grid_axis<T>(x[2], nz, a.ginv_f[2], k0, k1, fz);
    }
    const long long plane = (long long)nx * ny;
    const T *g = reinterpret_cast<const T *>(a.grid_il);
    T b0[6], e0[6], e1[6];
    edge_x<T>(g, k0 * plane + (long long)j0 * nx, i0, i1, fx, e0);
    edge_x<T>(g, k0 * plane + (long long)j1 * nx, i0, i1, fx, e1);
#pragma unroll
    for (int c = 0; c < 6; ++c) b0[c] = fma(fy, e1[c] - e0[c], e0[c]);
    edge_x<T>(g, k1 * plane + (long long)j0 * nx, i0, i1, fx, e0);
    edge_x<T>(g, k1 * plane + (long long)j1 * nx, i0, i1, fx, e1);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const T b1 = fma(fy, e1[c] - e0[c], e0[c]);
        const T v = fma(fz, b1 - b0[c], b0[c]);
        if (c < 3) E[c] = v;
        else B[c - 3] = v;
    }
}

template <class T, class A>
__device__ __forceinline__ void eval_field_at(const A &a, const T xv[3], const Phase<T> &q, T E[3], T B[3]) {
    const T x = xv[0];
    if (a.field_kind == QED_FIELD_UNIFORM) {
        E[0] = prm_of<T, A>(a, 0); E[1] = prm_of<T, A>(a, 1); E[2] = prm_of<T, A>(a, 2);
        B[0] = prm_of<T, A>(a, 3); B[1] = prm_of<T, A>(a, 4); B[2] = prm_of<T, A>(a, 5);
        return;
    }
    const T s = q.s, c = q.c;
    const T a0 = prm_of<T, A>(a, 0);
    if (a.field_kind == QED_FIELD_ROTATING_E) {
        E[0] = a0 * c; E[1] = a0 * s; E[2] = 0;
        B[0] = 0; B[1] = 0; B[2] = 0;
    } else {   // standing circularly polarised wave, E antinode at x = 0
        T sx, cx;
        m_sincos(x, &sx, &cx);
        const T e = a0 * cx, b = a0 * sx;
        E[0] = 0; E[1] = e * c; E[2] = e * s;
        B[0] = 0; B[1] = b * c; B[2] = b * s;
    }
}

template <class T, class A>
__device__ __forceinline__ void eval_field(const A &a, const T x[3], double tau, T E[3], T B[3]) {
    eval_field_at<T, A>(a, x, time_phase<T, A>(a, tau), E, B);
}

// ---------------------------------------------------------------------------
// chi = sqrt((e0 E + p x B)^2 - (p.E)^2) / R, always in FP64 (the difference
// cancels for particles moving with a wave).  e0 = gamma (lepton) or k0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double chi_fp64(double e0, double px, double py, double pz,
                                           double Ex, double Ey, double Ez,
                                           double Bx, double By, double Bz) {
    const double ux = fma(e0, Ex, fma(py, Bz, -pz * By));
    const double uy = fma(e0, Ey, fma(pz, Bx, -px * Bz));
    const double uz = fma(e0, Ez, fma(px, By, -py * Bx));
    const double pe = fma(px, Ex, fma(py, Ey, pz * Ez));
    double q = fma(ux, ux, fma(uy, uy, uz * uz)) - pe * pe;
    q = q > 0.0 ? q : 0.0;
    return sqrt(q) * (1.0 / RS);
}

// ---------------------------------------------------------------------------
// FP32-mode chi, FP64-accurate where it matters.  With e0^2 = 1 + p^2
// (lepton) or k^2 (photon), Lagrange's identity turns the cancelling form into
//   chi^2 R^2 = S + T,  S = [E^2] + |p x E|^2 + |p x B|^2  (>= 0, no cancellation),
//                       T = 2 e0 E.(p x B)
// so only T can cancel S.  Cross products use Kahan's difference of products
// (error about one ulp of the result).  When the magnitude of the terms,
// S + 2 e0 sum|E_i (p x B)_i|, exceeds four times S + T the cancellation is
// real and the direct form is evaluated in FP64 instead.  Returns chi.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    // a*b - c*d
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

// zero: 1 if B = 0 everywhere (then chi^2 R^2 = [E^2] + |p x E|^2, a sum of
// squares), 2 if E = 0 everywhere (chi^2 R^2 = |p x B|^2), 3 if E and B are
// parallel everywhere (T = 2 e0 E.(p x B) = 2 e0 p.(B x E) = 0, so
// chi^2 R^2 = S, again a sum of squares), else 0.
template <bool LEPTON>
__device__ __forceinline__ float chi_guarded(float e0, const float p[3], const float E[3], const float B[3],
                                             unsigned *fp64_used, int zero = 0) {
    if (zero == 3) {
        const float ax = diff_of_products(p[1], E[2], p[2], E[1]);
        const float ay = diff_of_products(p[2], E[0], p[0], E[2]);
        const float az = diff_of_products(p[0], E[1], p[1], E[0]);
        const float bx = diff_of_products(p[1], B[2], p[2], B[1]);
        const float by = diff_of_products(p[2], B[0], p[0], B[2]);
        const float bz = diff_of_products(p[0], B[1], p[1], B[0]);
        float S = ax * ax + ay * ay + az * az + bx * bx + by * by + bz * bz;
        if (LEPTON) S += E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
        return f_sqrt(S) * (float)(1.0 / RS);
    }
    if (zero == 1) {
        const float ax = diff_of_products(p[1], E[2], p[2], E[1]);
        const float ay = diff_of_products(p[2], E[0], p[0], E[2]);
        const float az = diff_of_products(p[0], E[1], p[1], E[0]);
        float S = ax * ax + ay * ay + az * az;
        if (LEPTON) S += E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
        return f_sqrt(S) * (float)(1.0 / RS);
    }
    if (zero == 2) {
        const float bx = diff_of_products(p[1], B[2], p[2], B[1]);
        const float by = diff_of_products(p[2], B[0], p[0], B[2]);
        const float bz = diff_of_products(p[0], B[1], p[1], B[0]);
        return f_sqrt(bx * bx + by * by + bz * bz) * (float)(1.0 / RS);
    }
    const float ax = diff_of_products(p[1], E[2], p[2], E[1]);
    const float ay = diff_of_products(p[2], E[0], p[0], E[2]);
    const float az = diff_of_products(p[0], E[1], p[1], E[0]);
    const float bx = diff_of_products(p[1], B[2], p[2], B[1]);
    const float by = diff_of_products(p[2], B[0], p[0], B[2]);
    const float bz = diff_of_products(p[0], B[1], p[1], B[0]);
    float S = ax * ax + ay * ay + az * az + bx * bx + by * by + bz * bz;
    if (LEPTON) S += E[0] * E[0] + E[1] * E[1] + E[2] * E[2];
    const float te = 2.0f * e0;
    const float T = te * (E[0] * bx + E[1] * by + E[2] * bz);
    const float M = S + te * (fabsf(E[0] * bx) + fabsf(E[1] * by) + fabsf(E[2] * bz));
    const float r = S + T;
    if (M <= 4.0f * r) return f_sqrt(r) * (float)(1.0 / RS);
    ++*fp64_used;
    const double pd0 = p[0], pd1 = p[1], pd2 = p[2];
    const double e0d = LEPTON ? sqrt(1.0 + (pd0 * pd0 + pd1 * pd1 + pd2 * pd2)) : sqrt(pd0 * pd0 + pd1 * pd1 + pd2 * pd2);
    return (float)chi_fp64(e0d, pd0, pd1, pd2, E[0], E[1], E[2], B[0], B[1], B[2]);
}

// chi of a lepton (also gamma and p^2) or a photon in the mode's precision
template <class T>
__device__ __forceinline__ void lepton_chi(const T p[3], const T E[3], const T B[3], T &gam, T &chi, T &p2,
                                           unsigned &n64, int zero = 0) {
    if constexpr (sizeof(T) == 8) {
        p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        gam = sqrt(1.0 + p2);
        chi = chi_fp64(gam, p[0], p[1], p[2], E[0], E[1], E[2], B[0], B[1], B[2]);
    } else {
        p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        gam = f_sqrt(1.0f + p2);
        chi = chi_guarded<true>(gam, p, E, B, &n64, zero);
    }
}

template <class T>
__device__ __forceinline__ T photon_chi(T k0, const T k[3], const T E[3], const T B[3], unsigned &n64, int zero = 0) {
    if constexpr (sizeof(T) == 8) return chi_fp64(k0, k[0], k[1], k[2], E[0], E[1], E[2], B[0], B[1], B[2]);
    else return chi_guarded<false>(k0, k, E, B, &n64, zero);
}

// ---------------------------------------------------------------------------
// FP32 position update.  Rounding x + dx to the nearest float loses every
// displacement below half an ulp of x (an ulp is 2.4e-7 at |x| ~ pi) and
// biases those of a few ulp: a slow lepton at an electric antinode away from
// the origin would stop moving in x, stay in the strongest field and radiate
// there, which the FP64 arithmetic does not do (over 20 wave periods of the
// standing-wave cascade such leptons piled up at x = +-pi and raised the
// growth rate by ~3%).  Displacements of at least 2^-16 |x| take the plain
// sum (rounding changes them by at most 2^-7 of themselves); smaller ones are
// rounded stochastically to one of the two neighbouring floats, with the
// probabilities that make the expected result x + dx exact (the rounding
// error from TwoSum, written with explicitly rounded operations so that no
// step is contracted).  The random bits come from (id, step, k, coordinate).
__device__ __forceinline__ uint32_t round_bits(unsigned long long id, unsigned step, unsigned k) {
    // a lowbias32-style integer finaliser (xor-shifts and odd multipliers)
    uint32_t h = (uint32_t)id ^ ((uint32_t)(id >> 32) * 0x9E3779B1u) ^ (step * 0x85EBCA77u) ^ (k * 0xC2B2AE3Du);
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ float add_sr(float x, float dx, unsigned long long id, unsigned step, unsigned k) {
    const float s = __fadd_rn(x, dx);
    if (!(fabsf(dx) < __fmul_rn(fabsf(x), 0x1p-16f))) return s;
    const float bp = __fsub_rn(s, x);
    const float err = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bp)), __fsub_rn(dx, bp));   // x + dx - s exactly
    if (err == 0.f || s == 0.f) return s;
    const int bits = __float_as_int(s);
    const float nb = __int_as_float(bits + (((err > 0.f) == (s > 0.f)) ? 1 : -1));   // neighbour on err's side
    const float gap = fabsf(__fsub_rn(nb, s));
    const uint32_t r = round_bits(id, step, k);
    return __fmul_rn((float)(r >> 8) * 0x1p-24f, gap) < fabsf(err) ? nb : s;
}

// ---------------------------------------------------------------------------
// Boris push: half electric kick, magnetic rotation, half kick, then
// x += p/gamma h with the new momentum (FP32: add_sr, keyed by the particle's
// id, the step and its iteration k).  q = -1 (e-) or +1 (e+).  no_b: B = 0
// wherever the field is evaluated (the rotation is the identity and is
// skipped).  FP32 mode takes 1/gamma from the hardware reciprocal square root
// and the rotation factor from the fast division.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void boris(T x[3], T p[3], T q, const T E[3], const T B[3], T h, bool no_b,
                                      unsigned long long id, unsigned step, unsigned k) {
    const T qh2 = (T)0.5 * q * h;
    T m0 = p[0] + qh2 * E[0], m1 = p[1] + qh2 * E[1], m2 = p[2] + qh2 * E[2];
    if (!no_b) {
        const T ig = f_rsqrt((T)1 + m0 * m0 + m1 * m1 + m2 * m2);
        const T t0 = qh2 * B[0] * ig, t1 = qh2 * B[1] * ig, t2 = qh2 * B[2] * ig;
        const T f = f_div((T)2, (T)1 + t0 * t0 + t1 * t1 + t2 * t2);
        const T s0 = f * t0, s1 = f * t1, s2 = f * t2;
        const T a0 = m0 + (m1 * t2 - m2 * t1);
        const T a1 = m1 + (m2 * t0 - m0 * t2);
        const T a2 = m2 + (m0 * t1 - m1 * t0);
        m0 += a1 * s2 - a2 * s1;
        m1 += a2 * s0 - a0 * s2;
        m2 += a0 * s1 - a1 * s0;
    }
    p[0] = m0 + qh2 * E[0];
    p[1] = m1 + qh2 * E[1];
    p[2] = m2 + qh2 * E[2];
    if constexpr (sizeof(T) == 8) {
        const double vh = h / sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        x[0] += p[0] * vh;
        x[1] += p[1] * vh;
        x[2] += p[2] * vh;
    } else {
        const float vh = h * rsqrtf(1.0f + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        x[0] = add_sr(x[0], __fmul_rn(p[0], vh), id, step, 3u * k);
        x[1] = add_sr(x[1], __fmul_rn(p[1], vh), id, step, 3u * k + 1u);
        x[2] = add_sr(x[2], __fmul_rn(p[2], vh), id, step, 3u * k + 2u);
    }
}

// ---------------------------------------------------------------------------
// Rate approximant (Sec. 3, Sec. 4.3: polynomial approximation with a fixed
// operation count).  Coefficient layout: 6 emission decades [-3..3] then 5
// pair decades [-2..3], 11 Chebyshev coefficients each (first term halved).
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T clenshaw(const T *c, T x) {
    T b1 = 0, b2 = 0;
    const T x2 = x + x;
#pragma unroll
    for (int j = CHEB_N - 1; j >= 1; --j) {
        const T b0 = c[j] + x2 * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return (T)0.5 * c[0] + x * b1 - b2;
}

// F_gamma(chi)
template <class T> __device__ __forceinline__ T rate_em(const T *coef, T chi) {
    if (!(chi > (T)0)) return (T)0;
    const T s = f_log10(chi);
    if (s < (T)-3) return chi * clenshaw(coef, (T)-1);
    if (s > (T)3) return (T)1e3 * clenshaw(coef + 5 * CHEB_N, (T)1) * m_cbrt2(chi * (T)1e-3);
    int d = (int)m_floor(s + (T)3);
    d = d > 5 ? 5 : d;
    const T x = (T)2 * (s - (T)(d - 3)) - (T)1;
    return chi * clenshaw(coef + d * CHEB_N, x);
}

// F_pair(chi)
template <class T> __device__ __forceinline__ T rate_pair(const T *coef, T chi) {
    if (!(chi >= (T)PAIR_CHI_MIN)) return (T)0;
    const T *c = coef + EM_NDEC * CHEB_N;
    const T s = f_log10(chi);
    if (s > (T)3) return f_exp(clenshaw(c + 4 * CHEB_N, (T)1) - (T)(8.0 / 3e3)) * m_cbrt2(chi * (T)1e-3);
    int d = (int)m_floor(s + (T)2);
    d = d > 4 ? 4 : (d < 0 ? 0 : d);
    const T x = (T)2 * (s - (T)(d - 2)) - (T)1;
    return f_exp(clenshaw(c + d * CHEB_N, x) - f_div((T)(8.0 / 3.0), chi));
}

// FP32: the cubic pieces (tab: EM_NSEG then PAIR_NSEG float4 pieces, 16-byte
// aligned).  Outside [1e-3, 1e3] the same limit forms as above, from the end
// values of the first and last pieces.  Every operation is rounded
// explicitly, so each inlined copy computes the same bits whatever the
// compiler fuses around it.
constexpr float PIECES_PER_LOG2 = (float)(RSEG * 0.30102999566398119521);   // RSEG log10(2)

__device__ __forceinline__ float piece_eval(const float *tab, int i, float t) {
    const float4 c = reinterpret_cast<const float4 *>(tab)[i];
    return __fmaf_rn(t, __fmaf_rn(t, __fmaf_rn(t, c.w, c.z), c.y), c.x);
}

// piece coordinate RSEG (log10 chi - s0)
__device__ __forceinline__ float piece_coord(float chi, int s0_times_rseg) {
    return __fmaf_rn(__log2f(chi), PIECES_PER_LOG2, (float)s0_times_rseg);
}

template <> __device__ __forceinline__ float rate_em<float>(const float *tab, float chi) {
    if (!(chi > 0.f)) return 0.f;
    const float u = piece_coord(chi, 3 * RSEG);
    if (u < 0.f) return __fmul_rn(chi, tab[0]);
    if (u >= (float)EM_NSEG) return 1e3f * piece_eval(tab, EM_NSEG - 1, 1.f) * m_cbrt2(chi * 1e-3f);
    const int i = (int)u;
    return __fmul_rn(chi, piece_eval(tab, i, __fsub_rn(u, (float)i)));
}

template <> __device__ __forceinline__ float rate_pair<float>(const float *tab, float chi) {
    if (!(chi >= (float)PAIR_CHI_MIN)) return 0.f;
    const float *c = tab + 4 * EM_NSEG;
    const float u = piece_coord(chi, 2 * RSEG);
    if (u >= (float)PAIR_NSEG)
        return f_exp(piece_eval(c, PAIR_NSEG - 1, 1.f) - (float)(8.0 / 3e3)) * m_cbrt2(chi * 1e-3f);
    const int i = u > 0.f ? (int)u : 0;      // chi = 0.01 may land a rounding below the first piece
    return f_exp(__fsub_rn(piece_eval(c, i, __fsub_rn(u, (float)i)), f_div(8.0f / 3.0f, chi)));
}

// ---------------------------------------------------------------------------
// Inverse-CDF sampling (Sec. 3).  Bilinear in (log10 chi, logit u); chi is
// clamped to the table, logit u extrapolated linearly from the end cells.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T bilinear(const T *tab, int nchi, int ns, T c, T t) {
    c = c < (T)0 ? (T)0 : (c > (T)(nchi - 1) ? (T)(nchi - 1) : c);
    int i0 = (int)m_floor(c);
    i0 = i0 > nchi - 2 ? nchi - 2 : i0;
    const T fc = c - (T)i0;
    int j0 = (int)m_floor(t);
    j0 = j0 < 0 ? 0 : (j0 > ns - 2 ? ns - 2 : j0);
    const T ft = t - (T)j0;
    const T *r0 = tab + (size_t)i0 * ns + j0;
    const T *r1 = r0 + ns;
    const T a = __ldg(r0), b = __ldg(r0 + 1), cc = __ldg(r1), d = __ldg(r1 + 1);
    const T lo = a + ft * (b - a), hi = cc + ft * (d - cc);
    return lo + fc * (hi - lo);
}

// logit u = ln u - ln(1 - u) from (u, v = 1 - u); FP32: hardware logarithms
// (u and v each hold full relative precision, and the table coordinate needs
// about 1e-5 absolute)
__device__ __forceinline__ double logit(double u, double) { return log(u) - log1p(-u); }
__device__ __forceinline__ float logit(float u, float v) { return __logf(u) - __logf(v); }
// log10 chi and exp of the table value: IEEE in FP64 mode, hardware in FP32
__device__ __forceinline__ double s_log10(double a) { return log10(a); }
__device__ __forceinline__ float s_log10(float a) { return __log10f(a); }
__device__ __forceinline__ double s_exp(double a) { return exp(a); }
__device__ __forceinline__ float s_exp(float a) { return __expf(a); }

// photon energy fraction delta (returned) and 1 - delta
template <class T>
__device__ __forceinline__ T sample_emission(const T *tab, T chi, T u, T v, T *one_minus) {
    const T s = logit(u, v);
    const T c = (s_log10(chi) + (T)3) * (T)20;
    const T t = (s + (T)16) * (T)8;
    const T zeta = bilinear(tab, EM_NCHI, EM_NS, c, t);
    const T a = (T)3 * chi * s_exp(zeta);
    if constexpr (sizeof(T) == 8) {
        *one_minus = 2.0 / (2.0 + a);
        return a / (2.0 + a);
    } else {
        const float inv = __fdividef(1.0f, 2.0f + a);
        *one_minus = 2.0f * inv;
        return a * inv;
    }
}

// electron energy fraction delta (returned) and 1 - delta (positron fraction)
template <class T>
__device__ __forceinline__ T sample_pair(const T *tab, T chi, T u, T v, T *one_minus) {
    const bool flip = u > (T)0.5;
    const T s = flip ? logit(v, u) : logit(u, v);   // logit of min(u, 1 - u)
    const T c = (s_log10(chi) + (T)2) * (T)20;
    const T t = (s + (T)16) * (T)8;
    const T d = s_exp(bilinear(tab, PAIR_NCHI, PAIR_NS, c, t));
    if (flip) { *one_minus = d; return (T)1 - d; }
    *one_minus = (T)1 - d;
    return d;
}

// ---------------------------------------------------------------------------
// Warp-aggregated append: the lanes that want a slot get consecutive slots
// from one atomicAdd per converged group.  Returns the slot (may be beyond
// capacity; the caller checks).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *counter, unsigned n_each) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)(__popc(mask) * n_each));
    base = __shfl_sync(mask, base, leader);
    const unsigned below = __popc(mask & ((1u << lane) - 1u));
    return base + (unsigned long long)below * n_each;
}

}  // namespace sfq
