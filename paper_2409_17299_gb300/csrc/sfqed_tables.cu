// K1: build the rate approximant and the inverse-CDF tables on the device.
//
// arXiv:2409.17299 Sec. 3: event rates come from polynomial approximations of
// precomputed rates and photon / pair energies from precomputed tables of the
// inverse cumulative probability over (chi, energy).  The underlying
// probabilities are the quasi-classical (LCFA) ones:
//   emission  dW/dd ~ ((1-d) + 1/(1-d)) K_{2/3}(y) - int_y^inf K_{1/3},  y = 2d/(3 chi (1-d))
//   pair      dW/dd ~ (d/(1-d) + (1-d)/d) K_{2/3}(y) + int_y^inf K_{1/3},  y = 2/(3 chi d (1-d))
// Both are integrated on the whole line in z (emission y = e^z; pair
// d = 1/(1+e^-z)) with composite 16-point Gauss-Legendre panels.
#include <math.h>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"

namespace sfq {
namespace {

constexpr int GLN = 16;
constexpr double PI = 3.14159265358979323846;

// emission: z in [-110, 8] (below: analytic tail C e^{z/3}); pair: z in [-38, 0]
constexpr double EZ_LO = -110.0, EZ_W = 0.25;
constexpr int EZ_NP = 472;
constexpr double PZ_LO = -38.0, PZ_W = 0.1;
constexpr int PZ_NP = 380;

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
__global__ void k_gauss_legendre(double *gl) {
    const int i = threadIdx.x;
    if (i >= GLN) return;
    double x = cos(PI * (i + 0.75) / (GLN + 0.5));
    double pn = 0, pn1 = 0;
    for (int it = 0; it < 60; ++it) {
        double a = 1.0, b = x;
        for (int k = 2; k <= GLN; ++k) {
            const double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
            a = b;
            b = c;
        }
        pn = b;
        pn1 = a;
        const double dp = GLN * (x * pn - pn1) / (x * x - 1.0);
        const double dx = pn / dp;
        x -= dx;
        if (fabs(dx) < 1e-17) break;
    }
    double a = 1.0, b = x;
    for (int k = 2; k <= GLN; ++k) {
        const double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    const double dp = GLN * (x * b - a) / (x * x - 1.0);
    gl[i] = x;
    gl[GLN + i] = 2.0 / ((1.0 - x * x) * dp * dp);
}

// Modified Bessel function of the second kind and int_y^inf K_{1/3}.
//   y < 1 : ascending series, K_nu = pi/(2 sin(nu pi)) (I_{-nu} - I_nu)
//   y >= 1: trapezoid rule on K_nu(y) = int_0^inf e^{-y cosh t} cosh(nu t) dt
//           (and the same with 1/cosh t for the integral of K_{1/3})
__device__ double series_I(double mu, double y, bool integrated) {
    const double h = 0.5 * y, h2 = h * h;
    double term = pow(h, mu) / tgamma(mu + 1.0);
    double s = integrated ? term * y / (mu + 1.0) : term;
    for (int k = 1; k < 40; ++k) {
        term *= h2 / (k * (k + mu));
        const double add = integrated ? term * y / (2.0 * k + mu + 1.0) : term;
        s += add;
        if (fabs(add) < 1e-18 * fabs(s)) break;
    }
    return s;
}

__device__ double trap(double nu, double y, bool over_cosh) {
    if (y > 740.0) return 0.0;
    const double h = fmin(0.1, 0.4 * rsqrt(y));
    double s = 0.5 * exp(-y);
    for (int j = 1; j < 20000; ++j) {
        const double t = j * h, ch = cosh(t);
        double f = exp(-y * ch) * cosh(nu * t);
        if (over_cosh) f /= ch;
        s += f;
        if (y * ch > 1.0 && f <= 1e-18 * s) break;
    }
    return h * s;
}

__device__ double bessel_k(double nu, double y) {
    if (y < 1.0) return PI / (2.0 * sin(nu * PI)) * (series_I(-nu, y, false) - series_I(nu, y, false));
    return trap(nu, y, false);
}

__device__ double int_k13(double y) {
    if (y < 1.0) {
        const double c = PI / sqrt(3.0);   // int_0^inf K_{1/3} = pi/sqrt3 = pi/(2 sin(pi/3))
        return c * (1.0 - series_I(-1.0 / 3.0, y, true) + series_I(1.0 / 3.0, y, true));
    }
    return trap(1.0 / 3.0, y, true);
}

// emission integrand in z = ln y (bracket times d delta / dz)
__device__ double g_emission(double z, double chi) {
    const double y = exp(z);
    const double a = 3.0 * chi * y;
    const double om = 2.0 / (2.0 + a);                   // 1 - delta
    const double jac = y * 6.0 * chi / ((2.0 + a) * (2.0 + a));
    return ((om + 1.0 / om) * bessel_k(2.0 / 3.0, y) - int_k13(y)) * jac;
}

// pair integrand in z, delta = 1/(1+e^-z)
__device__ double g_pairs(double z, double chi) {
    const double d = 1.0 / (1.0 + exp(-z));
    const double om = 1.0 / (1.0 + exp(z));
    const double jac = d * om;
    const double y = 2.0 / (3.0 * chi * jac);
    return ((d / om + om / d) * bessel_k(2.0 / 3.0, y) + int_k13(y)) * jac;
}

__device__ double gl_panel(bool pair, double chi, double a, double b, const double *gl) {
    const double m = 0.5 * (a + b), hw = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < GLN; ++i) {
        const double z = m + hw * gl[i];
        s += gl[GLN + i] * (pair ? g_pairs(z, chi) : g_emission(z, chi));
    }
    return s * hw;
}

__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    __syncthreads();
    return s;
}

// Total rate at the Chebyshev nodes: block b = decade * 11 + node.
// Emission decades 0..5 on log10 chi in [-3, 3] store F/chi; pair decades
// 6..10 on [-2, 3] store ln F + 8/(3 chi).
__global__ void k_rate_nodes(const double *gl, double *fnode) {
    __shared__ double red[32];
    __shared__ double sgl[2 * GLN];
    if (threadIdx.x < 2 * GLN) sgl[threadIdx.x] = gl[threadIdx.x];
    __syncthreads();
    const int dec = blockIdx.x / CHEB_N, k = blockIdx.x % CHEB_N;
    const bool pair = dec >= EM_NDEC;
    const double lo = pair ? -2.0 + (dec - EM_NDEC) : -3.0 + dec;
    const double s = lo + 0.5 + 0.5 * cos(PI * (k + 0.5) / CHEB_N);
    const double chi = pow(10.0, s);
    double acc = 0.0;
    if (!pair) {
        for (int p = threadIdx.x; p < EZ_NP; p += blockDim.x)
            acc += gl_panel(false, chi, EZ_LO + p * EZ_W, EZ_LO + (p + 1) * EZ_W, sgl);
    } else {
        for (int p = threadIdx.x; p < PZ_NP; p += blockDim.x)
            acc += gl_panel(true, chi, PZ_LO + p * PZ_W, PZ_LO + (p + 1) * PZ_W, sgl);
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) {
        if (!pair) {
            const double F = (tot + 3.0 * g_emission(EZ_LO, chi)) / (sqrt(3.0) * PI);
            fnode[blockIdx.x] = F / chi;
        } else {
            const double F = 2.0 * tot / (sqrt(3.0) * PI);
            fnode[blockIdx.x] = log(F) + 8.0 / (3.0 * chi);
        }
    }
}

// Chebyshev coefficients from the node values (discrete cosine transform).
__global__ void k_cheb_coef(const double *fnode, double *coef64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NCOEF) return;
    const int dec = i / CHEB_N, j = i % CHEB_N;
    double s = 0.0;
    for (int k = 0; k < CHEB_N; ++k) s += fnode[dec * CHEB_N + k] * cos(PI * j * (k + 0.5) / CHEB_N);
    coef64[i] = 2.0 * s / CHEB_N;
}

// FP32 cubic pieces: piece i of a decade interpolates the FP64 Chebyshev form
// at t = 0, 1/3, 2/3, 1 (so neighbouring pieces meet), written as monomial
// coefficients in t from the forward differences.  Interpolation error below
// 1e-8 of the function; the FP32 evaluation rounds at ~3e-7.
__global__ void k_rate_segments(const double *coef64, float *seg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= EM_NSEG + PAIR_NSEG) return;
    const bool pair = i >= EM_NSEG;
    const int k = pair ? i - EM_NSEG : i;
    const int dec = k / RSEG, r = k % RSEG;
    const double *c = coef64 + (pair ? EM_NDEC * CHEB_N : 0) + dec * CHEB_N;
    double f[4];
    for (int q = 0; q < 4; ++q) {
        const double x = 2.0 * ((r + q / 3.0) / RSEG) - 1.0;    // Chebyshev variable of the decade
        double b1 = 0.0, b2 = 0.0;
        for (int j = CHEB_N - 1; j >= 1; --j) {
            const double b0 = c[j] + 2.0 * x * b1 - b2;
            b2 = b1;
            b1 = b0;
        }
        f[q] = 0.5 * c[0] + x * b1 - b2;
    }
    const double d1 = f[1] - f[0], d2 = f[2] - 2.0 * f[1] + f[0], d3 = f[3] - 3.0 * f[2] + 3.0 * f[1] - f[0];
    // p(t) = f0 + d1 tau + d2 tau (tau - 1)/2 + d3 tau (tau - 1)(tau - 2)/6, tau = 3 t
    seg[4 * i + 0] = (float)f[0];
    seg[4 * i + 1] = (float)(3.0 * (d1 - d2 / 2.0 + d3 / 3.0));
    seg[4 * i + 2] = (float)(9.0 * (d2 / 2.0 - d3 / 2.0));
    seg[4 * i + 3] = (float)(27.0 * (d3 / 6.0));
}

// Newton's method inside one panel [za, zb] for int_za^z g = target
// (from_top: int_z^zb g = target), bracketed by bisection.
__device__ double solve_panel(bool pair, double chi, double za, double zb, double target, bool from_top,
                              const double *gl) {
    double lo = za, hi = zb;
    const double whole = gl_panel(pair, chi, za, zb, gl);
    double f = whole > 0.0 ? fmin(fmax(target / whole, 0.0), 1.0) : 0.5;
    double z = from_top ? zb - f * (zb - za) : za + f * (zb - za);
    for (int it = 0; it < 100; ++it) {
        const double gz = pair ? g_pairs(z, chi) : g_emission(z, chi);
        double r, d;
        if (!from_top) { r = gl_panel(pair, chi, za, z, gl) - target; d = gz; }
        else { r = gl_panel(pair, chi, z, zb, gl) - target; d = -gz; }
        const bool z_high = from_top ? (r < 0.0) : (r > 0.0);
        if (z_high) hi = z; else lo = z;
        double zn = d != 0.0 ? z - r / d : 0.5 * (lo + hi);
        if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
        const double step = fabs(zn - z);
        z = zn;
        if (step <= 1e-15 * (1.0 + fabs(z)) || hi - lo <= 1e-15 * (1.0 + fabs(z))) break;
    }
    return z;
}

// One block per table row: rows 0..120 emission (ln y), 121..221 pair (ln delta).
__global__ void k_icdf_rows(const double *gl, double *em64, double *pair64) {
    __shared__ double sgl[2 * GLN];
    __shared__ double mass[EZ_NP];
    __shared__ double below[EZ_NP + 1];
    __shared__ double above[EZ_NP + 1];
    if (threadIdx.x < 2 * GLN) sgl[threadIdx.x] = gl[threadIdx.x];
    __syncthreads();
    const bool pair = blockIdx.x >= EM_NCHI;
    const int row = pair ? blockIdx.x - EM_NCHI : blockIdx.x;
    const double chi = pow(10.0, (pair ? -2.0 : -3.0) + row / 20.0);
    const int np = pair ? PZ_NP : EZ_NP;
    const double zlo = pair ? PZ_LO : EZ_LO, wp = pair ? PZ_W : EZ_W;
    for (int p = threadIdx.x; p < np; p += blockDim.x)
        mass[p] = gl_panel(pair, chi, zlo + p * wp, zlo + (p + 1) * wp, sgl);
    __syncthreads();
    const double tail = pair ? 0.0 : 3.0 * g_emission(EZ_LO, chi);
    if (threadIdx.x == 0) {
        below[0] = tail;
        for (int p = 0; p < np; ++p) below[p + 1] = below[p] + mass[p];
        above[np] = 0.0;
        for (int p = np - 1; p >= 0; --p) above[p] = above[p + 1] + mass[p];
    }
    __syncthreads();
    const double total = pair ? 2.0 * below[np] : below[np];
    const int ns = pair ? PAIR_NS : EM_NS;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        const double s = pair ? -16.0 + 16.0 * j / (PAIR_NS - 1) : -16.0 + 32.0 * j / (EM_NS - 1);
        const double u = 1.0 / (1.0 + exp(-s)), v = 1.0 / (1.0 + exp(s));
        double z;
        if (pair || u <= 0.5) {
            const double target = u * total;
            if (target <= tail) {
                z = zlo + 3.0 * log(target / tail);
            } else {
                int a = 0, b = np - 1;              // first panel with below[p+1] >= target
                while (a < b) {
                    const int m = (a + b) >> 1;
                    if (below[m + 1] < target) a = m + 1; else b = m;
                }
                z = solve_panel(pair, chi, zlo + a * wp, zlo + (a + 1) * wp, target - below[a], false, sgl);
            }
        } else {
            const double target = v * total;
            int a = 0, b = np - 1;                  // last panel with above[p] >= target
            while (a < b) {
                const int m = (a + b + 1) >> 1;
                if (above[m] >= target) a = m; else b = m - 1;
            }
            z = solve_panel(pair, chi, zlo + a * wp, zlo + (a + 1) * wp, target - above[a + 1], true, sgl);
        }
        if (pair) pair64[(size_t)row * PAIR_NS + j] = -log1p(exp(-z));
        else em64[(size_t)row * EM_NS + j] = z;
    }
}

__global__ void k_to_f32(const double *a, float *b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

}  // namespace
}  // namespace sfq

qed_status sfq_build_tables(qed_ctx *ctx) {
    using namespace sfq;
    cudaStream_t st = ctx->stream;
    double *fnode = nullptr;
    SFQ_CUDA(cudaMallocAsync(&fnode, sizeof(double) * NCOEF, st));
    k_gauss_legendre<<<1, 32, 0, st>>>(ctx->gl);
    k_rate_nodes<<<NCOEF, 128, 0, st>>>(ctx->gl, fnode);
    k_cheb_coef<<<1, 128, 0, st>>>(fnode, ctx->coef64);
    k_rate_segments<<<1, 256, 0, st>>>(ctx->coef64, ctx->coef32);
    k_icdf_rows<<<EM_NCHI + PAIR_NCHI, 128, 0, st>>>(ctx->gl, ctx->icdf_em64, ctx->icdf_pair64);
    k_to_f32<<<(EM_NCHI * EM_NS + 255) / 256, 256, 0, st>>>(ctx->icdf_em64, ctx->icdf_em32, EM_NCHI * EM_NS);
    k_to_f32<<<(PAIR_NCHI * PAIR_NS + 255) / 256, 256, 0, st>>>(ctx->icdf_pair64, ctx->icdf_pair32,
                                                                PAIR_NCHI * PAIR_NS);
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaFreeAsync(fnode, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    return QED_OK;
}
