// K4 / K5: removal of dead particles and global leveling
// (arXiv:2409.17299 Sec. 4.2: the merge step is where filtering and thinning
// happen; Sec. 5.1: "global leveling" keeps the particle count bounded).
//
// Compaction is in place and deterministic: with A alive entries among
// [0, N), the r-th dead slot below A receives the r-th alive entry at or
// above A (ranks from block scans), so no entry is read after it is written.
//
// Leveling: the threshold w* solves sum_i min(1, w_i / w*) = cap (solved on
// the device, see k_lev_next).  Particle i is kept with probability
// min(1, w_i / w*) from Philox(seed; id, step, 0xFFFFFFFF), and kept
// particles below w* get weight w*.
#include <math.h>
#include <string.h>

#include <chrono>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"

namespace sfq {
namespace {

constexpr int CT = 256;            // threads per compaction block
constexpr int CITEMS = 4;          // items per thread
constexpr int CTILE = CT * CITEMS; // entries per block

template <class T> __device__ __forceinline__ bool alive_at(const void *w, unsigned long long i) {
    return ld<T>(w, i) > (T)0;
}

// exclusive scan of one value per thread over the block; returns the prefix,
// writes the block total
__device__ __forceinline__ unsigned block_scan(unsigned v, unsigned *sw, unsigned *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sw[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    const unsigned before = (wid > 0 ? sw[wid - 1] : 0u) + x - v;
    *total = sw[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

template <class T>
__global__ void __launch_bounds__(CT) k_count_alive(const void *w, const DevCtl *ctl, int s,
                                                    unsigned long long *blk) {
    const unsigned long long n = ctl->count[s];
    const unsigned long long base = (unsigned long long)blockIdx.x * CTILE;
    unsigned c = 0;
    for (int r = 0; r < CITEMS; ++r) {
        const unsigned long long i = base + r * CT + threadIdx.x;
        if (i < n && alive_at<T>(w, i)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ unsigned sw[32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int k = 0; k < CT / 32; ++k) t += sw[k];
        blk[blockIdx.x] = t;
    }
}

// single block: exclusive scan of the per-block counts, total -> alive[s]
__global__ void k_scan_blocks(unsigned long long *blk, long long nb, DevCtl *ctl, int s) {
    __shared__ unsigned long long sw[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long b0 = 0; b0 < nb; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? blk[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sw[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            sw[lane] = t;
        }
        __syncthreads();
        const unsigned long long before = carry + (wid > 0 ? sw[wid - 1] : 0ull) + x - v;
        if (i < nb) blk[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += sw[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctl->alive[s] = carry;
        ctl->holes[s] = 0;
    }
}

// dead slots below A record their rank (= number of dead entries before them)
// and are counted (H, the number of holes)
template <class T>
__global__ void __launch_bounds__(CT) k_mark_holes(const void *w, DevCtl *ctl, int s,
                                                   const unsigned long long *blk, unsigned long long *slots) {
    __shared__ unsigned sw[32];
    const unsigned long long n = ctl->count[s], A = ctl->alive[s];
    const unsigned long long base = (unsigned long long)blockIdx.x * CTILE;
    unsigned long long run = blk[blockIdx.x];
    unsigned my_holes = 0;
    for (int r = 0; r < CITEMS; ++r) {
        const unsigned long long i = base + r * CT + threadIdx.x;
        const bool al = i < n && alive_at<T>(w, i);
        unsigned tot;
        const unsigned before = block_scan(al ? 1u : 0u, sw, &tot);
        if (i < A && !al) {
            slots[i - (run + before)] = i;     // rank < A <= n (slots holds n entries)
            ++my_holes;
        }
        run += tot;
    }
    for (int o = 16; o > 0; o >>= 1) my_holes += __shfl_down_sync(0xffffffffu, my_holes, o);
    if ((threadIdx.x & 31) == 0 && my_holes) atomicAdd(&ctl->holes[s], (unsigned long long)my_holes);
}

template <class T> __device__ __forceinline__ void move_entry(const SpeciesDev &S, unsigned long long d,
                                                              unsigned long long i) {
    st<T>(S.x, d, ld<T>(S.x, i)); st<T>(S.y, d, ld<T>(S.y, i)); st<T>(S.z, d, ld<T>(S.z, i));
    st<T>(S.px, d, ld<T>(S.px, i)); st<T>(S.py, d, ld<T>(S.py, i)); st<T>(S.pz, d, ld<T>(S.pz, i));
    st<T>(S.w, d, ld<T>(S.w, i));
    S.id[d] = S.id[i];
    S.nev[d] = S.nev[i];
    if (S.od) st<T>(S.od, d, ld<T>(S.od, i));
}

// alive entries at or above A move into the holes, in rank order: the mover
// rank is the number of alive entries in [A, i) = alive_before(i) - (A - H)
template <class T>
__global__ void __launch_bounds__(CT) k_fill_holes(SpeciesDev S, DevCtl *ctl, int s, const unsigned long long *blk,
                                                   const unsigned long long *slots) {
    __shared__ unsigned sw[32];
    const unsigned long long n = ctl->count[s], A = ctl->alive[s], H = ctl->holes[s];
    const unsigned long long alive_below_A = A - H;
    const unsigned long long base = (unsigned long long)blockIdx.x * CTILE;
    if (base + CTILE <= A) return;                 // whole tile below A: nothing moves
    unsigned long long run = blk[blockIdx.x];
    for (int r = 0; r < CITEMS; ++r) {
        const unsigned long long i = base + r * CT + threadIdx.x;
        const bool al = i < n && alive_at<T>(S.w, i);
        unsigned tot;
        const unsigned before = block_scan(al ? 1u : 0u, sw, &tot);
        if (al && i >= A) {
            const unsigned long long ab = run + before;     // alive entries before i
            const unsigned long long rank = ab - alive_below_A;
            if (ab >= alive_below_A && rank < H) {
                const unsigned long long d = slots[rank];
                if (d < A) move_entry<T>(S, d, i);
                else atomicExch(&ctl->bad_index, i + 1);
            } else {
                atomicExch(&ctl->bad_index, i + 1);
            }
        }
        run += tot;
    }
}

// Entries a tile pass covers: the count (at most the capacity), none once a
// step ran out of capacity or a device check failed (the state is then left
// as it is for the caller's replay).
__device__ __forceinline__ unsigned long long tile_count(const DevCtl *ctl, int s) {
    if (ctl->overflow || ctl->timeout || ctl->bad_index) return 0;
    const unsigned long long c = ctl->count[s], cp = ctl->capacity[s];
    return c < cp ? c : cp;
}

__global__ void k_set_count(DevCtl *ctl, int s) {
    if (ctl->overflow || ctl->timeout || ctl->bad_index) return;
    ctl->count[s] = ctl->alive[s];
    ctl->end[s] = ctl->alive[s];
    ctl->begin[s] = ctl->alive[s];
}

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
constexpr unsigned long long INF_BITS = 0x7ff0000000000000ull;    // +inf as double bits

// ---- leveling: device-resident piecewise-exact Newton iteration ----
// S(w) = sum_i min(1, w_i / w) = A(w) / w + C(w) with A = sum of weights below
// w and C = count at or above w.  On the piece of w containing the root,
// S = A/w + C, whose root is A / (cap - C): evaluating (A, C) at w and jumping
// to A / (cap - C) lands on the root once the piece is right, otherwise it
// moves toward it; a bisection bracket keeps every step inside [lo, hi].
// Block partial sums are reduced in a fixed order (deterministic result).
constexpr int LEVEL_ITERS = 40;

// smallest float >= a positive double (v < d <=> v < ceil_f(d) for floats v)
__host__ __device__ __forceinline__ float ceil_f(double d) {
#ifdef __CUDA_ARCH__
    return __double2float_ru(d);
#else
    float f = (float)d;
    if ((double)f < d) f = nextafterf(f, INFINITY);
    return f;
#endif
}

__host__ __device__ __forceinline__ double double_of_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// Warm start: the first pass evaluates at the species' previous threshold
// (after a leveling most weights equal it, and the next root usually lies
// in the piece just above it), else at +inf.  The start changes only the
// path: the root of its own piece is the same from any start.
__device__ __forceinline__ void lev_start(LevelWork *lw, int s) {
    LevelIter &it = lw->it[s];
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const double w0 = lw->prev[s] > 0.0 && lw->prev[s] < inf ? lw->prev[s] : inf;
    it.lo = 0.0;
    it.hi = inf;
    it.w = w0;
    it.w_up = w0 < inf ? ceil_f(w0) : __int_as_float(0x7f800000);
    it.wstar = 0.0;
    it.wstar_inv_f = 0.f;
    it.done = 0;
    it.iters = 0;
    it.alive = 0;
    it.mode = 0;
    lw->arrive[s] = 0;
    lw->passes[s] = 0;
}

__global__ void k_lev_begin(LevelWork *lw, int s) { lev_start(lw, s); }

// error-free float-float accumulation (TwoSum), accurate to ~2^-48 relative
struct FF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float b) {
        const float t = hi + b;
        const float bp = t - hi;
        const float e = (hi - (t - bp)) + (b - bp);
        hi = t;
        lo += e;
    }
};

// double-double accumulation (TwoSum) for the reduction of block partials
struct DD {
    double hi = 0.0, lo = 0.0;
    __device__ __forceinline__ void add(double b) {
        const double t = hi + b;
        const double bp = t - hi;
        lo += (hi - (t - bp)) + (b - bp);
        hi = t;
    }
};

__host__ __device__ __forceinline__ void lev_finish(LevelIter &it, double wstar) {
    it.done = 1;
    it.wstar = wstar;
    it.wstar_up = wstar > 0.0 ? ceil_f(wstar) : 0.f;
    it.wstar_f = (float)wstar;
    it.wstar_inv_f = wstar > 0.0 ? (float)(1.0 / wstar) : 0.f;
}

// Newton step from the sums at it.w: A (weights below w), C (count at or
// above w), N (alive count), M (largest weight, double bits).  PL and PH
// (double bits; PH = 0: not given) bound the piece of w: the largest weight
// below w and the smallest at or above it.  A Newton point c with
// PL < c <= PH lies on w's piece, where A and C are those just summed, so the
// next pass would return c itself and finish there: the iteration finishes at
// c now, with the same result and one pass fewer.
__host__ __device__ void lev_advance(LevelIter &it, double A, unsigned long long C, unsigned long long N,
                                     unsigned long long M, long long cap, unsigned long long PL = 0,
                                     unsigned long long PH = 0) {
    const double inf = double_of_bits(0x7ff0000000000000ull);
    const double w = it.w;
    if (it.iters == 0) {                           // first pass: at +inf or at a warm start w
        it.alive = N;
        if (N <= (unsigned long long)cap) { lev_finish(it, 0.0); return; }
        it.hi = double_of_bits(M) * (double)N / (double)cap;                    // S(hi) <= cap
        it.lo = 0.0;
        if (w < inf) {
            const double S = A / w + (double)C;
            if (S > (double)cap) it.lo = w;
            else if (w < it.hi) it.hi = w;
        }
    } else {
        const double S = A / w + (double)C;
        if (S > (double)cap) it.lo = w; else it.hi = w;
    }
    ++it.iters;
    double c = (double)cap > (double)C ? A / ((double)cap - (double)C) : inf;
    if (c == w) { lev_finish(it, w); return; }     // root of its own piece
    const bool newton = c > it.lo && c <= it.hi;
    if (!newton) c = 0.5 * (it.lo + it.hi);
    // stop at double resolution of the bracket (hi, evaluated, is the answer)
    if (!(c > it.lo && c <= it.hi) || (c == it.hi && it.hi == w) || it.iters >= LEVEL_ITERS) {
        lev_finish(it, it.hi);
        return;
    }
    if (newton && PH != 0 && c > double_of_bits(PL) && c <= double_of_bits(PH)) {
        lev_finish(it, c);
        return;
    }
    it.w = c;
    it.w_up = ceil_f(c);
}

// One pass of the iteration.  Every block sums its share of the weights at
// it.w; the last block to finish reduces the block partials in block order
// (a fixed order: the result does not depend on which block is last) and
// advances the iteration, so a pass is one launch and needs no host.
constexpr int LEV_T = 256;

// This thread's share of the sums at it.w over entries t0, t0 + stride, ...
template <class T>
__device__ __forceinline__ void lev_accumulate(const void *w, unsigned long long n, unsigned long long t0,
                                               unsigned long long stride, const LevelIter &it, double &A,
                                               unsigned long long &C, unsigned long long &N, unsigned long long &M,
                                               unsigned long long &L, unsigned long long &H) {
    C = 0;
    N = 0;
    M = 0;
    L = 0;
    H = INF_BITS;
    if constexpr (sizeof(T) == 4) {
        // FP32 weights: exact float comparisons and float-float sums, no FP64 per element
        const float wc = it.w_up;
        FF acc;
        unsigned mb = 0, c = 0, nn = 0, lb = 0, hb = 0x7f800000u;    // positive floats order like their bits
        auto one = [&](float v) {
            if (v > 0.f) {
                ++nn;
                mb = max(mb, __float_as_uint(v));
                if (v < wc) {
                    acc.add(v);
                    lb = max(lb, __float_as_uint(v));
                } else {
                    ++c;
                    hb = min(hb, __float_as_uint(v));
                }
            }
        };
        const float *wf = reinterpret_cast<const float *>(w);
        unsigned long long i0 = 0;
        if ((reinterpret_cast<uintptr_t>(wf) & 15u) == 0) {
            const float4 *w4 = reinterpret_cast<const float4 *>(wf);
            const unsigned long long n4 = n / 4;
            unsigned long long j = t0;
            for (; j + 3 * stride < n4; j += 4 * stride) {      // four 16-byte loads in flight
                const float4 a = __ldg(w4 + j), b = __ldg(w4 + j + stride);
                const float4 c4 = __ldg(w4 + j + 2 * stride), d = __ldg(w4 + j + 3 * stride);
                one(a.x); one(a.y); one(a.z); one(a.w);
                one(b.x); one(b.y); one(b.z); one(b.w);
                one(c4.x); one(c4.y); one(c4.z); one(c4.w);
                one(d.x); one(d.y); one(d.z); one(d.w);
            }
            for (; j < n4; j += stride) {
                const float4 a = __ldg(w4 + j);
                one(a.x); one(a.y); one(a.z); one(a.w);
            }
            i0 = n4 * 4;
        }
        for (unsigned long long i = i0 + t0; i < n; i += stride) one(wf[i]);
        A = (double)acc.hi + (double)acc.lo;
        C = c;
        N = nn;
        M = nn ? dbits((double)__uint_as_float(mb)) : 0ull;
        L = lb ? dbits((double)__uint_as_float(lb)) : 0ull;
        H = hb < 0x7f800000u ? dbits((double)__uint_as_float(hb)) : INF_BITS;
    } else {
        const double wc = it.w;
        double comp = 0.0;           // Kahan
        A = 0.0;
        for (unsigned long long i = t0; i < n; i += stride) {
            const double v = (double)ld<T>(w, i);
            if (!(v > 0.0)) continue;
            ++N;
            M = max(M, dbits(v));
            if (v < wc) {
                const double y = v - comp;
                const double t = A + y;
                comp = (t - A) - y;
                A = t;
                L = max(L, dbits(v));
            } else {
                ++C;
                H = min(H, dbits(v));
            }
        }
    }
}

// One pass of the iteration.  Every block sums its share of the weights at
// it.w; the last block to finish reduces the block partials in block order
// (a fixed order: the result does not depend on which block is last) and
// advances the iteration, so a pass is one launch and needs no host.
template <class T>
__global__ void __launch_bounds__(LEV_T) k_lev_step(const void *w, const DevCtl *ctl, int s, LevelWork *lw,
                                                    long long cap) {
    LevelIter &it = lw->it[s];
    if (*reinterpret_cast<volatile unsigned long long *>(&it.done)) return;
    const unsigned long long n = min(ctl->count[s], ctl->capacity[s]);
    const unsigned long long t0 = (unsigned long long)blockIdx.x * LEV_T + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * LEV_T;
    double A;
    unsigned long long C, N, M, L, H;
    lev_accumulate<T>(w, n, t0, stride, it, A, C, N, M, L, H);
    __shared__ double sA[LEV_T / 32];
    __shared__ unsigned long long sC[LEV_T / 32], sN[LEV_T / 32], sM[LEV_T / 32], sL[LEV_T / 32], sH[LEV_T / 32];
    __shared__ int s_last;
    for (int o = 16; o > 0; o >>= 1) {
        A += __shfl_down_sync(0xffffffffu, A, o);
        C += __shfl_down_sync(0xffffffffu, C, o);
        N += __shfl_down_sync(0xffffffffu, N, o);
        M = max(M, __shfl_down_sync(0xffffffffu, M, o));
        L = max(L, __shfl_down_sync(0xffffffffu, L, o));
        H = min(H, __shfl_down_sync(0xffffffffu, H, o));
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sA[wid] = A; sC[wid] = C; sN[wid] = N; sM[wid] = M; sL[wid] = L; sH[wid] = H; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        unsigned long long c = 0, nn = 0, m = 0, pl = 0, ph = INF_BITS;
        for (int k = 0; k < LEV_T / 32; ++k) {
            a += sA[k]; c += sC[k]; nn += sN[k]; m = max(m, sM[k]); pl = max(pl, sL[k]); ph = min(ph, sH[k]);
        }
        lw->partA[blockIdx.x] = a;
        lw->partC[blockIdx.x] = c;
        lw->partN[blockIdx.x] = nn;
        lw->partM[blockIdx.x] = m;
        lw->partL[blockIdx.x] = pl;
        lw->partH[blockIdx.x] = ph;
        __threadfence();
        const unsigned prev = atomicAdd(&lw->arrive[s], 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: partials b = t, t + LEV_T, ... per thread, then a tree of fixed shape
    __shared__ double rh[LEV_T], rl[LEV_T];
    __shared__ unsigned long long rc[LEV_T], rn[LEV_T], rm[LEV_T], rpl[LEV_T], rph[LEV_T];
    const int t = threadIdx.x;
    DD acc;
    unsigned long long c = 0, nn = 0, m = 0, pl = 0, ph = INF_BITS;
    for (int b = t; b < (int)gridDim.x; b += LEV_T) {
        acc.add(__ldcg(&lw->partA[b]));
        c += __ldcg(&lw->partC[b]);
        nn += __ldcg(&lw->partN[b]);
        m = max(m, __ldcg(&lw->partM[b]));
        pl = max(pl, __ldcg(&lw->partL[b]));
        ph = min(ph, __ldcg(&lw->partH[b]));
    }
    rh[t] = acc.hi; rl[t] = acc.lo; rc[t] = c; rn[t] = nn; rm[t] = m; rpl[t] = pl; rph[t] = ph;
    __syncthreads();
    for (int o = LEV_T / 2; o > 0; o >>= 1) {
        if (t < o) {
            DD x;
            x.hi = rh[t];
            x.lo = rl[t];
            x.add(rh[t + o]);
            x.lo += rl[t + o];
            rh[t] = x.hi;
            rl[t] = x.lo;
            rc[t] += rc[t + o];
            rn[t] += rn[t + o];
            rm[t] = max(rm[t], rm[t + o]);
            rpl[t] = max(rpl[t], rpl[t + o]);
            rph[t] = min(rph[t], rph[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        if (it.mode == 1) {         // sums only: the caller combines them across shards
            it.sumA = rh[0] + rl[0];
            it.sumC = rc[0];
            it.sumN = rn[0];
            it.sumM = rm[0];
        } else {
            lev_advance(it, rh[0] + rl[0], rc[0], rn[0], rm[0], cap, rpl[0], rph[0]);
            if (it.done && it.wstar > 0.0) lw->prev[s] = it.wstar;
        }
        lw->arrive[s] = 0;
    }
}

// Graph-driven leveling: after each pass, one thread decides whether the
// graph's while loop runs another (the only setter of the condition, so no
// two writes race).  The loop ends when the iteration is done, and in any
// case after LEVEL_ITERS + 1 passes (the iteration itself finishes by then).
__global__ void k_lev_cond(LevelWork *lw, int s, DevCtl *ctl, cudaGraphConditionalHandle h) {
    const LevelIter &it = lw->it[s];
    const unsigned long long n = ++lw->passes[s];
    ctl->graph_kernels += 2;                 // this pass: k_lev_step and this kernel
    cudaGraphSetConditional(h, (!it.done && n <= (unsigned long long)LEVEL_ITERS) ? 1u : 0u);
}

// ---- compaction by tiles (used after leveling and for converted photons) ----
// A tile of 4096 entries is one block of 256 threads; warp k owns entries
// [512 k, 512 k + 512) of the tile, 32 per round (coalesced).  Pass 1 lists
// the dead entries of each tile in index order (16-bit tile offsets) and
// counts the alive ones; a scan gives A (alive total) and H (dead entries
// below A); pass 2 lists the alive entries at or above A (the movers) by
// rank; pass 3 moves mover r into the r-th dead slot below A.
constexpr int LT = 256;
constexpr int LROUNDS = 16;
constexpr int LTILE = LT * LROUNDS;       // entries per tile (offsets fit 16 bits)
constexpr int LSPAN = 32 * LROUNDS;       // contiguous entries per warp

// Tiles holding entries of a species of n entries, and the tile grid: a
// kernel loops over tiles (grid stride), so its grid can be fixed by the
// species' capacity (a captured step graph) while the device count decides
// the work.
__device__ __forceinline__ long long tiles_of(unsigned long long n) { return (long long)((n + LTILE - 1) / LTILE); }

// Pass 1.  LEVEL: first keep particle i (0 < w_i < w*) with probability
// w_i / w*: the comparison u < w_i / w* is made in FP32 with a relative
// margin, and in FP64 (the oracle's test) only for draws within that margin
// of the boundary; kept particles get weight w*.  The step index keying the
// draws is `step`, or the control block's current step when step_from_ctl.
template <class T, bool LEVEL>
__global__ void __launch_bounds__(LT, 4) k_tile_dead(SpeciesDev S, DevCtl *ctl, int s, const LevelWork *lw,
                                                  const PhiloxKeys keys, unsigned step, int step_from_ctl,
                                                  unsigned long long *blk, unsigned short *dl) {
    __shared__ unsigned wdead[LT / 32];
    const unsigned long long n = tile_count(ctl, s);
    const long long nbe = tiles_of(n);
    if (step_from_ctl) step = ctl->sv_step;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bool thin = false;
    double wstar = 0.0;
    float inv_f = 0.f, wup = 0.f, wnew = 0.f;
    if constexpr (LEVEL) {
        const LevelIter &it = lw->it[s];
        wstar = it.wstar;
        thin = it.done && wstar > 0.0;
        inv_f = it.wstar_inv_f;
        wup = it.wstar_up;
        wnew = it.wstar_f;
    }
    unsigned removed = 0;
    // FP32 leveling: groups of four entries whose draws are computed together
    constexpr bool SPEC = LEVEL && sizeof(T) == 4;
    constexpr int G = SPEC ? 4 : 8;           // entries per group of loads
    static_assert(LROUNDS % G == 0, "groups tile the rounds");
    for (long long tile = blockIdx.x; tile < nbe; tile += gridDim.x) {
        const unsigned long long base = (unsigned long long)tile * LTILE;
        const unsigned long long wbase = base + (unsigned long long)wid * LSPAN;
        unsigned mask[LROUNDS];
        unsigned cnt = 0;
#pragma unroll
        for (int c0 = 0; c0 < LROUNDS; c0 += G) {
            // weights and (leveling) ids of G entries issued together: at
            // the cap nearly every entry is below w* and needs its id
            T v[G];
            unsigned long long idv[G];
#pragma unroll
            for (int r = 0; r < G; ++r) {
                const unsigned long long i = wbase + (c0 + r) * 32 + lane;
                v[r] = i < n ? ld<T>(S.w, i) : (T)0;
                idv[r] = (LEVEL && thin && i < n) ? S.id[i] : 0ull;
            }
            bool below[G];
#pragma unroll
            for (int r = 0; r < G; ++r) {
                if constexpr (sizeof(T) == 4) below[r] = LEVEL && thin && v[r] > (T)0 && (float)v[r] < wup;
                else below[r] = LEVEL && thin && v[r] > (T)0 && (double)v[r] < wstar;
            }
            // FP32 leveling: the G draws are computed together, outside the
            // per-entry branch, so their Philox rounds interleave (one draw
            // per branch ran the ten dependent rounds back to back); only the
            // entries below w* use theirs
            uint4 qv[G];
            if constexpr (SPEC) {
                if (thin) {
#pragma unroll
                    for (int r = 0; r < G; ++r) qv[r] = event_draw(keys, idv[r], step, 0xFFFFFFFFu);
                }
            }
#pragma unroll
            for (int r = 0; r < G; ++r) {
                const unsigned long long i = wbase + (c0 + r) * 32 + lane;
                bool dead = i < n && !(v[r] > (T)0);
                if (LEVEL && below[r]) {
                    const uint4 q = SPEC ? qv[r] : event_draw(keys, idv[r], step, 0xFFFFFFFFu);
                    const float uf = __uint2float_rn(q.x) * 0x1p-32f;     // u to within 2^-32 + FP32 rounding
                    const float pf = (float)v[r] * inv_f;
                    bool keep;
                    if (uf < pf * (1.0f - 1e-6f) - 0x1p-31f) keep = true;
                    else if (uf > pf * (1.0f + 1e-6f) + 0x1p-31f) keep = false;
                    else {
                        double u, vv;
                        Uniform<double>::draw(q.x, q.y, u, vv);
                        keep = u < (double)v[r] / wstar;
                    }
                    if (keep) {
                        if constexpr (sizeof(T) == 4) st<T>(S.w, i, wnew);
                        else st<T>(S.w, i, wstar);
                    } else {
                        st<T>(S.w, i, (T)0);
                        dead = true;
                        ++removed;
                    }
                }
                mask[c0 + r] = __ballot_sync(0xffffffffu, dead);
                cnt += __popc(mask[c0 + r]);
            }
        }
        if (lane == 0) wdead[wid] = cnt;
        __syncthreads();
        unsigned before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < LT / 32; ++k) {
            const unsigned c = wdead[k];
            before += k < wid ? c : 0u;
            total += c;
        }
        unsigned short *tdl = dl + base;
        const unsigned lt = (1u << lane) - 1u;
        unsigned run = before;
#pragma unroll
        for (int r = 0; r < LROUNDS; ++r) {
            if ((mask[r] >> lane) & 1u) tdl[run + __popc(mask[r] & lt)] = (unsigned short)(wid * LSPAN + r * 32 + lane);
            run += __popc(mask[r]);
        }
        if (threadIdx.x == 0) {
            const unsigned long long tn = n - base < (unsigned long long)LTILE ? n - base : (unsigned long long)LTILE;
            blk[tile] = tn - total;
        }
        __syncthreads();                       // wdead is rewritten by the next tile
    }
    if constexpr (LEVEL) {
        for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
        if (lane == 0 && removed) atomicAdd(&ctl->thinned, (unsigned long long)removed);
    }
}

// single block: exclusive scan of the counts of the tiles holding entries
// (blk[nbe] = A), then H from the alive entries of the tile that holds A.
// may_defer: while dead entries are at most DEFER_DEN-th of the species and
// the count leaves a fifth of the capacity free, the move is deferred (H = 0,
// the count stays): the dead entries (weight 0) are skipped by every pass
// until a later step compacts, with holes denser and fewer moves per step.
constexpr unsigned long long DEFER_DEN = 4;

template <class T>
__global__ void k_scan_tiles(const void *w, unsigned long long *blk, long long nb, DevCtl *ctl, int s,
                             int may_defer) {
    __shared__ unsigned long long sw[32];
    __shared__ unsigned long long carry;
    const long long nbe_all = tiles_of(tile_count(ctl, s));
    const long long nbe = nbe_all < nb ? nbe_all : nb;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long b0 = 0; b0 < nbe; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const unsigned long long v = i < nbe ? blk[i] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sw[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long t = lane < nw ? sw[lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            sw[lane] = t;
        }
        __syncthreads();
        const unsigned long long before = carry + (wid > 0 ? sw[wid - 1] : 0ull) + x - v;
        if (i < nbe) blk[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry += sw[nw - 1];
        __syncthreads();
    }
    const unsigned long long A = carry;
    const unsigned long long a = A / LTILE;
    unsigned long long below = A;                   // A on a tile boundary past the data: no holes
    if ((long long)a < nbe) {
        unsigned c = 0;
        for (unsigned long long i = a * LTILE + threadIdx.x; i < A; i += blockDim.x) c += alive_at<T>(w, i) ? 1u : 0u;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        __syncthreads();
        if (lane == 0) sw[wid] = c;
        __syncthreads();
        unsigned long long tc = 0;
        for (int k = 0; k < nw; ++k) tc += sw[k];
        below = blk[a] + tc;
    }
    if (threadIdx.x == 0) {
        const unsigned long long n = tile_count(ctl, s);
        blk[nbe] = A;
        if (may_defer && (n - A) * DEFER_DEN <= n && 5 * n <= 4 * ctl->capacity[s]) {
            ctl->alive[s] = n;                      // nothing moves; count unchanged
            ctl->holes[s] = 0;
            ctl->deferred[s] = n - A;
        } else {
            ctl->alive[s] = A;
            ctl->holes[s] = A - below;
            ctl->moved += A - below;
            ctl->deferred[s] = 0;
        }
    }
}

// pass 2: movers (alive entries at or above A) by rank, over the tiles that
// reach past A
template <class T>
__global__ void __launch_bounds__(LT) k_tile_movers(const void *w, DevCtl *ctl, int s, const unsigned long long *blk,
                                                    unsigned long long *movers) {
    __shared__ unsigned walive[LT / 32];
    const unsigned long long n = tile_count(ctl, s), A = ctl->alive[s], H = ctl->holes[s];
    if (H == 0) return;
    const unsigned long long below_A = A - H;      // alive entries below A
    const long long nbe = tiles_of(n);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long tile = (long long)(A / LTILE) + blockIdx.x; tile < nbe; tile += gridDim.x) {
        const unsigned long long base = (unsigned long long)tile * LTILE;
        const unsigned long long wbase = base + (unsigned long long)wid * LSPAN;
        unsigned amask[LROUNDS];
        unsigned cnt = 0;
#pragma unroll
        for (int r = 0; r < LROUNDS; ++r) {
            const unsigned long long i = wbase + r * 32 + lane;
            amask[r] = __ballot_sync(0xffffffffu, i < n && alive_at<T>(w, i));
            cnt += __popc(amask[r]);
        }
        if (lane == 0) walive[wid] = cnt;
        __syncthreads();
        unsigned before = 0;
        for (int k = 0; k < wid; ++k) before += walive[k];
        const unsigned lt = (1u << lane) - 1u;
        unsigned long long run = blk[tile] + before;   // alive entries before this warp's span
#pragma unroll
        for (int r = 0; r < LROUNDS; ++r) {
            const unsigned long long i = wbase + r * 32 + lane;
            if (((amask[r] >> lane) & 1u) && i >= A) {
                const unsigned long long ab = run + __popc(amask[r] & lt);
                const unsigned long long rank = ab - below_A;
                if (ab >= below_A && rank < H) movers[rank] = i;
                else atomicExch(&ctl->bad_index, i + 1);
            }
            run += __popc(amask[r]);
        }
        __syncthreads();                       // walive is rewritten by the next tile
    }
}

// pass 3: the k-th dead entry of tile b has rank (dead entries before the
// tile) + k; dead entries below A receive the mover of their rank.  (One
// warp per tile with four moves in flight per lane was measured slower: the
// moves are bound by the scattered 32-byte sectors they write, not by the
// latency of their loads.)
template <class T>
__global__ void __launch_bounds__(LT) k_tile_fill(SpeciesDev S, DevCtl *ctl, int s, const unsigned long long *blk,
                                                  const unsigned short *dl, const unsigned long long *movers) {
    const unsigned long long n = tile_count(ctl, s), A = ctl->alive[s], H = ctl->holes[s];
    if (H == 0) return;
    const long long nfill = tiles_of(A);
    for (long long tile = blockIdx.x; tile < nfill; tile += gridDim.x) {
        const unsigned long long base = (unsigned long long)tile * LTILE;
        const unsigned long long tn = n - base < (unsigned long long)LTILE ? n - base : (unsigned long long)LTILE;
        const unsigned long long alive_t = blk[tile + 1] - blk[tile];
        const unsigned dead_t = (unsigned)(tn - alive_t);
        const unsigned long long dead_before = base - blk[tile];
        const unsigned short *tdl = dl + base;
        for (unsigned k = threadIdx.x; k < dead_t; k += LT) {
            const unsigned long long i = base + tdl[k];
            if (i >= A) break;                      // offsets ascend: the rest lie at or above A too
            const unsigned long long r = dead_before + k;
            if (r < H) {
                const unsigned long long src = movers[r];
                if (src >= A && src < n) move_entry<T>(S, i, src);
                else atomicExch(&ctl->bad_index, i + 1);
            } else {
                atomicExch(&ctl->bad_index, i + 1);
            }
        }
    }
}

// Resident blocks of a tile kernel (its grid loops over tiles), at most one
// block per tile.
template <class K> static unsigned tile_grid(const qed_ctx *ctx, K kernel, long long nb) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, LT, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    const long long g = (long long)ctx->sm_count * per_sm;
    return (unsigned)(nb < g ? (nb > 0 ? nb : 1) : g);
}

// The four passes and the count update.  bound: an upper bound of the device
// count (the host count, or the capacity when the count is only known on the
// device); step_from_ctl: the leveling draws take the step index from the
// control block (a captured step graph).  The work buffers must hold
// bound / 1024 + 2 block words and bound hole words (sfq_ensure_work).
template <class T, bool LEVEL>
qed_status compact_tiles_bounded(qed_ctx *ctx, qed_species *sp, int s, int64_t step, int64_t bound,
                                 bool step_from_ctl, bool may_defer = false) {
    if (bound <= 0) return QED_OK;
    const int64_t nb = (bound + LTILE - 1) / LTILE;
    if (ctx->blk_cap < nb + 1 || ctx->slots_cap < bound) return QED_ERR_STATE;
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr, ctx->od[s]};
    // slots: bound 16-bit dead-list entries, then at most bound/2 mover indices
    unsigned short *dl = reinterpret_cast<unsigned short *>(ctx->slots);
    unsigned long long *movers = ctx->slots + (bound + 3) / 4;
    cudaStream_t st = ctx->stream;
    k_tile_dead<T, LEVEL><<<tile_grid(ctx, k_tile_dead<T, LEVEL>, nb), LT, 0, st>>>(
        S, ctx->ctl, s, ctx->lev, philox_keys(ctx->cfg.seed), (unsigned)step, step_from_ctl ? 1 : 0, ctx->blk, dl);
    k_scan_tiles<T><<<1, 1024, 0, st>>>(sp->w, ctx->blk, nb, ctx->ctl, s, may_defer ? 1 : 0);
    k_tile_movers<T><<<tile_grid(ctx, k_tile_movers<T>, nb), LT, 0, st>>>(sp->w, ctx->ctl, s, ctx->blk, movers);
    k_tile_fill<T><<<tile_grid(ctx, k_tile_fill<T>, nb), LT, 0, st>>>(S, ctx->ctl, s, ctx->blk, dl, movers);
    k_set_count<<<1, 1, 0, st>>>(ctx->ctl, s);
    SFQ_LAUNCHED(ctx, 5);
    SFQ_CUDA(cudaGetLastError());
    return QED_OK;
}

template <class T, bool LEVEL>
qed_status compact_tiles(qed_ctx *ctx, qed_species *sp, int s, int64_t step, bool may_defer = false) {
    const int64_t n = sp->count;   // upper bound; kernels read the device count
    if (n <= 0) return QED_OK;
    qed_status e = sfq_ensure_work(ctx, (n + LTILE - 1) / LTILE + 1, n);
    if (e != QED_OK) return e;
    return compact_tiles_bounded<T, LEVEL>(ctx, sp, s, step, n, false, may_defer);
}

template <class T>
qed_status compact_impl(qed_ctx *ctx, qed_species *sp, int s, bool may_defer) {
    return compact_tiles<T, false>(ctx, sp, s, 0, may_defer);
}

// The leveling iteration of one species as a CUDA graph: k_lev_begin, then
// a while node whose body is one pass (k_lev_step) and k_lev_cond.  The
// graph is kept while the weight array, the cap and the grid stay the same.
struct LevGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *w = nullptr;
    long long cap = 0;
    int blocks = 0;
};

static void lev_graph_drop(LevGraph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

template <class T>
static cudaError_t lev_graph_build(qed_ctx *ctx, LevGraph *G, const void *w, int s, long long cap, int blocks) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    LevelWork *lw = ctx->lev;
    DevCtl *ctl = ctx->ctl;
    cudaGraphConditionalHandle h;
    cudaGraphNode_t nb, nw, n1, n2;
    cudaKernelNodeParams kb{}, ks{}, kc{};
    cudaGraphNodeParams cp{};
    void *args_b[] = {&lw, &s};
    void *args_s[] = {const_cast<void **>(&w), &ctl, &s, &lw, &cap};
    void *args_c[] = {&lw, &s, &ctl, &h};
    cudaGraph_t body = nullptr;
    e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) goto fail;
    kb.func = reinterpret_cast<void *>(k_lev_begin);
    kb.gridDim = dim3(1);
    kb.blockDim = dim3(1);
    kb.kernelParams = args_b;
    e = cudaGraphAddKernelNode(&nb, g, nullptr, 0, &kb);
    if (e != cudaSuccess) goto fail;
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&nw, g, &nb, nullptr, 1, &cp);
    if (e != cudaSuccess) goto fail;
    body = cp.conditional.phGraph_out[0];
    ks.func = reinterpret_cast<void *>(k_lev_step<T>);
    ks.gridDim = dim3((unsigned)blocks);
    ks.blockDim = dim3(LEV_T);
    ks.kernelParams = args_s;
    e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &ks);
    if (e != cudaSuccess) goto fail;
    kc.func = reinterpret_cast<void *>(k_lev_cond);
    kc.gridDim = dim3(1);
    kc.blockDim = dim3(1);
    kc.kernelParams = args_c;
    e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &kc);
    if (e != cudaSuccess) goto fail;
    e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) goto fail;
    G->graph = g;
    G->w = w;
    G->cap = cap;
    G->blocks = blocks;
    return cudaSuccess;
fail:
    cudaGraphDestroy(g);
    return e;
}

// Launch species s's leveling graph (building it when needed).  false: the
// graph could not be built (conditional nodes unavailable); the caller then
// checks the passes from the host.
template <class T>
static bool lev_graph_launch(qed_ctx *ctx, const void *w, int s, long long cap, int blocks) {
    if (ctx->lev_graph_failed) return false;
    LevGraph *G = static_cast<LevGraph *>(ctx->lev_graph[s]);
    if (!G || G->w != w || G->cap != cap || G->blocks != blocks) {
        lev_graph_drop(G);
        G = new LevGraph;
        ctx->lev_graph[s] = nullptr;
        if (lev_graph_build<T>(ctx, G, w, s, cap, blocks) != cudaSuccess) {
            delete G;
            cudaGetLastError();                  // clear the failed call's error
            ctx->lev_graph_failed = 1;
            return false;
        }
        ctx->lev_graph[s] = G;
    }
    if (cudaGraphLaunch(G->exec, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        ctx->lev_graph_failed = 1;
        return false;
    }
    return true;
}

// Leveling of one species at `step`: the iteration runs on the device (a
// graph whose while loop runs one pass per iteration; without conditional
// graph nodes, one launch per pass with a host check per chunk), then
// keep/drop fused with the first compaction pass.  sp->count must bound the
// device count.
template <class T>
qed_status level_impl(qed_ctx *ctx, qed_species *sp, int s, int64_t step, bool may_defer) {
    const int64_t cap = ctx->cfg.thin_cap;
    cudaStream_t st = ctx->stream;
    if (cap <= 0 || sp->count <= cap) return QED_OK;
    int blocks = ctx->sm_count * 4;
    blocks = blocks > LEVEL_MAX_BLOCKS ? LEVEL_MAX_BLOCKS : blocks;
    if (!ctx->cfg.profile && lev_graph_launch<T>(ctx, sp->w, s, (long long)cap, blocks)) {
        SFQ_LAUNCHED(ctx, 1);                    // k_lev_begin; the passes are counted on the device
        SFQ_CUDA(cudaGetLastError());
        return compact_tiles<T, true>(ctx, sp, s, step, may_defer);
    }
    k_lev_begin<<<1, 1, 0, st>>>(ctx->lev, s);
    SFQ_LAUNCHED(ctx, 1);
    // passes in chunks (a pass after convergence returns at once); the host
    // reads the done flag and the pass count between chunks.  A chunk is as
    // long as the previous leveling of this species needed, so one check
    // usually suffices.
    int chunk = ctx->lev_chunk[s] >= 2 ? ctx->lev_chunk[s] : 3;
    for (int launched = 0; launched < LEVEL_ITERS; launched += chunk, chunk = 2) {
        for (int c = 0; c < chunk; ++c)
            k_lev_step<T><<<blocks, LEV_T, 0, st>>>(sp->w, ctx->ctl, s, ctx->lev, (long long)cap);
        SFQ_LAUNCHED(ctx, chunk);
        // done and iters are adjacent words of the iteration state
        SFQ_CUDA(cudaMemcpyAsync(ctx->pin, &ctx->lev->it[s].done, 2 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        const auto t0 = std::chrono::steady_clock::now();
        SFQ_CUDA(cudaStreamSynchronize(st));
        ctx->sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ctx->pin[0]) break;
    }
    const int used = (int)ctx->pin[1];
    ctx->lev_chunk[s] = used < 2 ? 2 : (used > 12 ? 12 : used);
    SFQ_CUDA(cudaGetLastError());
    return compact_tiles<T, true>(ctx, sp, s, step, may_defer);
}

// ---- the merge step of a captured step graph ----
// One thread decides on the device what a species' merge step does (no host
// round trip): leveling when its count exceeds the cap (the iteration is
// started as by k_lev_begin), dead entries removed when it was leveled or
// may hold converted photons (otherwise the iteration is finished with w* = 0,
// so the compaction only removes dead entries).  Nothing runs once a step
// ran out of capacity or a device check failed.
__global__ void k_merge_begin(DevCtl *ctl, LevelWork *lw, int s, long long cap, int always_compact,
                              cudaGraphConditionalHandle h_lev, cudaGraphConditionalHandle h_cmp) {
    const bool stop = ctl->overflow || ctl->timeout || ctl->bad_index;
    const unsigned long long c = ctl->count[s], cp = ctl->capacity[s];
    const unsigned long long n = c < cp ? c : cp;
    const bool level = !stop && cap > 0 && n > (unsigned long long)cap;
    lev_start(lw, s);
    if (!level) lev_finish(lw->it[s], 0.0);
    const bool compact = !stop && n > 0 && (level || always_compact);
    if (cap > 0) cudaGraphSetConditional(h_lev, level ? 1u : 0u);
    cudaGraphSetConditional(h_cmp, compact ? 1u : 0u);
    if (compact) ctl->graph_kernels += 5;          // the compaction passes below
}

// Appends species s's merge step to a step graph under capture (ctx->stream
// is the capture stream): the decision kernel, a while node running the
// leveling passes, and an if node holding the compaction passes sized by the
// capacity (their loops follow the device count).
template <class T>
qed_status capture_merge(qed_ctx *ctx, GraphBuild &gb, qed_species *sp, int s, bool always_compact) {
    const long long cap = ctx->cfg.thin_cap;
    if (sp->capacity <= 0 || (cap <= 0 && !always_compact)) return QED_OK;
    cudaGraphConditionalHandle h_lev = 0, h_cmp = 0;
    if (cap > 0 && cudaGraphConditionalHandleCreate(&h_lev, gb.g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
        return QED_ERR_CUDA;
    if (cudaGraphConditionalHandleCreate(&h_cmp, gb.g, 0, cudaGraphCondAssignDefault) != cudaSuccess)
        return QED_ERR_CUDA;
    LevelWork *lw = ctx->lev;
    DevCtl *ctl = ctx->ctl;
    const int ac = always_compact ? 1 : 0;
    if (gb.capture(gb.g, [&] {
            k_merge_begin<<<1, 1, 0, ctx->stream>>>(ctl, lw, s, cap, ac, h_lev, h_cmp);
            return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
        }) != cudaSuccess)
        return QED_ERR_CUDA;
    gb.top_kernels += 1;
    if (cap > 0) {
        cudaGraph_t body;
        if (gb.conditional(h_lev, cudaGraphCondTypeWhile, &body) != cudaSuccess) return QED_ERR_CUDA;
        int blocks = ctx->sm_count * 4;
        blocks = blocks > LEVEL_MAX_BLOCKS ? LEVEL_MAX_BLOCKS : blocks;
        const void *w = sp->w;
        if (gb.capture(body, [&] {
                k_lev_step<T><<<blocks, LEV_T, 0, ctx->stream>>>(w, ctl, s, lw, cap);
                k_lev_cond<<<1, 1, 0, ctx->stream>>>(lw, s, ctl, h_lev);
                return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
            }) != cudaSuccess)
            return QED_ERR_CUDA;
    }
    cudaGraph_t cbody;
    if (gb.conditional(h_cmp, cudaGraphCondTypeIf, &cbody) != cudaSuccess) return QED_ERR_CUDA;
    if (gb.capture(cbody, [&] { return compact_tiles_bounded<T, true>(ctx, sp, s, 0, sp->capacity, true, true); }) !=
        cudaSuccess)
        return QED_ERR_CUDA;
    return QED_OK;
}

// ---- leveling over shards (one species split across processes) ----
// The threshold is a property of all shards together: each shard evaluates
// its sums at the current point (level_eval), the caller adds them over the
// shards (an all-reduce) and advances the iteration with the same step the
// device uses (sfq_level_advance), then each shard applies w* (level_apply).
template <class T>
qed_status level_eval_impl(qed_ctx *ctx, qed_species *sp, int s, double w, double *A, int64_t *C, int64_t *N,
                           double *M) {
    cudaStream_t st = ctx->stream;
    int blocks = ctx->sm_count * 4;
    blocks = blocks > LEVEL_MAX_BLOCKS ? LEVEL_MAX_BLOCKS : blocks;
    LevelIter h{};
    h.w = w;
    h.w_up = ceil_f(w);
    h.iters = 1;
    h.mode = 1;
    const unsigned long long n = (unsigned long long)sp->count;
    const unsigned zero = 0;
    SFQ_CUDA(cudaMemcpyAsync(&ctx->ctl->count[s], &n, sizeof n, cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(&ctx->ctl->capacity[s], &n, sizeof n, cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(&ctx->lev->it[s], &h, sizeof h, cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(&ctx->lev->arrive[s], &zero, sizeof zero, cudaMemcpyHostToDevice, st));
    if (n > 0) {
        k_lev_step<T><<<blocks, LEV_T, 0, st>>>(sp->w, ctx->ctl, s, ctx->lev, 0);
        SFQ_LAUNCHED(ctx, 1);
    }
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaMemcpyAsync(&h, &ctx->lev->it[s], sizeof h, cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    *A = n > 0 ? h.sumA : 0.0;
    *C = n > 0 ? (int64_t)h.sumC : 0;
    *N = n > 0 ? (int64_t)h.sumN : 0;
    *M = n > 0 ? double_of_bits(h.sumM) : 0.0;
    return QED_OK;
}

template <class T>
qed_status level_apply_impl(qed_ctx *ctx, qed_species *sp, int s, double wstar, int64_t step) {
    LevelIter h{};
    lev_finish(h, wstar > 0.0 ? wstar : 0.0);
    SFQ_CUDA(cudaMemcpyAsync(&ctx->lev->it[s], &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
    return compact_tiles<T, true>(ctx, sp, s, step);
}

}  // namespace
}  // namespace sfq

using namespace sfq;

qed_status sfq_ensure_work(qed_ctx *ctx, int64_t n_blocks, int64_t n_slots) {
    if (ctx->blk_cap < n_blocks) {
        if (ctx->blk) SFQ_CUDA(cudaFreeAsync(ctx->blk, ctx->stream));
        ctx->blk = nullptr;
        ctx->blk_cap = 0;
        if (cudaMallocAsync(&ctx->blk, sizeof(unsigned long long) * (size_t)n_blocks, ctx->stream) != cudaSuccess)
            return QED_ERR_NOMEM;
        ctx->blk_cap = n_blocks;
    }
    if (ctx->slots_cap < n_slots) {
        if (ctx->slots) SFQ_CUDA(cudaFreeAsync(ctx->slots, ctx->stream));
        ctx->slots = nullptr;
        ctx->slots_cap = 0;
        if (cudaMallocAsync(&ctx->slots, sizeof(unsigned long long) * (size_t)n_slots, ctx->stream) != cudaSuccess)
            return QED_ERR_NOMEM;
        ctx->slots_cap = n_slots;
    }
    return QED_OK;
}

qed_status sfq_capture_merge(qed_ctx *ctx, GraphBuild &gb, qed_species *sp, int s, bool always_compact) {
    if (ctx->cfg.precision == QED_FP32) return capture_merge<float>(ctx, gb, sp, s, always_compact);
    return capture_merge<double>(ctx, gb, sp, s, always_compact);
}

// Removes every dead entry of the species, its count known only on the device
// (bounded by the capacity): the end of a batch whose steps deferred moves.
qed_status sfq_compact_pending(qed_ctx *ctx, qed_species *sp, int s) {
    if (sp->capacity <= 0) return QED_OK;
    if (ctx->cfg.precision == QED_FP32) return compact_tiles_bounded<float, false>(ctx, sp, s, 0, sp->capacity, false);
    return compact_tiles_bounded<double, false>(ctx, sp, s, 0, sp->capacity, false);
}

qed_status sfq_compact_species(qed_ctx *ctx, qed_species *sp, int s, bool may_defer) {
    if (ctx->cfg.precision == QED_FP32) return compact_impl<float>(ctx, sp, s, may_defer);
    return compact_impl<double>(ctx, sp, s, may_defer);
}

void sfq_level_graphs_free(qed_ctx *ctx) {
    for (int s = 0; s < 3; ++s) {
        lev_graph_drop(static_cast<LevGraph *>(ctx->lev_graph[s]));
        ctx->lev_graph[s] = nullptr;
    }
}

qed_status sfq_level_species(qed_ctx *ctx, qed_species *sp, int s, int64_t step, bool may_defer) {
    if (ctx->cfg.precision == QED_FP32) return level_impl<float>(ctx, sp, s, step, may_defer);
    return level_impl<double>(ctx, sp, s, step, may_defer);
}

qed_status sfq_level_eval(qed_ctx *ctx, qed_species *sp, int s, double w, double *A, int64_t *C, int64_t *N,
                          double *M) {
    if (ctx->cfg.precision == QED_FP32) return level_eval_impl<float>(ctx, sp, s, w, A, C, N, M);
    return level_eval_impl<double>(ctx, sp, s, w, A, C, N, M);
}

qed_status sfq_level_apply_species(qed_ctx *ctx, qed_species *sp, int s, double wstar, int64_t step) {
    if (ctx->cfg.precision == QED_FP32) return level_apply_impl<float>(ctx, sp, s, wstar, step);
    return level_apply_impl<double>(ctx, sp, s, wstar, step);
}

void sfq_level_advance(double *lo, double *hi, double *w, double *wstar, int64_t *iters, int64_t *done,
                       int64_t *alive, double A, int64_t C, int64_t N, double M, int64_t cap) {
    LevelIter it{};
    it.lo = *lo;
    it.hi = *hi;
    it.w = *w;
    it.wstar = *wstar;
    it.iters = (unsigned long long)*iters;
    it.done = (unsigned long long)*done;
    it.alive = (unsigned long long)*alive;
    unsigned long long mb;
    memcpy(&mb, &M, sizeof mb);
    lev_advance(it, A, (unsigned long long)C, (unsigned long long)N, mb, (long long)cap);
    *lo = it.lo;
    *hi = it.hi;
    *w = it.w;
    *wstar = it.wstar;
    *iters = (int64_t)it.iters;
    *done = (int64_t)it.done;
    *alive = (int64_t)it.alive;
}

// ---------------------------------------------------------------------------
// Compaction that allocates nothing.  Some callers cannot call cudaMalloc:
// their device memory is owned entirely by another allocator (a host code's
// memory pool), or they cannot accept the device-wide synchronisation that
// cudaMalloc / cudaFree may cause inside their time loop.  This variant keeps
// its scratch (control words, per-block counts, hole ranks) in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
// ---------------------------------------------------------------------------
namespace sfq {
namespace {
constexpr long long NA_MAX_ENTRIES = 1ll << 20;                       // largest species count accepted
constexpr long long NA_CTL_WORDS = ((long long)sizeof(DevCtl) + 255) / 256 * 32;
constexpr long long NA_BLK_WORDS = (NA_MAX_ENTRIES / CTILE + 2 + 31) / 32 * 32;
constexpr long long NA_WORDS = NA_CTL_WORDS + NA_BLK_WORDS + NA_MAX_ENTRIES;

__global__ void k_noalloc_begin(DevCtl *ctl, unsigned long long count) {
    // the array keeps the previous call's contents: reset what must start at zero
    ctl->count[0] = count;
    ctl->capacity[0] = count;
    ctl->alive[0] = 0;
    ctl->holes[0] = 0;
    ctl->bad_index = 0;
}
}  // namespace
}  // namespace sfq

static __device__ __align__(256) unsigned long long g_noalloc_scratch[sfq::NA_WORDS];

namespace {
constexpr int NA_MAX_DEVICES = 64;
unsigned long long *g_noalloc_addr[NA_MAX_DEVICES];   // device address of the array, per device
}

template <class T>
static qed_status noalloc_compact(qed_species *sp, void *od, cudaStream_t st, unsigned long long *base) {
    using namespace sfq;
    DevCtl *ctl = reinterpret_cast<DevCtl *>(base);
    unsigned long long *blk = base + NA_CTL_WORDS;
    unsigned long long *slots = blk + NA_BLK_WORDS;
    const long long n = sp->count;
    const long long nb = (n + CTILE - 1) / CTILE;
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr, od};
    k_noalloc_begin<<<1, 1, 0, st>>>(ctl, (unsigned long long)n);
    k_count_alive<T><<<(unsigned)nb, CT, 0, st>>>(sp->w, ctl, 0, blk);
    k_scan_blocks<<<1, 1024, 0, st>>>(blk, nb, ctl, 0);
    k_mark_holes<T><<<(unsigned)nb, CT, 0, st>>>(sp->w, ctl, 0, blk, slots);
    k_fill_holes<T><<<(unsigned)nb, CT, 0, st>>>(S, ctl, 0, blk, slots);
    SFQ_CUDA(cudaGetLastError());
    unsigned long long res[2];   // alive, bad index
    SFQ_CUDA(cudaMemcpyAsync(&res[0], &ctl->alive[0], sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaMemcpyAsync(&res[1], &ctl->bad_index, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    if (res[1]) return QED_ERR_STATE;
    sp->count = (int64_t)res[0];
    return QED_OK;
}

extern "C" qed_status qed_compact_species_noalloc(qed_species *sp, void *od_dev, int precision, void *cuda_stream) {
    using namespace sfq;
    if (!sp || (precision != QED_FP64 && precision != QED_FP32)) return QED_ERR_INVALID;
    // the optical-depth array moves with the particles; element alignment as in qed_set_optical_depth
    if (od_dev && (reinterpret_cast<uintptr_t>(od_dev) % (precision == QED_FP32 ? 4u : 8u))) return QED_ERR_INVALID;
    if (sp->count < 0 || sp->count > sp->capacity) return QED_ERR_INVALID;
    if (sp->count > NA_MAX_ENTRIES) return QED_ERR_INVALID;
    if (sp->count == 0) return QED_OK;
    const void *ptrs[] = {sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w, sp->id, sp->nevents};
    for (const void *q : ptrs)
        if (!q || (reinterpret_cast<uintptr_t>(q) & 15u)) return QED_ERR_INVALID;
    int dev = 0;
    SFQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return QED_ERR_INVALID;
    if (!g_noalloc_addr[dev]) {
        // once per device, with that device current: the host-side name of the
        // array is not a device address, so ask the runtime for it
        void *p = nullptr;
        SFQ_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = static_cast<unsigned long long *>(p);
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (precision == QED_FP32) return noalloc_compact<float>(sp, od_dev, st, g_noalloc_addr[dev]);
    return noalloc_compact<double>(sp, od_dev, st, g_noalloc_addr[dev]);
}
