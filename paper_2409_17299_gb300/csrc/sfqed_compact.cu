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

__global__ void k_set_count(DevCtl *ctl, int s) {
    ctl->count[s] = ctl->alive[s];
    ctl->end[s] = ctl->alive[s];
    ctl->begin[s] = ctl->alive[s];
}

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// ---- leveling: device-resident piecewise-exact Newton iteration ----
// S(w) = sum_i min(1, w_i / w) = A(w) / w + C(w) with A = sum of weights below
// w and C = count at or above w.  On the piece of w containing the root,
// S = A/w + C, whose root is A / (cap - C): evaluating (A, C) at w and jumping
// to A / (cap - C) lands on the root once the piece is right, otherwise it
// moves toward it; a bisection bracket keeps every step inside [lo, hi].
// Block partial sums are reduced in a fixed order (deterministic result).
constexpr int LEVEL_ITERS = 40;

// smallest float >= a positive double (v < d <=> v < ceil_f(d) for floats v)
__device__ __forceinline__ float ceil_f(double d) {
    float f = __double2float_ru(d);
    return f;
}

__global__ void k_lev_begin(LevelWork *lw, int s) {
    LevelIter &it = lw->it[s];
    it.lo = 0.0;
    it.hi = __longlong_as_double(0x7ff0000000000000ll);
    it.w = it.hi;
    it.w_up = __int_as_float(0x7f800000);
    it.wstar = 0.0;
    it.done = 0;
    it.iters = 0;
    it.alive = 0;
}

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

template <class T>
__global__ void __launch_bounds__(256) k_lev_eval(const void *w, const DevCtl *ctl, int s, LevelWork *lw) {
    const LevelIter &it = lw->it[s];
    if (it.done) return;
    const unsigned long long n = ctl->count[s];
    double A;
    unsigned long long C = 0, N = 0, M = 0;
    if constexpr (sizeof(T) == 4) {
        // FP32 weights: exact float comparisons and float-float sums, no FP64 per element
        const float wc = it.w_up;
        FF acc;
        unsigned mb = 0;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (unsigned long long)gridDim.x * blockDim.x) {
            const float v = reinterpret_cast<const float *>(w)[i];
            if (!(v > 0.f)) continue;
            ++N;
            mb = max(mb, __float_as_uint(v));
            if (v < wc) acc.add(v);
            else ++C;
        }
        A = (double)acc.hi + (double)acc.lo;
        M = N ? dbits((double)__uint_as_float(mb)) : 0ull;
    } else {
        const double wc = it.w;
        double comp = 0.0;           // Kahan
        A = 0.0;
        for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (unsigned long long)gridDim.x * blockDim.x) {
            const double v = (double)ld<T>(w, i);
            if (!(v > 0.0)) continue;
            ++N;
            M = max(M, dbits(v));
            if (v < wc) {
                const double y = v - comp;
                const double t = A + y;
                comp = (t - A) - y;
                A = t;
            } else {
                ++C;
            }
        }
    }
    __shared__ double sA[8];
    __shared__ unsigned long long sC[8], sN[8], sM[8];
    for (int o = 16; o > 0; o >>= 1) {
        A += __shfl_down_sync(0xffffffffu, A, o);
        C += __shfl_down_sync(0xffffffffu, C, o);
        N += __shfl_down_sync(0xffffffffu, N, o);
        M = max(M, __shfl_down_sync(0xffffffffu, M, o));
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sA[wid] = A; sC[wid] = C; sN[wid] = N; sM[wid] = M; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        unsigned long long c = 0, nn = 0, m = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += sA[k]; c += sC[k]; nn += sN[k]; m = max(m, sM[k]); }
        lw->partA[blockIdx.x] = a;
        lw->partC[blockIdx.x] = c;
        lw->partN[blockIdx.x] = nn;
        lw->partM[blockIdx.x] = m;
    }
}

__global__ void k_lev_next(LevelWork *lw, int s, int nblocks, long long cap) {
    if (threadIdx.x != 0) return;
    LevelIter &it = lw->it[s];
    if (it.done) return;
    double A = 0.0, comp = 0.0;
    unsigned long long C = 0, N = 0, M = 0;
    for (int b = 0; b < nblocks; ++b) {            // fixed order
        const double y = lw->partA[b] - comp;
        const double t = A + y;
        comp = (t - A) - y;
        A = t;
        C += lw->partC[b];
        N += lw->partN[b];
        M = max(M, lw->partM[b]);
    }
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const double w = it.w;
    if (it.iters == 0) {                           // first pass: w = +inf, all alive weights below it
        it.alive = N;
        if (N <= (unsigned long long)cap) { it.done = 1; it.wstar = 0.0; it.wstar_up = 0.f; it.wstar_f = 0.f; return; }
        it.hi = __longlong_as_double((long long)M) * (double)N / (double)cap;   // S(hi) <= cap
        it.lo = 0.0;
    } else {
        const double S = A / w + (double)C;
        if (S > (double)cap) it.lo = w; else it.hi = w;
    }
    ++it.iters;
    double c = (double)cap > (double)C ? A / ((double)cap - (double)C) : inf;
    if (c == w) {                                          // root of its own piece
        it.done = 1;
        it.wstar = w;
        it.wstar_up = ceil_f(w);
        it.wstar_f = (float)w;
        return;
    }
    if (!(c > it.lo && c <= it.hi)) c = 0.5 * (it.lo + it.hi);
    // stop at double resolution of the bracket (hi, evaluated, is the answer)
    if (!(c > it.lo && c <= it.hi) || (c == it.hi && it.hi == w) || it.iters >= LEVEL_ITERS) {
        it.done = 1;
        it.wstar = it.hi;
        it.wstar_up = ceil_f(it.hi);
        it.wstar_f = (float)it.hi;
        return;
    }
    it.w = c;
    it.w_up = ceil_f(c);
}

// keep particle i (0 < w_i < w*) with probability w_i / w*: the comparison
// u < w_i / w* is made in FP32 with a relative margin, and in FP64 (the
// oracle's test) only for draws within that margin of the boundary
template <class T>
__global__ void __launch_bounds__(256) k_lev_apply(SpeciesDev S, DevCtl *ctl, int s, const LevelWork *lw,
                                                   uint64_t seed, unsigned step) {
    const LevelIter &it = lw->it[s];
    const double wstar = it.wstar;
    if (!it.done || !(wstar > 0.0)) return;
    const float inv_f = (float)(1.0 / wstar);
    const float wup = it.wstar_up, wnew = it.wstar_f;
    const unsigned long long n = ctl->count[s];
    unsigned long long removed = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const T v = ld<T>(S.w, i);
        bool below;
        if constexpr (sizeof(T) == 4) below = v > 0.f && v < wup;     // v < w* exactly
        else below = v > 0.0 && v < wstar;
        if (!below) continue;
        const uint4 r = event_draw(seed, S.id[i], step, 0xFFFFFFFFu);
        const float uf = __uint2float_rn(r.x) * 0x1p-32f;        // u to within 2^-32 + FP32 rounding
        const float pf = (float)v * inv_f;
        bool keep;
        if (uf < pf * (1.0f - 1e-6f) - 0x1p-31f) keep = true;
        else if (uf > pf * (1.0f + 1e-6f) + 0x1p-31f) keep = false;
        else {
            double u, vv;
            Uniform<double>::draw(r.x, r.y, u, vv);
            keep = u < (double)v / wstar;
        }
        if constexpr (sizeof(T) == 4) {
            if (keep) st<T>(S.w, i, wnew);
            else { st<T>(S.w, i, 0.f); ++removed; }
        } else {
            if (keep) st<T>(S.w, i, wstar);
            else { st<T>(S.w, i, 0.0); ++removed; }
        }
    }
    for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
    if ((threadIdx.x & 31) == 0 && removed) atomicAdd(&ctl->thinned, removed);
}

template <class T>
qed_status compact_impl(qed_ctx *ctx, qed_species *sp, int s) {
    const int64_t n = sp->count;   // upper bound; kernels read the device count
    if (n <= 0) return QED_OK;
    const int64_t nb = (n + CTILE - 1) / CTILE;
    qed_status e = sfq_ensure_work(ctx, nb + 1, n);
    if (e != QED_OK) return e;
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr};
    cudaStream_t st = ctx->stream;
    k_count_alive<T><<<(unsigned)nb, CT, 0, st>>>(sp->w, ctx->ctl, s, ctx->blk);
    k_scan_blocks<<<1, 1024, 0, st>>>(ctx->blk, nb, ctx->ctl, s);
    k_mark_holes<T><<<(unsigned)nb, CT, 0, st>>>(sp->w, ctx->ctl, s, ctx->blk, ctx->slots);
    k_fill_holes<T><<<(unsigned)nb, CT, 0, st>>>(S, ctx->ctl, s, ctx->blk, ctx->slots);
    k_set_count<<<1, 1, 0, st>>>(ctx->ctl, s);
    SFQ_LAUNCHED(ctx, 5);
    SFQ_CUDA(cudaGetLastError());
    return QED_OK;
}

// Leveling of one species at `step`: the iteration runs on the device (a
// fixed number of early-exit launches, no host round trip), then keep/drop
// and compaction.  sp->count must bound the device count from above.
template <class T>
qed_status level_impl(qed_ctx *ctx, qed_species *sp, int s, int64_t step) {
    const int64_t cap = ctx->cfg.thin_cap;
    cudaStream_t st = ctx->stream;
    if (cap <= 0 || sp->count <= cap) return QED_OK;
    int blocks = ctx->sm_count * 4;
    blocks = blocks > LEVEL_MAX_BLOCKS ? LEVEL_MAX_BLOCKS : blocks;
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr};
    k_lev_begin<<<1, 1, 0, st>>>(ctx->lev, s);
    SFQ_LAUNCHED(ctx, 1);
    // iterations in chunks of three; the host reads the done flag between chunks
    // (two to five passes are typical)
    for (int it = 0; it < LEVEL_ITERS; it += 3) {
        for (int c = 0; c < 3; ++c) {
            k_lev_eval<T><<<blocks, 256, 0, st>>>(sp->w, ctx->ctl, s, ctx->lev);
            k_lev_next<<<1, 32, 0, st>>>(ctx->lev, s, blocks, (long long)cap);
        }
        SFQ_LAUNCHED(ctx, 6);
        SFQ_CUDA(cudaMemcpyAsync(ctx->pin, &ctx->lev->it[s].done, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        const auto t0 = std::chrono::steady_clock::now();
        SFQ_CUDA(cudaStreamSynchronize(st));
        ctx->sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ctx->pin[0]) break;
    }
    k_lev_apply<T><<<blocks, 256, 0, st>>>(S, ctx->ctl, s, ctx->lev, ctx->cfg.seed, (unsigned)step);
    SFQ_LAUNCHED(ctx, 1);
    SFQ_CUDA(cudaGetLastError());
    return compact_impl<T>(ctx, sp, s);
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

qed_status sfq_compact_species(qed_ctx *ctx, qed_species *sp, int s) {
    if (ctx->cfg.precision == QED_FP32) return compact_impl<float>(ctx, sp, s);
    return compact_impl<double>(ctx, sp, s);
}

qed_status sfq_level_species(qed_ctx *ctx, qed_species *sp, int s, int64_t step) {
    if (ctx->cfg.precision == QED_FP32) return level_impl<float>(ctx, sp, s, step);
    return level_impl<double>(ctx, sp, s, step);
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
static qed_status noalloc_compact(qed_species *sp, cudaStream_t st, unsigned long long *base) {
    using namespace sfq;
    DevCtl *ctl = reinterpret_cast<DevCtl *>(base);
    unsigned long long *blk = base + NA_CTL_WORDS;
    unsigned long long *slots = blk + NA_BLK_WORDS;
    const long long n = sp->count;
    const long long nb = (n + CTILE - 1) / CTILE;
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr};
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

extern "C" qed_status qed_compact_species_noalloc(qed_species *sp, int precision, void *cuda_stream) {
    using namespace sfq;
    if (!sp || (precision != QED_FP64 && precision != QED_FP32)) return QED_ERR_INVALID;
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
    if (precision == QED_FP32) return noalloc_compact<float>(sp, st, g_noalloc_addr[dev]);
    return noalloc_compact<double>(sp, st, g_noalloc_addr[dev]);
}
