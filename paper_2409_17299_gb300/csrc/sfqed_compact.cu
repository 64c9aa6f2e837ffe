// K4 / K5: removal of dead particles and global leveling
// (arXiv:2409.17299 Sec. 4.2: the merge step is where filtering and thinning
// happen; Sec. 5.1: "global leveling" keeps the particle count bounded).
//
// Compaction is in place and deterministic: with A alive entries among
// [0, N), the r-th dead slot below A receives the r-th alive entry at or
// above A (ranks from block scans), so no entry is read after it is written.
//
// Leveling: the threshold w* solves sum_i min(1, w_i / w*) = cap.  A weight
// histogram over 32 candidate values brackets w*; inside a bracket with no
// weights the sum is A / w + C, solved in closed form.  Particle i is kept
// with probability min(1, w_i / w*) from Philox(seed; id, step, 0xFFFFFFFF),
// and kept particles below w* get weight w*.
#include <math.h>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"

namespace sfq {
namespace {

constexpr int CT = 256;            // threads per compaction block
constexpr int CITEMS = 4;          // items per thread
constexpr int CTILE = CT * CITEMS; // entries per block
constexpr int NCAND = 33;          // candidate thresholds (32 brackets)
constexpr int NBIN = NCAND + 1;

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

// ---- leveling ----
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

template <class T>
__global__ void k_weight_range(const void *w, DevCtl *ctl, int s, unsigned long long *out /* min bits, max bits */) {
    const unsigned long long n = ctl->count[s];
    unsigned long long lo = ~0ull, hi = 0ull;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double v = (double)ld<T>(w, i);
        if (v > 0.0) {   // positive doubles order like their bit patterns
            lo = min(lo, dbits(v));
            hi = max(hi, dbits(v));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, lo);
        atomicMax(out + 1, hi);
    }
}

// per-bracket count, weight sum and largest weight; bin 0 below cand[0],
// bin m+1 for cand[m] <= w < cand[m+1], bin NCAND at or above cand[NCAND-1]
struct Hist {
    unsigned long long cnt[NBIN];
    double sum[NBIN];
    unsigned long long maxbits[NBIN];
};

template <class T>
__global__ void k_weight_hist(const void *w, const DevCtl *ctl, int s, const double *cand, Hist *h) {
    __shared__ double c[NCAND];
    __shared__ unsigned long long sc[NBIN], smax[NBIN];
    __shared__ double ss[NBIN];
    if (threadIdx.x < NCAND) c[threadIdx.x] = cand[threadIdx.x];
    if (threadIdx.x < NBIN) { sc[threadIdx.x] = 0; ss[threadIdx.x] = 0.0; smax[threadIdx.x] = 0; }
    __syncthreads();
    const unsigned long long n = ctl->count[s];
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double v = (double)ld<T>(w, i);
        if (!(v > 0.0)) continue;
        int b;
        if (v < c[0]) b = 0;
        else {
            int lo = 0, hi = NCAND - 1;                // largest m with c[m] <= v
            while (lo < hi) {
                const int m = (lo + hi + 1) >> 1;
                if (c[m] <= v) lo = m; else hi = m - 1;
            }
            b = lo + 1;
        }
        atomicAdd(&sc[b], 1ull);
        atomicAdd(&ss[b], v);
        atomicMax(&smax[b], dbits(v));
    }
    __syncthreads();
    if (threadIdx.x < NBIN && sc[threadIdx.x]) {
        atomicAdd(&h->cnt[threadIdx.x], sc[threadIdx.x]);
        atomicAdd(&h->sum[threadIdx.x], ss[threadIdx.x]);
        atomicMax(&h->maxbits[threadIdx.x], smax[threadIdx.x]);
    }
}

template <class T>
__global__ void k_level_apply(SpeciesDev S, DevCtl *ctl, int s, double wstar, uint64_t seed, unsigned step) {
    const unsigned long long n = ctl->count[s];
    unsigned long long removed = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double v = (double)ld<T>(S.w, i);
        if (!(v > 0.0) || v >= wstar) continue;
        const uint4 r = event_draw(seed, S.id[i], step, 0xFFFFFFFFu);
        double u, v_unused;
        Uniform<double>::draw(r.x, r.y, u, v_unused);
        if (u < v / wstar) st<T>(S.w, i, (T)wstar);
        else { st<T>(S.w, i, (T)0); ++removed; }
    }
    for (int o = 16; o > 0; o >>= 1) removed += __shfl_down_sync(0xffffffffu, removed, o);
    if ((threadIdx.x & 31) == 0 && removed) atomicAdd(&ctl->thinned, removed);
}

// ---- leveling by weight classes (one pass, no host round trip) ----
__device__ __forceinline__ void class_flush(LevelWork *lw, int s, unsigned long long b, unsigned long long c) {
    if (!c) return;
    unsigned j = (unsigned)((b >> 20) ^ (b >> 40)) & (LEVEL_K - 1);
    for (int probe = 0; probe < LEVEL_K; ++probe, j = (j + 1) & (LEVEL_K - 1)) {
        const unsigned long long prev = atomicCAS(&lw->bits[s][j], 0ull, b);
        if (prev == 0ull || prev == b) {
            atomicAdd(&lw->cnt[s][j], c);
            return;
        }
    }
    atomicExch(&lw->overflow[s], 1ull);
}

// distinct alive weights and their counts; a 4-entry register cache per
// thread keeps the table atomics rare when few weight values exist
template <class T>
__global__ void k_level_classes(const void *w, const DevCtl *ctl, int s, LevelWork *lw, long long cap) {
    const unsigned long long n = ctl->count[s];
    if (n <= (unsigned long long)cap) return;
    unsigned long long cb[4] = {0, 0, 0, 0}, cc[4] = {0, 0, 0, 0};
    unsigned victim = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double v = (double)ld<T>(w, i);
        if (!(v > 0.0)) continue;
        const unsigned long long b = dbits(v);
        int hit = -1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (cc[q] && cb[q] == b) hit = q;
        if (hit < 0) {
#pragma unroll
            for (int q = 3; q >= 0; --q)
                if (!cc[q]) hit = q;
        }
        if (hit < 0) {
            hit = (int)(victim++ & 3u);
            class_flush(lw, s, cb[hit], cc[hit]);
            cc[hit] = 0;
        }
        cb[hit] = b;
        ++cc[hit];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) class_flush(lw, s, cb[q], cc[q]);
}

// one warp: sort the classes, solve sum_c n_c min(1, v_c / w*) = cap on the
// piece (v_j, v_{j+1}] where it changes sign (there S = A_j / w + C_j), and
// set per class the integer keep threshold: u = (m + 1/2) 2^-52 < v_c / w*
// exactly when m < ceil(2^52 v_c / w* - 1/2)
__global__ void k_level_solve(DevCtl *ctl, int s, LevelWork *lw, long long cap) {
    if (threadIdx.x != 0) return;
    const unsigned long long n = ctl->count[s];
    lw->wstar[s] = 0.0;
    lw->ncls[s] = 0;
    ctl->need_hist[s] = 0;
    if (n <= (unsigned long long)cap) return;
    if (lw->overflow[s]) { ctl->need_hist[s] = 1; return; }
    double v[LEVEL_K];
    unsigned long long c[LEVEL_K], bb[LEVEL_K];
    int k = 0;
    for (int j = 0; j < LEVEL_K; ++j)
        if (lw->bits[s][j]) {
            bb[k] = lw->bits[s][j];
            v[k] = __longlong_as_double((long long)bb[k]);
            c[k] = lw->cnt[s][j];
            ++k;
        }
    for (int i = 1; i < k; ++i) {          // insertion sort, ascending weight
        const double vv = v[i];
        const unsigned long long cv = c[i], bv = bb[i];
        int j = i - 1;
        while (j >= 0 && v[j] > vv) { v[j + 1] = v[j]; c[j + 1] = c[j]; bb[j + 1] = bb[j]; --j; }
        v[j + 1] = vv; c[j + 1] = cv; bb[j + 1] = bv;
    }
    double wstar = 0.0, A = 0.0;
    unsigned long long C = 0;
    for (int j = 0; j < k; ++j) C += c[j];
    for (int j = 0; j < k; ++j) {
        A += (double)c[j] * v[j];
        C -= c[j];
        const double hi = j + 1 < k ? v[j + 1] : INFINITY;
        // S(hi) = A / hi + C: the solution lies in (v_j, hi] once S(hi) <= cap
        const double S_hi = j + 1 < k ? A / hi + (double)C : 0.0;
        if (S_hi <= (double)cap) {
            wstar = A / ((double)cap - (double)C);
            if (!(wstar > v[j])) wstar = __longlong_as_double(__double_as_longlong(v[j]) + 1);  // next double up
            if (wstar > hi) wstar = hi;
            break;
        }
    }
    for (int j = 0; j < k; ++j) {
        lw->cls_bits[s][j] = bb[j];
        unsigned long long thr = 1ull << 52;          // kept, weight unchanged
        if (v[j] < wstar) {
            const double P = (v[j] / wstar) * 0x1p52;  // exact scaling of the keep probability
            thr = (unsigned long long)ceil(P - 0.5);
        }
        lw->cls_thr[s][j] = thr;
    }
    lw->ncls[s] = (unsigned long long)k;
    lw->wstar[s] = wstar;
}

template <class T>
__global__ void k_level_apply_classes(SpeciesDev S, DevCtl *ctl, int s, const LevelWork *lw, uint64_t seed,
                                      unsigned step) {
    __shared__ unsigned long long sb[LEVEL_K], sthr[LEVEL_K];
    __shared__ int sk;
    __shared__ double sw;
    if (threadIdx.x == 0) { sk = (int)lw->ncls[s]; sw = lw->wstar[s]; }
    if (threadIdx.x < LEVEL_K) { sb[threadIdx.x] = lw->cls_bits[s][threadIdx.x]; sthr[threadIdx.x] = lw->cls_thr[s][threadIdx.x]; }
    __syncthreads();
    const double wstar = sw;
    if (!(wstar > 0.0)) return;
    const int k = sk;
    const unsigned long long n = ctl->count[s];
    unsigned long long removed = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const double v = (double)ld<T>(S.w, i);
        if (!(v > 0.0) || v >= wstar) continue;
        const unsigned long long b = dbits(v);
        unsigned long long thr = 0;
        for (int j = 0; j < k; ++j)
            if (sb[j] == b) thr = sthr[j];
        const uint4 r = event_draw(seed, S.id[i], step, 0xFFFFFFFFu);
        const unsigned long long m = ((unsigned long long)r.x << 20) | (unsigned long long)(r.y >> 12);
        if (m < thr) st<T>(S.w, i, (T)wstar);
        else { st<T>(S.w, i, (T)0); ++removed; }
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

// Histogram path, for species with more than LEVEL_K distinct weights.
template <class T>
qed_status level_hist(qed_ctx *ctx, qed_species *sp, int s, int64_t step, int64_t n) {
    const int64_t cap = ctx->cfg.thin_cap;
    cudaStream_t st = ctx->stream;
    const int blocks = ctx->sm_count * 4;
    struct Work { unsigned long long range[2]; double cand[NCAND]; Hist h; };
    Work *dw = nullptr;
    SFQ_CUDA(cudaMallocAsync(&dw, sizeof(Work), st));
    Work hw;
    hw.range[0] = ~0ull;
    hw.range[1] = 0ull;
    SFQ_CUDA(cudaMemcpyAsync(dw->range, hw.range, sizeof(hw.range), cudaMemcpyHostToDevice, st));
    k_weight_range<T><<<blocks, 256, 0, st>>>(sp->w, ctx->ctl, s, dw->range);
    SFQ_LAUNCHED(ctx, 1);
    SFQ_CUDA(cudaMemcpyAsync(hw.range, dw->range, sizeof(hw.range), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    double wmin, wmax;
    memcpy(&wmin, &hw.range[0], 8);
    memcpy(&wmax, &hw.range[1], 8);
    double lo = wmin, hi = wmax * (double)n / (double)cap;
    double wstar = hi;
    for (int it = 0; it < 24; ++it) {
        for (int m = 0; m < NCAND; ++m) hw.cand[m] = lo + (hi - lo) * m / (NCAND - 1);
        hw.cand[NCAND - 1] = hi;
        memset(&hw.h, 0, sizeof(Hist));
        SFQ_CUDA(cudaMemcpyAsync(dw->cand, hw.cand, sizeof(hw.cand) + sizeof(Hist), cudaMemcpyHostToDevice, st));
        k_weight_hist<T><<<blocks, 256, 0, st>>>(sp->w, ctx->ctl, s, dw->cand, &dw->h);
        SFQ_LAUNCHED(ctx, 1);
        SFQ_CUDA(cudaMemcpyAsync(&hw.h, &dw->h, sizeof(Hist), cudaMemcpyDeviceToHost, st));
        SFQ_CUDA(cudaStreamSynchronize(st));
        // S(c_m) = (sum of weights below c_m) / c_m + (count at or above c_m)
        double below = 0.0;
        unsigned long long above = 0;
        for (int bi = 0; bi < NBIN; ++bi) above += hw.h.cnt[bi];
        int m_hit = -1;
        double A = 0.0;
        unsigned long long C = 0;
        for (int m = 0; m < NCAND; ++m) {
            below += hw.h.sum[m];        // bins 0..m hold weights below c_m
            above -= hw.h.cnt[m];
            const double S = below / hw.cand[m] + (double)above;
            if (S <= (double)cap) { m_hit = m; A = below; C = above; break; }
        }
        if (m_hit <= 0) { wstar = hi; break; }
        const double clo = hw.cand[m_hit - 1], chi_ = hw.cand[m_hit];
        double bmax;
        memcpy(&bmax, &hw.h.maxbits[m_hit], 8);
        if (hw.h.cnt[m_hit] == 0 || bmax <= clo) {
            // for w in (c_{m-1}, c_m]: S(w) = A / w + C with A over weights < c_m
            wstar = A / ((double)cap - (double)C);
            if (!(wstar > clo && wstar <= chi_)) wstar = chi_;
            break;
        }
        lo = clo;
        hi = chi_;
        wstar = hi;
        if (hi - lo <= 4.0 * (nextafter(hi, INFINITY) - hi)) break;
    }
    SFQ_CUDA(cudaFreeAsync(dw, st));
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr};
    k_level_apply<T><<<blocks, 256, 0, st>>>(S, ctx->ctl, s, wstar, ctx->cfg.seed, (unsigned)step);
    SFQ_LAUNCHED(ctx, 1);
    SFQ_CUDA(cudaGetLastError());
    return compact_impl<T>(ctx, sp, s);
}

// Leveling of one species at `step`: weight classes, device-side solve,
// keep/drop, compaction.  No host round trip unless the species has more
// than LEVEL_K distinct weights (then the histogram path runs).  sp->count
// must bound the device count from above; it is refreshed on return when
// `sync` is set.
template <class T>
qed_status level_impl(qed_ctx *ctx, qed_species *sp, int s, int64_t step, bool sync) {
    const int64_t cap = ctx->cfg.thin_cap;
    cudaStream_t st = ctx->stream;
    if (cap <= 0 || sp->count <= cap) return QED_OK;
    const int blocks = ctx->sm_count * 4;
    SpeciesDev S{sp->x, sp->y, sp->z, sp->px, sp->py, sp->pz, sp->w,
                 reinterpret_cast<unsigned long long *>(sp->id), sp->nevents, nullptr};
    SFQ_CUDA(cudaMemsetAsync(ctx->lev->bits[s], 0, sizeof(ctx->lev->bits[s]), st));
    SFQ_CUDA(cudaMemsetAsync(ctx->lev->cnt[s], 0, sizeof(ctx->lev->cnt[s]), st));
    SFQ_CUDA(cudaMemsetAsync(&ctx->lev->overflow[s], 0, sizeof(unsigned long long), st));
    k_level_classes<T><<<blocks, 256, 0, st>>>(sp->w, ctx->ctl, s, ctx->lev, (long long)cap);
    k_level_solve<<<1, 32, 0, st>>>(ctx->ctl, s, ctx->lev, (long long)cap);
    k_level_apply_classes<T><<<blocks, 256, 0, st>>>(S, ctx->ctl, s, ctx->lev, ctx->cfg.seed, (unsigned)step);
    SFQ_LAUNCHED(ctx, 3);
    SFQ_CUDA(cudaGetLastError());
    qed_status e = compact_impl<T>(ctx, sp, s);
    if (e != QED_OK) return e;
    if (!sync) return QED_OK;
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    if (ctx->ctl_host->need_hist[s]) {
        e = level_hist<T>(ctx, sp, s, step, (int64_t)ctx->ctl_host->count[s]);
        if (e != QED_OK) return e;
        SFQ_CUDA(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
        SFQ_CUDA(cudaStreamSynchronize(st));
    }
    sp->count = (int64_t)ctx->ctl_host->count[s];
    return QED_OK;
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
    if (ctx->cfg.precision == QED_FP32) return level_impl<float>(ctx, sp, s, step, true);
    return level_impl<double>(ctx, sp, s, step, true);
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
