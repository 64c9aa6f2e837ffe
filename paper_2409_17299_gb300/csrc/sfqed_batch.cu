// K6: batched, step-fused emission push (arXiv:2409.17299 Sec. 3, Algorithm 1)
// for many independent ensembles in one persistent launch.
//
// When photons are recorded and not pushed and no leveling runs, nothing
// couples particles across steps: each lepton can be carried through all
// steps of the call while it sits in registers, and is read and written
// once.  Tiles of particles from all ensembles are handed out by a device
// work counter (uneven ensemble sizes balance themselves).  As in the
// per-step pass, particles at an event go to a per-block shared-memory stack
// and are processed densely; a stack item carries its own step index, so
// the stack mixes steps freely.  Arithmetic per particle and step is the
// same as in the per-step pass, so results are identical to nsteps calls of
// one step each.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"

namespace sfq {
namespace {

struct EnsDev {
    SpeciesDev lep[2];             // e-, e+
    SpeciesDev ph;                 // photons (appended)
    unsigned long long n_lep[2];
    unsigned long long tile0;      // first global tile of this ensemble
    unsigned long long ph_cap;
    int kind;
    int zero;                      // chi shortcut of the field (see chi_guarded)
    double prm[6];
    float prm_f[6];
};

struct BatchArgs {
    const EnsDev *ens;
    int n_ens;
    unsigned long long n_tiles;
    unsigned long long *ph_count;  // per-ensemble photon append cursor (counts demand)
    unsigned long long *tile_next; // dynamic tile counter
    DevCtl *ctl;                   // statistics
    const void *coef, *icdf;
    double dt;
    float dt_f, dt_f_gt;
    unsigned step0;
    int nsteps;
    const double *t_n;             // per step of the call: step * dt
    const float *t_red_f;          // per step: step * dt reduced mod 2 pi, in FP32
    unsigned long long seed;
    PhiloxKeys keys;               // round keys of seed
    int soft_filter;
    int budget;                    // waiting-time iterations per item before it is queued again (>= 1)
};

// field view of one ensemble at one step (eval_field's argument block),
// holding only what the precision reads (it stays in registers across steps)
template <class T> struct FieldView;
template <> struct FieldView<double> {
    int field_kind, field_zero;
    double prm[6];
    double t_n;
};
template <> struct FieldView<float> {
    int field_kind, field_zero;
    float prm_f[6];
    float t_n_red_f;
};

constexpr unsigned PENDING = 0x80000000u;   // stack item flag: the particle is at an event

template <class T, int NT> struct FusedStack {
    static constexpr int Q = 2 * NT;
    T x[3][Q], p[3][Q];
    double tau[Q];
    unsigned long long id[Q];
    unsigned long long ref[Q];     // ensemble << 40 | species << 39 | index
    T w[Q];
    unsigned k[Q];                 // events of the current step so far (pending one not counted)
    unsigned evtot[Q];             // events in this call so far
    unsigned step[Q];
    uint2 r[Q];
    int n;
};

struct FusedCtx {
    const BatchArgs &b;
    const float *coef_f;
    const double *coef_d;
};

// default number of waiting-time iterations a particle runs before it
// rejoins the block's queue (bounds the work one lane does between block
// barriers)
constexpr int BATCH_STEP_BUDGET = 4;

template <class T> __device__ __forceinline__ const T *coef_of(const FusedCtx &c);
template <> __device__ __forceinline__ const float *coef_of<float>(const FusedCtx &c) { return c.coef_f; }
template <> __device__ __forceinline__ const double *coef_of<double>(const FusedCtx &c) { return c.coef_d; }

template <class T>
__device__ __forceinline__ void set_step(FieldView<T> &v, const BatchArgs &b, unsigned step) {
    if constexpr (sizeof(T) == 8) v.t_n = b.t_n[step - b.step0];
    else v.t_n_red_f = b.t_red_f[step - b.step0];
}

template <class T>
__device__ __forceinline__ void load_view(FieldView<T> &v, const EnsDev &e, const BatchArgs &b, unsigned step) {
    v.field_kind = e.kind;
    v.field_zero = e.zero;
    for (int i = 0; i < 6; ++i) {
        if constexpr (sizeof(T) == 8) v.prm[i] = e.prm[i];
        else v.prm_f[i] = e.prm_f[i];
    }
    set_step<T>(v, b, step);
}

// One waiting-time iteration (see the per-step pass): true = stopped at an event.
template <class T, bool FRESH>
__device__ __forceinline__ bool fused_advance(const FusedCtx &c, const FieldView<T> &v, T x[3], T p[3], T q,
                                              double &tau, unsigned long long id, unsigned step, unsigned k,
                                              uint2 &rz, unsigned &n64) {
    const BatchArgs &b = c.b;
    T E[3], B[3];
    eval_field<T>(v, x, FRESH ? 0.0 : tau, E, B);
    T p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    T gam, chi;
    if constexpr (sizeof(T) == 8) {
        gam = sqrt(1.0 + p2);
        chi = chi_fp64(gam, p[0], p[1], p[2], E[0], E[1], E[2], B[0], B[1], B[2]);
    } else {
        gam = sqrtf(1.0f + p2);
        chi = chi_guarded<true>(gam, p, E, B, &n64, v.field_zero);
    }
    const T lam = p2 > (T)0 ? (T)(ALPHA * RS) / gam * rate_em<T>(coef_of<T>(c), chi) : (T)0;
    T dth = (T)INFINITY;
    if (lam > (T)0) {
        const uint4 r = event_draw(b.keys, id, step, k);
        T uw, vw;
        Uniform<T>::draw(r.x, r.y, uw, vw);
        dth = Uniform<T>::neglog(uw, vw) / lam;
        rz = make_uint2(r.z, r.w);
    }
    bool no_event;
    T h;
    if constexpr (FRESH && sizeof(T) == 4) { no_event = dth >= b.dt_f_gt; h = b.dt_f; }
    else if constexpr (FRESH) { no_event = dth > b.dt; h = b.dt; }
    else { no_event = tau + (double)dth > b.dt; h = (T)(b.dt - tau); }
    if (no_event) {
        boris<T>(x, p, q, E, B, h, false, id, step, k);
        tau = b.dt;
        return false;
    }
    boris<T>(x, p, q, E, B, dth, false, id, step, k);
    if constexpr (FRESH) tau = (double)dth;
    else tau += (double)dth;
    return true;
}

// Carry a particle forward from (step, tau) until its next event
// (RUN_EVENT), the end of the call (RUN_END), or until it has used its
// budget of waiting-time iterations (RUN_MORE: resume fresh at the start of
// `step`).  fresh: tau == 0 at the start of `step`.  The budget bounds the
// work of one item per round, so the lanes of a block do similar work
// between block barriers; a budget of one makes every item of a round one
// iteration (plus the pending emission).
constexpr int RUN_END = 0, RUN_EVENT = 1, RUN_MORE = 2;
template <class T>
__device__ __forceinline__ int fused_run(const FusedCtx &c, FieldView<T> &v, T x[3], T p[3], T q, double &tau,
                                         unsigned long long id, unsigned &step, unsigned &k, uint2 &rz, bool fresh,
                                         unsigned &mx, unsigned &n64) {
    const unsigned end = c.b.step0 + (unsigned)c.b.nsteps;
    unsigned left = (unsigned)c.b.budget;
    if (!fresh) {
        if (tau < c.b.dt) {
            --left;
            if (fused_advance<T, false>(c, v, x, p, q, tau, id, step, k, rz, n64)) return RUN_EVENT;
        }
        mx = max(mx, k);
        ++step;
    }
    for (; step < end; ++step) {
        if (left == 0) return RUN_MORE;
        --left;
        set_step<T>(v, c.b, step);
        k = 0;
        if (fused_advance<T, true>(c, v, x, p, q, tau, id, step, 0u, rz, n64)) return RUN_EVENT;
    }
    return RUN_END;
}

template <class T>
__device__ __forceinline__ void fused_emit(const FusedCtx &c, const EnsDev &e, unsigned ens, const FieldView<T> &v,
                                           const T x[3], T p[3], double tau, T w, unsigned long long id,
                                           unsigned step, unsigned k, uint2 rz, unsigned &n64) {
    const BatchArgs &b = c.b;
    T E[3], B[3];
    eval_field<T>(v, x, tau, E, B);
    T p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    T gam, chi;
    if constexpr (sizeof(T) == 8) {
        gam = sqrt(1.0 + p2);
        chi = chi_fp64(gam, p[0], p[1], p[2], E[0], E[1], E[2], B[0], B[1], B[2]);
    } else {
        gam = sqrtf(1.0f + p2);
        chi = chi_guarded<true>(gam, p, E, B, &n64, v.field_zero);
    }
    T om, ue, ve;
    Uniform<T>::draw(rz.x, rz.y, ue, ve);
    const T delta = sample_emission<T>(reinterpret_cast<const T *>(b.icdf), chi, ue, ve, &om);
    T g_after = om * gam, k0 = delta * gam;
    if (g_after < (T)1) { g_after = (T)1; k0 = gam - (T)1; }
    const T inv = f_rsqrt(p2);
    const T nx = p[0] * inv, ny = p[1] * inv, nz = p[2] * inv;
    const T pa = f_sqrt((g_after - (T)1) * (g_after + (T)1));
    if (!(b.soft_filter && k0 < (T)2)) {
        const uint4 rid = event_draw(b.seed ^ CHILD_KEY_XOR, id, step, k);
        const unsigned long long slot = warp_append(&b.ph_count[ens], 1);
        if (slot < e.ph_cap) {
            const SpeciesDev &P = e.ph;
            st<T>(P.x, slot, x[0]); st<T>(P.y, slot, x[1]); st<T>(P.z, slot, x[2]);
            st<T>(P.px, slot, k0 * nx); st<T>(P.py, slot, k0 * ny); st<T>(P.pz, slot, k0 * nz);
            st<T>(P.w, slot, w);
            P.id[slot] = (unsigned long long)rid.x | ((unsigned long long)rid.y << 32);
            P.nev[slot] = 0u;
        } else {
            atomicExch(&b.ctl->overflow, 1ull);
        }
    }
    p[0] = pa * nx; p[1] = pa * ny; p[2] = pa * nz;
}

template <class T>
__device__ __forceinline__ void fused_finish(const EnsDev &e, unsigned sp, unsigned long long i, const T x[3],
                                             const T p[3], unsigned evtot) {
    const SpeciesDev &S = e.lep[sp];
    st<T>(S.x, i, x[0]); st<T>(S.y, i, x[1]); st<T>(S.z, i, x[2]);
    st<T>(S.px, i, p[0]); st<T>(S.py, i, p[1]); st<T>(S.pz, i, p[2]);
    if (evtot) S.nev[i] += evtot;
}

template <class T, int NT>
__device__ __forceinline__ void fused_push(FusedStack<T, NT> &q, const T x[3], const T p[3], double tau,
                                           unsigned long long id, unsigned long long ref, T w, unsigned k,
                                           unsigned evtot, unsigned step, uint2 rz) {
    const int s = atomicAdd(&q.n, 1);
    q.x[0][s] = x[0]; q.x[1][s] = x[1]; q.x[2][s] = x[2];
    q.p[0][s] = p[0]; q.p[1][s] = p[1]; q.p[2][s] = p[2];
    q.tau[s] = tau; q.id[s] = id; q.ref[s] = ref; q.w[s] = w; q.k[s] = k; q.evtot[s] = evtot;
    q.step[s] = step; q.r[s] = rz;
}

template <class T, int NT>
__device__ __forceinline__ void fused_round(const FusedCtx &c, FusedStack<T, NT> &q, unsigned long long &ev,
                                            unsigned &mx, unsigned &n64) {
    const int n = q.n;
    const int take = n < NT ? n : NT;
    const int t = threadIdx.x;
    T x[3], p[3], w = 0;
    double tau = 0.0;
    unsigned long long id = 0, ref = 0;
    unsigned k = 0, evtot = 0, step = 0;
    uint2 rz = make_uint2(0, 0);
    const bool mine = t < take;
    bool pend = false;
    if (mine) {
        const int s = n - take + t;
        x[0] = q.x[0][s]; x[1] = q.x[1][s]; x[2] = q.x[2][s];
        p[0] = q.p[0][s]; p[1] = q.p[1][s]; p[2] = q.p[2][s];
        tau = q.tau[s]; id = q.id[s]; ref = q.ref[s]; w = q.w[s]; k = q.k[s]; evtot = q.evtot[s];
        step = q.step[s]; rz = q.r[s];
        pend = (k & PENDING) != 0u;     // at an event (else: resume at the start of `step`)
        k &= ~PENDING;
    }
    __syncthreads();
    if (t == 0) q.n = n - take;
    __syncthreads();
    if (mine) {
        const unsigned ens = (unsigned)(ref >> 40), sp = (unsigned)(ref >> 39) & 1u;
        const unsigned long long i = ref & ((1ull << 39) - 1);
        const EnsDev &e = c.b.ens[ens];
        FieldView<T> v;
        load_view<T>(v, e, c.b, step);
        if (pend) {
            fused_emit<T>(c, e, ens, v, x, p, tau, w, id, step, k, rz, n64);
            ++k;
            ++evtot;
            ++ev;
        }
        const T qch = sp ? (T)1 : (T)-1;
        const int r = fused_run<T>(c, v, x, p, qch, tau, id, step, k, rz, !pend, mx, n64);
        if (r == RUN_END) fused_finish<T>(e, sp, i, x, p, evtot);
        else fused_push<T, NT>(q, x, p, tau, id, ref, w, r == RUN_EVENT ? (k | PENDING) : k, evtot, step, rz);
    }
    __syncthreads();
}

template <class T, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT == 128 ? 7 : 1)) k_emission_fused(BatchArgs b) {
    __shared__ __align__(16) T s_coef[RateWords<T>::N];
    __shared__ FusedStack<T, NT> q;
    __shared__ unsigned long long s_tile;
    __shared__ int s_ens;
    for (int i = threadIdx.x; i < RateWords<T>::N; i += NT) s_coef[i] = reinterpret_cast<const T *>(b.coef)[i];
    if (threadIdx.x == 0) q.n = 0;
    __syncthreads();
    FusedCtx c{b, reinterpret_cast<const float *>(s_coef), reinterpret_cast<const double *>(s_coef)};
    unsigned long long my_ev = 0, my_ps = 0;
    unsigned my_max = 0, n64 = 0;
    // One loop with one call of fused_round: the queue is refilled from the
    // next tile while it holds less than a round, and drained at the end.
    // fused_round (and the step arithmetic in it) therefore has a single
    // inlined copy, so the budget cannot change how a result is rounded.
    bool tiles_left = true;
    for (;;) {
        if (tiles_left && q.n < NT) {
            if (threadIdx.x == 0) {
                const unsigned long long t = atomicAdd(b.tile_next, 1ull);
                s_tile = t;
                int e = -1;
                if (t < b.n_tiles) {                   // last ensemble with tile0 <= t
                    int lo = 0, hi = b.n_ens - 1;
                    while (lo < hi) {
                        const int m = (lo + hi + 1) >> 1;
                        if (b.ens[m].tile0 <= t) lo = m; else hi = m - 1;
                    }
                    e = lo;
                }
                s_ens = e;
            }
            __syncthreads();
            const unsigned long long tile = s_tile;
            const int ens = s_ens;
            __syncthreads();
            if (tile >= b.n_tiles) {
                tiles_left = false;
                continue;
            }
            const EnsDev &e = b.ens[ens];
            const unsigned long long j = (tile - e.tile0) * NT + threadIdx.x;
            const unsigned long long n0 = e.n_lep[0], n = n0 + e.n_lep[1];
            if (j < n) {
                const unsigned sp = j < n0 ? 0u : 1u;
                const unsigned long long i = sp ? j - n0 : j;
                const SpeciesDev &S = e.lep[sp];
                const T w = ld<T>(S.w, i);
                if (w > (T)0) {
                    const T x[3] = {ld<T>(S.x, i), ld<T>(S.y, i), ld<T>(S.z, i)};
                    const T p[3] = {ld<T>(S.px, i), ld<T>(S.py, i), ld<T>(S.pz, i)};
                    const unsigned long long id = __ldg(S.id + i);
                    const unsigned long long ref =
                        ((unsigned long long)ens << 40) | ((unsigned long long)sp << 39) | i;
                    my_ps += (unsigned long long)b.nsteps;
                    fused_push<T, NT>(q, x, p, 0.0, id, ref, w, 0u, 0u, b.step0, make_uint2(0, 0));
                }
            }
            __syncthreads();
            continue;
        }
        if (q.n == 0) break;
        fused_round<T, NT>(c, q, my_ev, my_max, n64);
    }
    __syncwarp();
    for (int o = 16; o > 0; o >>= 1) {
        my_ps += __shfl_down_sync(0xffffffffu, my_ps, o);
        my_ev += __shfl_down_sync(0xffffffffu, my_ev, o);
        my_max = max(my_max, __shfl_down_sync(0xffffffffu, my_max, o));
        n64 += __shfl_down_sync(0xffffffffu, n64, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (my_ps) { atomicAdd(&b.ctl->particle_steps, my_ps); atomicAdd(&b.ctl->lepton_steps, my_ps); }
        if (my_ev) atomicAdd(&b.ctl->emit_events, my_ev);
        if (my_max) atomicMax(&b.ctl->max_subevents, (unsigned long long)my_max);
        if (n64) atomicAdd(&b.ctl->chi_fp64, (unsigned long long)n64);
    }
}

template <class T, int NT> static int fused_blocks(const qed_ctx *ctx) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_emission_fused<T, NT>, NT, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (ctx->cfg.blocks_per_sm > 0 && ctx->cfg.blocks_per_sm < per_sm) per_sm = ctx->cfg.blocks_per_sm;
    return ctx->sm_count * per_sm;
}

template <class T>
static cudaError_t launch_fused(const qed_ctx *ctx, int nt, const BatchArgs &b, cudaStream_t st) {
    switch (nt) {
    case 128: k_emission_fused<T, 128><<<fused_blocks<T, 128>(ctx), 128, 0, st>>>(b); break;
    case 512: k_emission_fused<T, 512><<<fused_blocks<T, 512>(ctx), 512, 0, st>>>(b); break;
    default: k_emission_fused<T, 256><<<fused_blocks<T, 256>(ctx), 256, 0, st>>>(b); break;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace sfq

using namespace sfq;

// Work buffers of the batched push (owned by the context).
struct BatchWork {
    EnsDev *ens_d = nullptr;
    EnsDev *ens_h = nullptr;                // pinned staging
    unsigned long long *cnt_d = nullptr;    // [n_ens photon cursors, tile counter]
    unsigned long long *cnt_h = nullptr;    // pinned
    double *tn_d = nullptr;
    float *tr_d = nullptr;
    double *tn_h = nullptr;
    float *tr_h = nullptr;
    int n_ens_cap = 0;
    int nsteps_cap = 0;
};

static BatchWork *work_of(qed_ctx *ctx) { return static_cast<BatchWork *>(ctx->batch); }

void sfq_batch_free(qed_ctx *ctx) {
    BatchWork *w = work_of(ctx);
    if (!w) return;
    cudaFree(w->ens_d); cudaFree(w->cnt_d); cudaFree(w->tn_d); cudaFree(w->tr_d);
    cudaFreeHost(w->ens_h); cudaFreeHost(w->cnt_h); cudaFreeHost(w->tn_h); cudaFreeHost(w->tr_h);
    delete w;
    ctx->batch = nullptr;
}

static qed_status batch_reserve(qed_ctx *ctx, int n_ens, int nsteps) {
    BatchWork *w = work_of(ctx);
    if (!w) { w = new BatchWork(); ctx->batch = w; }
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (w->n_ens_cap < n_ens) {
        cudaFree(w->ens_d); cudaFree(w->cnt_d); cudaFreeHost(w->ens_h); cudaFreeHost(w->cnt_h);
        w->ens_d = nullptr; w->cnt_d = nullptr; w->ens_h = nullptr; w->cnt_h = nullptr;
        if (cudaMalloc(&w->ens_d, sizeof(EnsDev) * n_ens) != cudaSuccess ||
            cudaMalloc(&w->cnt_d, sizeof(unsigned long long) * (n_ens + 1)) != cudaSuccess ||
            cudaHostAlloc(&w->ens_h, sizeof(EnsDev) * n_ens, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&w->cnt_h, sizeof(unsigned long long) * (n_ens + 1), cudaHostAllocDefault) != cudaSuccess)
            return QED_ERR_NOMEM;
        w->n_ens_cap = n_ens;
    }
    if (w->nsteps_cap < nsteps) {
        cudaFree(w->tn_d); cudaFree(w->tr_d); cudaFreeHost(w->tn_h); cudaFreeHost(w->tr_h);
        w->tn_d = nullptr; w->tr_d = nullptr; w->tn_h = nullptr; w->tr_h = nullptr;
        if (cudaMalloc(&w->tn_d, sizeof(double) * nsteps) != cudaSuccess ||
            cudaMalloc(&w->tr_d, sizeof(float) * nsteps) != cudaSuccess ||
            cudaHostAlloc(&w->tn_h, sizeof(double) * nsteps, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&w->tr_h, sizeof(float) * nsteps, cudaHostAllocDefault) != cudaSuccess)
            return QED_ERR_NOMEM;
        w->nsteps_cap = nsteps;
    }
    return QED_OK;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Block shape used by the fused kernel: the configured one, else the one the
// autotuner picked for this context.
static int chosen_threads(const qed_ctx *ctx) {
    if (ctx->cfg.block_threads == 128 || ctx->cfg.block_threads == 256 || ctx->cfg.block_threads == 512)
        return ctx->cfg.block_threads;
    return ctx->tuned_threads > 0 ? ctx->tuned_threads : 256;
}

static int chosen_budget(const qed_ctx *ctx) {
    if (ctx->cfg.batch_step_budget >= 1 && ctx->cfg.batch_step_budget <= 64) return ctx->cfg.batch_step_budget;
    return ctx->tuned_budget > 0 ? ctx->tuned_budget : BATCH_STEP_BUDGET;
}

template <class T>
static qed_status batch_impl(qed_ctx *ctx, qed_particles *ens, const qed_field_desc *fields, int n_ens, double dt,
                             int nsteps, int64_t step0, qed_stats *out, int threads_override, int budget_override) {
    const auto call_t0 = std::chrono::steady_clock::now();
    qed_status e = batch_reserve(ctx, n_ens, nsteps);
    if (e != QED_OK) return e;
    BatchWork *w = work_of(ctx);
    cudaStream_t st = ctx->stream;
    const int nt = threads_override > 0 ? threads_override : chosen_threads(ctx);
    unsigned long long tiles = 0;
    for (int k = 0; k < n_ens; ++k) {
        const qed_particles &P = ens[k];
        EnsDev &d = w->ens_h[k];
        memset(&d, 0, sizeof(d));
        for (int s = 0; s < 3; ++s) {
            const qed_species &S = P.s[s];
            SpeciesDev sd{S.x, S.y, S.z, S.px, S.py, S.pz, S.w, reinterpret_cast<unsigned long long *>(S.id),
                          S.nevents, nullptr};
            if (s < 2) { d.lep[s] = sd; d.n_lep[s] = (unsigned long long)S.count; }
            else { d.ph = sd; d.ph_cap = (unsigned long long)S.capacity; }
        }
        d.tile0 = tiles;
        tiles += (d.n_lep[0] + d.n_lep[1] + nt - 1) / nt;
        d.kind = fields[k].kind;
        for (int i = 0; i < 6; ++i) { d.prm[i] = fields[k].params[i]; d.prm_f[i] = (float)fields[k].params[i]; }
        d.zero = field_zero_of(fields[k]);
        w->cnt_h[k] = (unsigned long long)P.s[2].count;
    }
    w->cnt_h[n_ens] = 0;
    for (int i = 0; i < nsteps; ++i) {
        const double tn = (double)(step0 + i) * dt;
        w->tn_h[i] = tn;
        w->tr_h[i] = (float)fmod(tn, 2.0 * 3.14159265358979323846);
    }
    memset(ctx->ctl_host, 0, sizeof(DevCtl));
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl, ctx->ctl_host, sizeof(DevCtl), cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(w->ens_d, w->ens_h, sizeof(EnsDev) * n_ens, cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(w->cnt_d, w->cnt_h, sizeof(unsigned long long) * (n_ens + 1), cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(w->tn_d, w->tn_h, sizeof(double) * nsteps, cudaMemcpyHostToDevice, st));
    SFQ_CUDA(cudaMemcpyAsync(w->tr_d, w->tr_h, sizeof(float) * nsteps, cudaMemcpyHostToDevice, st));
    BatchArgs b{};
    b.ens = w->ens_d;
    b.n_ens = n_ens;
    b.n_tiles = tiles;
    b.ph_count = w->cnt_d;
    b.tile_next = w->cnt_d + n_ens;
    b.ctl = ctx->ctl;
    const bool f32 = sizeof(T) == 4;
    b.coef = f32 ? (const void *)ctx->coef32 : (const void *)ctx->coef64;
    b.icdf = f32 ? (const void *)ctx->icdf_em32 : (const void *)ctx->icdf_em64;
    b.dt = dt;
    b.dt_f = (float)dt;
    b.dt_f_gt = (double)b.dt_f > dt ? b.dt_f : nextafterf(b.dt_f, INFINITY);
    b.step0 = (unsigned)step0;
    b.nsteps = nsteps;
    b.t_n = w->tn_d;
    b.t_red_f = w->tr_d;
    b.seed = ctx->cfg.seed;
    b.keys = philox_keys(ctx->cfg.seed);
    b.budget = budget_override > 0 ? budget_override : chosen_budget(ctx);
    b.soft_filter = ctx->cfg.soft_photon_filter;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (ctx->cfg.profile) {
        SFQ_CUDA(cudaEventCreate(&ev0));
        SFQ_CUDA(cudaEventCreate(&ev1));
        SFQ_CUDA(cudaEventRecord(ev0, st));
    }
    if (nsteps > 0 && tiles > 0) {
        // one persistent launch, replayed from a CUDA graph: captured on the
        // context's private stream (the caller's stream may be the legacy
        // default stream, which cannot be captured), launched on the caller's
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
        cudaError_t le = cudaSuccess;
        if (ce == cudaSuccess) {
            le = launch_fused<T>(ctx, nt, b, ctx->cap_stream);
            ce = cudaStreamEndCapture(ctx->cap_stream, &g);
        }
        if (ce == cudaSuccess && le == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
        if (ce == cudaSuccess && le == cudaSuccess) ce = cudaGraphLaunch(ge, st);
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (ce != cudaSuccess || le != cudaSuccess) {
            cudaGetLastError();                 // leave no stale error for the next call
            return QED_ERR_CUDA;
        }
        SFQ_LAUNCHED(ctx, 1);
    }
    if (ctx->cfg.profile) SFQ_CUDA(cudaEventRecord(ev1, st));
    SFQ_CUDA(cudaMemcpyAsync(w->cnt_h, w->cnt_d, sizeof(unsigned long long) * n_ens, cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    qed_stats s{};
    const DevCtl &c = *ctx->ctl_host;
    s.particle_steps = (int64_t)c.particle_steps;
    s.lepton_steps = (int64_t)c.lepton_steps;
    s.emit_events = (int64_t)c.emit_events;
    s.max_subevents = (int64_t)c.max_subevents;
    s.chi_fp64 = (int64_t)c.chi_fp64;
    s.launches = nsteps > 0 && tiles > 0 ? 1 : 0;
    qed_status rc = QED_OK;
    for (int k = 0; k < n_ens; ++k) {
        if (w->cnt_h[k] > (unsigned long long)ens[k].s[2].capacity) {
            rc = QED_ERR_CAPACITY;
            s.overflow = 1;
            if ((int64_t)w->cnt_h[k] > s.needed_capacity[2]) s.needed_capacity[2] = (int64_t)w->cnt_h[k];
        } else {
            ens[k].s[2].count = (int64_t)w->cnt_h[k];
        }
    }
    if (ctx->cfg.profile) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        s.kernel_ms[0] = ms;
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    s.call_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - call_t0).count();
    if (out) *out = s;
    ctx->acc.particle_steps += s.particle_steps;
    ctx->acc.lepton_steps += s.lepton_steps;
    ctx->acc.emit_events += s.emit_events;
    ctx->acc.launches += s.launches;
    return rc;
}

qed_status sfq_batch_push(qed_ctx *ctx, qed_particles *ens, const qed_field_desc *fields, int n_ens, double dt,
                          int nsteps, int64_t step0, qed_stats *out, int threads_override, int budget_override) {
    if (!ctx || !ens || !fields || n_ens <= 0 || nsteps < 0 || !(dt > 0.0) || step0 < 0 ||
        step0 + nsteps > 0xFFFFFFFFll)
        return QED_ERR_INVALID;
    if (ctx->cfg.push_photons || ctx->cfg.thin_cap > 0) return QED_ERR_INVALID;  // step fusion needs both off
    if (ctx->cfg.event_method != QED_METHOD_SUBSTEP) return QED_ERR_INVALID;      // Algorithm 1 only
    if (n_ens >= (1 << 20)) return QED_ERR_INVALID;
    for (int k = 0; k < n_ens; ++k) {
        if (fields[k].kind < QED_FIELD_UNIFORM || fields[k].kind > QED_FIELD_STANDING_CP) return QED_ERR_INVALID;
        for (int s = 0; s < 3; ++s) {
            const qed_species &S = ens[k].s[s];
            if (S.count < 0 || S.count > S.capacity || S.count >= (1ll << 39)) return QED_ERR_INVALID;
            if (S.capacity == 0) continue;
            const void *ptrs[] = {S.x, S.y, S.z, S.px, S.py, S.pz, S.w, S.id, S.nevents};
            for (const void *q : ptrs)
                if (!q || !aligned16(q)) return QED_ERR_INVALID;
        }
    }
    if (ctx->cfg.precision == QED_FP32)
        return batch_impl<float>(ctx, ens, fields, n_ens, dt, nsteps, step0, out, threads_override, budget_override);
    return batch_impl<double>(ctx, ens, fields, n_ens, dt, nsteps, step0, out, threads_override, budget_override);
}

// Autotuner: time each block shape of the fused kernel on scratch copies of
// a sample of the caller's ensembles (the caller's buffers are not touched)
// and keep the fastest for this context.
qed_status sfq_batch_autotune(qed_ctx *ctx, const qed_particles *ens, const qed_field_desc *fields, int n_ens,
                              double dt, int nsteps, int *chosen, double *ms3) {
    if (!ctx || !ens || !fields || n_ens <= 0 || nsteps <= 0 || !(dt > 0.0)) return QED_ERR_INVALID;
    if (ctx->cfg.push_photons || ctx->cfg.thin_cap > 0) return QED_ERR_INVALID;
    const size_t eb = ctx->cfg.precision == QED_FP32 ? 4 : 8;
    const int64_t budget = 1 << 20;                    // leptons in the sample
    int64_t total = 0;
    for (int k = 0; k < n_ens; ++k) total += ens[k].s[0].count + ens[k].s[1].count;
    if (total <= 0) return QED_ERR_INVALID;
    cudaStream_t st = ctx->stream;
    qed_particles *cp = static_cast<qed_particles *>(calloc((size_t)n_ens, sizeof(qed_particles)));
    if (!cp) return QED_ERR_NOMEM;
    void *pool = nullptr;
    size_t bytes = 0;
    int64_t take[1024][2];
    const int nk = n_ens < 1024 ? n_ens : 1024;
    for (int k = 0; k < nk; ++k)
        for (int s = 0; s < 2; ++s) {
            const int64_t c = ens[k].s[s].count;
            const int64_t t = total > budget ? (c * budget + total - 1) / total : c;
            take[k][s] = t < c ? t : c;
            bytes += (size_t)(take[k][s] + 16) * (7 * eb + 12) + 256;
        }
    const int64_t ph_cap = 4096 + budget / nk * nsteps / 2;
    bytes += (size_t)nk * ((size_t)ph_cap * (7 * eb + 12) + 256);
    qed_status rc = QED_OK;
    if (cudaMalloc(&pool, bytes) != cudaSuccess) { free(cp); return QED_ERR_NOMEM; }
    char *b = static_cast<char *>(pool);
    auto carve = [&](size_t n) { void *q = b; b += (n + 255) / 256 * 256; return q; };
    for (int k = 0; k < nk; ++k) {
        for (int s = 0; s < 3; ++s) {
            const int64_t cap = s < 2 ? take[k][s] + 16 : ph_cap;
            qed_species &S = cp[k].s[s];
            S.x = carve(cap * eb); S.y = carve(cap * eb); S.z = carve(cap * eb);
            S.px = carve(cap * eb); S.py = carve(cap * eb); S.pz = carve(cap * eb); S.w = carve(cap * eb);
            S.id = static_cast<uint64_t *>(carve(cap * 8));
            S.nevents = static_cast<uint32_t *>(carve(cap * 4));
            S.capacity = cap;
            S.count = s < 2 ? take[k][s] : 0;
        }
    }
    auto refill = [&]() -> qed_status {
        for (int k = 0; k < nk; ++k)
            for (int s = 0; s < 2; ++s) {
                const size_t n = (size_t)take[k][s];
                if (!n) continue;
                const qed_species &A = ens[k].s[s];
                qed_species &B = cp[k].s[s];
                const void *src[] = {A.x, A.y, A.z, A.px, A.py, A.pz, A.w};
                void *dst[] = {B.x, B.y, B.z, B.px, B.py, B.pz, B.w};
                for (int f = 0; f < 7; ++f) SFQ_CUDA(cudaMemcpyAsync(dst[f], src[f], n * eb, cudaMemcpyDeviceToDevice, st));
                SFQ_CUDA(cudaMemcpyAsync(B.id, A.id, n * 8, cudaMemcpyDeviceToDevice, st));
                SFQ_CUDA(cudaMemcpyAsync(B.nevents, A.nevents, n * 4, cudaMemcpyDeviceToDevice, st));
            }
        for (int k = 0; k < nk; ++k) cp[k].s[2].count = 0;
        return QED_OK;
    };
    const int cand[3] = {128, 256, 512};
    const int budgets[3] = {1, 2, 4};
    double best = 1e300;
    int best_nt = 256, best_b = BATCH_STEP_BUDGET;
    const int saved_profile = ctx->cfg.profile;
    ctx->cfg.profile = 1;
    for (int c = 0; c < 3 && rc == QED_OK; ++c) {
        double best_c = 1e300;
        for (int bi = 0; bi < 3 && rc == QED_OK; ++bi) {
            double ms = 0.0;
            for (int rep = 0; rep < 2 && rc == QED_OK; ++rep) {   // first repetition warms up
                rc = refill();
                if (rc != QED_OK) break;
                qed_stats s{};
                rc = sfq_batch_push(ctx, cp, fields, nk, dt, nsteps, 0, &s, cand[c], budgets[bi]);
                if (rc == QED_ERR_CAPACITY) rc = QED_OK;             // timing is still valid
                ms = s.kernel_ms[0];
            }
            if (ms < best_c) best_c = ms;
            if (ms < best) { best = ms; best_nt = cand[c]; best_b = budgets[bi]; }
        }
        if (ms3) ms3[c] = best_c;
    }
    ctx->cfg.profile = saved_profile;
    cudaStreamSynchronize(st);
    cudaFree(pool);
    free(cp);
    if (rc != QED_OK) return rc;
    ctx->tuned_threads = best_nt;
    ctx->tuned_budget = best_b;
    if (chosen) *chosen = best_nt;
    return QED_OK;
}

qed_status sfq_batch_shape(qed_ctx *ctx, int *threads, int *budget) {
    if (!ctx) return QED_ERR_INVALID;
    if (threads) *threads = chosen_threads(ctx);
    if (budget) *budget = chosen_budget(ctx);
    return QED_OK;
}
