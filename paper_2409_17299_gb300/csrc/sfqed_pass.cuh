// The pass kernels of the per-particle QED step (arXiv:2409.17299 Sec. 3,
// Algorithms 1-2) and their launcher, compiled twice: once for the analytic
// field descriptors (SFQ_GRID 0) and once for the gridded field (SFQ_GRID 1),
// each into its own namespace (SFQ_PASS_NS), so neither variant carries the
// other's field code or registers.
//
// One pass kernel per particle kind.  Each thread takes one particle of the
// pass range (grid-stride), runs Algorithm 1 for it to the end of the step
// (rate -> waiting time -> Boris push -> event), and appends every particle
// it creates with a warp-aggregated atomic.  Newborns carry their birth
// clock and are pushed by the next pass (Algorithm 2): leptons and photons
// are swept alternately until a pass creates nothing.
#pragma once

#include <math.h>
#include <string.h>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"
#include "sfqed_mma.cuh"

#if !defined(SFQ_GRID) || !defined(SFQ_PASS_NS)
#error "define SFQ_GRID and SFQ_PASS_NS before including sfqed_pass.cuh"
#endif

namespace sfq {
namespace SFQ_PASS_NS {

// the field at a particle: the gridded field in the grid variant, the
// analytic descriptor otherwise
template <class T>
__device__ __forceinline__ void field_at(const PassArgs &a, const T x[3], const Phase<T> &ph, T E[3], T B[3]) {
#if SFQ_GRID
    (void)ph;
    eval_grid<T, PassArgs>(a, x, E, B);
#else
    eval_field_at<T, PassArgs>(a, x, ph, E, B);
#endif
}

template <class T>
__device__ __forceinline__ void field_tau(const PassArgs &a, const StepTime &tm, const T x[3], double tau, T E[3],
                                          T B[3]) {
#if SFQ_GRID
    (void)tau;
    (void)tm;
    eval_grid<T, PassArgs>(a, x, E, B);
#else
    eval_field_at<T, PassArgs>(a, x, time_phase<T, StepTime>(tm, tau), E, B);
#endif
}

// The current step's time and index, written into the control block by the
// step-begin kernel (so a step captured in a CUDA graph takes no per-step
// kernel arguments)
__device__ __forceinline__ StepTime load_step_time(const PassArgs &a) {
    const DevCtl *c = a.ctl;
    StepTime t;
    t.field_kind = a.field_kind;
    t.t_n = c->sv_t_n;
    t.t_n_red_f = c->sv_t_red_f;
    t.step = c->sv_step;
    return t;
}

// tau < dt for the clock's non-negative doubles, as an integer comparison of
// their bit patterns (which order like the values): no FP64 instruction
__device__ __forceinline__ bool before_step_end(double tau, double dt) {
    return __double_as_longlong(tau) < __double_as_longlong(dt);
}

template <class T> __device__ __forceinline__ T t_inf();
template <> __device__ __forceinline__ double t_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }
template <> __device__ __forceinline__ float t_inf<float>() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ void flush_stats(DevCtl *ctl, unsigned long long steps, unsigned long long ev,
                                            unsigned mx, bool pair, unsigned n64) {
    // called by every lane of the warp after the grid-stride loop
    for (int o = 16; o > 0; o >>= 1) {
        steps += __shfl_down_sync(0xffffffffu, steps, o);
        ev += __shfl_down_sync(0xffffffffu, ev, o);
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        n64 += __shfl_down_sync(0xffffffffu, n64, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n64) atomicAdd(&ctl->chi_fp64, (unsigned long long)n64);
        if (steps) {
            atomicAdd(&ctl->particle_steps, steps);
            atomicAdd(pair ? &ctl->photon_steps : &ctl->lepton_steps, steps);
        }
        if (ev) atomicAdd(pair ? &ctl->pair_events : &ctl->emit_events, ev);
        if (mx) atomicMax(&ctl->max_subevents, (unsigned long long)mx);
    }
}

// chi and energy of a lepton / photon in the mode's precision: FP64 mode uses
// the direct FP64 form; FP32 mode the guarded form with FP64 fallback.
__device__ __forceinline__ void note_overflow(DevCtl *ctl, int s, unsigned long long slot) {
    atomicMax(&ctl->needed[s], slot + 1);
    atomicExch(&ctl->overflow, 1ull);
}

// Algorithm 1 for electrons and positrons (both species of one pass).
//
// Divergence control (the GPU form of Algorithm 3's "sort handled particles
// to the front"): phase 1 pushes every particle of a 256-particle tile to its
// first event or to the end of the step; particles at an event go to a
// per-block stack in shared memory.  Whenever the stack holds a full round,
// the block pops one item per thread and processes it densely: the event
// (chi at the point, energy draw, recoil, photon append), then the next
// waiting time, ending either at the step end (state stored) or at the next
// event (pushed back).  The stack is drained after the last tile.
constexpr int LB = 256;            // threads per block of the lepton pass
constexpr int LQ = 2 * LB;         // stack capacity: < LB left + LB pushed

template <class T> struct LeptonStack {
    T x[3][LQ], p[3][LQ];
    double tau[LQ];
    unsigned long long id[LQ];
    T w[LQ];
    unsigned idx[LQ];              // index | species << 31
    unsigned k[LQ];                // events so far in this step (the pending one not counted)
    uint2 r[LQ];                   // the pending event's energy draw words
    int n;
};

template <class T> struct LeptonCtx {
    const PassArgs &a;
    DevCtl *ctl;
    const T *coef;
    const T *icdf;
    unsigned long long cap_ph;
    T alpha_r;
    const StepTime &tm;     // the step's time and index (block's shared copy)
    Phase<T> ph0;           // time phase at the step start (tau = 0)
};

// A rate below 2^-54 / dt cannot give an event in a step: the waiting time
// -ln u / lambda is at least 2^-53 / lambda > 2 dt, because 1 - u is never
// below 2^-53 (FP64 and FP32 draws alike).  Such particles skip the draw (no
// draw is consumed without an event, so the counter sequence is unchanged);
// in the cascades this is most photons with chi below ~0.1.
template <class T> __device__ __forceinline__ T lam_skip(const PassArgs &a);
template <> __device__ __forceinline__ float lam_skip<float>(const PassArgs &a) { return a.lam_skip_f; }
template <> __device__ __forceinline__ double lam_skip<double>(const PassArgs &a) { return a.lam_skip; }

// One waiting-time iteration from (x, p, tau).  Returns true and leaves the
// particle at its event point (tau advanced, draw words in rz) if an event
// happens before the step end, else pushes it to the end and returns false.
// FRESH: tau == 0 (first iteration of a particle present at the step start);
// then the event test "0 + dt_hat > dt" and the push length need no FP64
// instruction in FP32 mode (the smallest float above dt decides exactly).
template <class T, bool FRESH>
__device__ __forceinline__ bool advance(const LeptonCtx<T> &c, T x[3], T p[3], T q, double &tau,
                                        unsigned long long id, unsigned k, uint2 &rz, unsigned &n64) {
    const PassArgs &a = c.a;
    T E[3], B[3];
    if constexpr (FRESH) field_at<T>(a, x, c.ph0, E, B);
    else field_tau<T>(a, c.tm, x, tau, E, B);
    T gam, chi, p2;
    lepton_chi<T>(p, E, B, gam, chi, p2, n64, a.field_zero);
    const T lam = p2 > (T)0 ? f_div(c.alpha_r, gam) * rate_em<T>(c.coef, chi) : (T)0;
    T dth = t_inf<T>();
    if (lam > lam_skip<T>(a)) {
        const uint4 r = event_draw(a.keys, id, c.tm.step, k);
        T uw, vw;
        Uniform<T>::draw(r.x, r.y, uw, vw);
        dth = f_div(Uniform<T>::neglog(uw, vw), lam);
        rz = make_uint2(r.z, r.w);
    }
    bool no_event;
    T h;
    if constexpr (FRESH && sizeof(T) == 4) { no_event = dth >= a.dt_f_gt; h = a.dt_f; }
    else if constexpr (FRESH) { no_event = dth > a.dt; h = a.dt; }
    else if constexpr (sizeof(T) == 4) {
        // FP32 mode after a particle's first event: the FP64 test
        // tau + dth > dt decided in FP32 wherever dth lies outside a margin
        // around the remaining time rem = dt - tau (rounded once to float);
        // the margin (2^-20 rem + 2^-40 dt) exceeds every rounding involved,
        // so the decision is the FP64 one, and within it the FP64 test runs
        const float rf = __double2float_rn(a.dt - tau);
        const float marg = fmaf(rf, 0x1p-20f, a.dt_f * 0x1p-40f);
        if (dth > rf + marg) no_event = true;
        else if (dth < rf - marg) no_event = false;
        else no_event = tau + (double)dth > a.dt;
        h = rf;
    } else { no_event = tau + (double)dth > a.dt; h = (T)(a.dt - tau); }
    if (no_event) {
        boris<T>(x, p, q, E, B, h, a.field_zero == 1, id, c.tm.step, k);
        tau = a.dt;
        return false;
    }
    boris<T>(x, p, q, E, B, dth, a.field_zero == 1, id, c.tm.step, k);
    if constexpr (FRESH) tau = (double)dth;
    else tau += (double)dth;
    return true;
}

// Kinematics of an emission with photon fraction delta (and 1 - delta) from a
// lepton of energy gam and momentum p at x: collinear, energy-conserving
// recoil; the photon is appended.
template <class T>
__device__ __forceinline__ void emit_with(const LeptonCtx<T> &c, const T x[3], T p[3], double tau, T w,
                                          unsigned long long id, unsigned k, T gam, T p2, T delta, T om) {
    const PassArgs &a = c.a;
    T g_after = om * gam, k0 = delta * gam;
    if (g_after < (T)1) { g_after = (T)1; k0 = gam - (T)1; }
    const T inv = f_rsqrt(p2);
    const T nx = p[0] * inv, ny = p[1] * inv, nz = p[2] * inv;
    const T pa = f_sqrt((g_after - (T)1) * (g_after + (T)1));
    if (!(a.soft_filter && k0 < (T)2)) {
        const uint4 rid = event_draw(a.seed ^ CHILD_KEY_XOR, id, c.tm.step, k);
        const unsigned long long slot = warp_append(&c.ctl->count[2], 1);
        if (slot < c.cap_ph) {
            const SpeciesDev &P = a.sp[2];
            st<T>(P.x, slot, x[0]); st<T>(P.y, slot, x[1]); st<T>(P.z, slot, x[2]);
            st<T>(P.px, slot, k0 * nx); st<T>(P.py, slot, k0 * ny); st<T>(P.pz, slot, k0 * nz);
            st<T>(P.w, slot, w);
            P.id[slot] = (unsigned long long)rid.x | ((unsigned long long)rid.y << 32);
            P.nev[slot] = 0u;
            if (a.record_newborn_tau) P.tau[slot] = tau;
            if (P.od) st<T>(P.od, slot, (T)0);       // optical depth not drawn yet
        } else {
            note_overflow(c.ctl, 2, slot);
        }
    }
    p[0] = pa * nx; p[1] = pa * ny; p[2] = pa * nz;
}

// The event at the particle's current point with the table sampler: chi
// there, energy fraction from the inverse CDF, then the kinematics.
template <class T>
__device__ __forceinline__ void emit(const LeptonCtx<T> &c, const T x[3], T p[3], double tau, T w,
                                     unsigned long long id, unsigned k, uint2 rz, unsigned &n64) {
    T E[3], B[3];
    field_tau<T>(c.a, c.tm, x, tau, E, B);
    T gam, chi, p2;
    lepton_chi<T>(p, E, B, gam, chi, p2, n64, c.a.field_zero);
    T om, ue, ve;
    Uniform<T>::draw(rz.x, rz.y, ue, ve);
    const T delta = sample_emission<T>(c.icdf, chi, ue, ve, &om);
    emit_with<T>(c, x, p, tau, w, id, k, gam, p2, delta, om);
}

// Network sampler of a block: the staged network (dynamic shared memory)
constexpr int MLP_SMEM_BYTES = MLP_INF_BYTES;

template <class T>
__device__ __forceinline__ void finish(const PassArgs &a, unsigned idx, const T x[3], const T p[3], unsigned k) {
    const SpeciesDev &S = a.sp[idx >> 31];
    const unsigned i = idx & 0x7FFFFFFFu;
    st<T>(S.x, i, x[0]); st<T>(S.y, i, x[1]); st<T>(S.z, i, x[2]);
    st<T>(S.px, i, p[0]); st<T>(S.py, i, p[1]); st<T>(S.pz, i, p[2]);
    if (k) S.nev[i] += k;
}

template <class T>
__device__ __forceinline__ void stack_push(LeptonStack<T> &q, const T x[3], const T p[3], double tau,
                                           unsigned long long id, T w, unsigned idx, unsigned k, uint2 rz) {
    const int slot = atomicAdd(&q.n, 1);
    q.x[0][slot] = x[0]; q.x[1][slot] = x[1]; q.x[2][slot] = x[2];
    q.p[0][slot] = p[0]; q.p[1][slot] = p[1]; q.p[2][slot] = p[2];
    q.tau[slot] = tau; q.id[slot] = id; q.w[slot] = w; q.idx[slot] = idx; q.k[slot] = k; q.r[slot] = rz;
}

// Pop min(n, LB) items, one per thread, and process each to its next event
// or the step end.  Every thread of the block calls this.
template <class T, bool MLP>
__device__ __forceinline__ void stack_round(const LeptonCtx<T> &c, LeptonStack<T> &q, unsigned long long &ev,
                                            unsigned &mx, unsigned &n64, const MlpInf &ms) {
    const int n = q.n;
    const int take = n < LB ? n : LB;
    const int t = threadIdx.x;
    T x[3], p[3], w = 0;
    double tau = 0.0;
    unsigned long long id = 0;
    unsigned idx = 0, k = 0;
    uint2 rz = make_uint2(0, 0);
    const bool mine = t < take;
    if (mine) {
        const int s = n - take + t;
        x[0] = q.x[0][s]; x[1] = q.x[1][s]; x[2] = q.x[2][s];
        p[0] = q.p[0][s]; p[1] = q.p[1][s]; p[2] = q.p[2][s];
        tau = q.tau[s]; id = q.id[s]; w = q.w[s]; idx = q.idx[s]; k = q.k[s]; rz = q.r[s];
    }
    __syncthreads();
    if (t == 0) q.n = n - take;
    __syncthreads();
    if constexpr (MLP) {
        // event-point state per item, then the whole warp evaluates the
        // network for its 32 items on the tensor cores
        T gam = (T)1, chi = (T)0, p2 = (T)0, ue = (T)0.5, ve = (T)0.5;
        float f0 = 0.f, f1 = 0.f;
        bool use_net = false;
        if (mine) {
            T E[3], B[3];
            field_tau<T>(c.a, c.tm, x, tau, E, B);
            lepton_chi<T>(p, E, B, gam, chi, p2, n64, c.a.field_zero);
            Uniform<T>::draw(rz.x, rz.y, ue, ve);
            const float sl = (float)logit(ue, ve);
            const float cf = (float)chi;
            use_net = cf >= 1e-3f && cf <= 1e3f && fabsf(sl) < 16.0f;
            if (use_net) { f0 = log10f(cf) / 3.0f; f1 = sl / 16.0f; }
        }
        const float y = mlp_forward_warp(f0, f1, ms);
        if (mine) {
            T delta, om;
            if (use_net) {
                const T aa = (T)3 * chi * (T)__expf(16.0f * (y - 0.5f));
                om = (T)2 / ((T)2 + aa);
                delta = aa / ((T)2 + aa);
            } else {
                delta = sample_emission<T>(c.icdf, chi, ue, ve, &om);
            }
            emit_with<T>(c, x, p, tau, w, id, k, gam, p2, delta, om);
        }
    } else {
        if (mine) emit<T>(c, x, p, tau, w, id, k, rz, n64);
    }
    if (mine) {
        ++k;
        ++ev;
        const T qch = (idx >> 31) ? (T)1 : (T)-1;
        if (before_step_end(tau, c.a.dt) && advance<T, false>(c, x, p, qch, tau, id, k, rz, n64)) {
            stack_push<T>(q, x, p, tau, id, w, idx, k, rz);
        } else {
            finish<T>(c.a, idx, x, p, k);
            mx = max(mx, k);
        }
    }
    __syncthreads();
}

template <class T, bool FRESH, bool MLP>
__global__ void __launch_bounds__(LB, (sizeof(T) == 4 ? (MLP ? 2 : 4) : 1)) k_lepton_pass(PassArgs a) {
    // blocks past the pass's range leave before staging anything (a newborn
    // pass is often far smaller than the resident grid)
    if ((unsigned long long)blockIdx.x * LB >= (a.ctl->end[0] - a.ctl->begin[0]) + (a.ctl->end[1] - a.ctl->begin[1]))
        return;
    __shared__ __align__(16) T s_coef[RateWords<T>::N];
    __shared__ LeptonStack<T> q;
    __shared__ StepTime s_tm;
    extern __shared__ __align__(16) unsigned char dyn[];
    MlpInf ms{nullptr, nullptr, nullptr};
    if constexpr (MLP) ms = mlp_stage(dyn, a.mlp_w16);
    for (int i = threadIdx.x; i < RateWords<T>::N; i += blockDim.x) s_coef[i] = reinterpret_cast<const T *>(a.coef)[i];
    if (threadIdx.x == 0) {
        q.n = 0;
        s_tm = load_step_time(a);
    }
    __syncthreads();
    DevCtl *ctl = a.ctl;
    // 32-bit indices (a species holds fewer than 2^31 entries: bit 31 of idx names the species)
    const unsigned b0 = (unsigned)ctl->begin[0], n0 = (unsigned)(ctl->end[0] - ctl->begin[0]);
    const unsigned b1 = (unsigned)ctl->begin[1], n1 = (unsigned)(ctl->end[1] - ctl->begin[1]);
    const unsigned n = n0 + n1;
    const LeptonCtx<T> c{a, ctl, s_coef, reinterpret_cast<const T *>(a.icdf_em), ctl->capacity[2], (T)(ALPHA * RS),
                         s_tm, time_phase<T, StepTime>(s_tm, 0.0)};
    unsigned long long my_steps = 0, my_ev = 0;
    unsigned my_max = 0, n64 = 0;

    // FP32 step-start pass: each thread stages its particle of the block's
    // next tile in shared memory while the block works on the current tile
    constexpr bool STAGE = FRESH && sizeof(T) == 4;
    constexpr int NF = STAGE ? 9 : 1, NT = STAGE ? LB : 1;
    __shared__ __align__(16) float stg[NF][NT];            // w x y z px py pz id(2 words)
    const unsigned stride = gridDim.x * LB;
    auto stage = [&](unsigned jj) {
        if constexpr (STAGE) {
            const int sp = jj < n0 ? 0 : 1;
            const unsigned ii = sp == 0 ? b0 + jj : b1 + (jj - n0);
            const SpeciesDev &P = a.sp[sp];
            const int t = threadIdx.x;
            cp_async4(&stg[0][t], reinterpret_cast<const float *>(P.w) + ii);
            cp_async4(&stg[1][t], reinterpret_cast<const float *>(P.x) + ii);
            cp_async4(&stg[2][t], reinterpret_cast<const float *>(P.y) + ii);
            cp_async4(&stg[3][t], reinterpret_cast<const float *>(P.z) + ii);
            cp_async4(&stg[4][t], reinterpret_cast<const float *>(P.px) + ii);
            cp_async4(&stg[5][t], reinterpret_cast<const float *>(P.py) + ii);
            cp_async4(&stg[6][t], reinterpret_cast<const float *>(P.pz) + ii);
            cp_async4(&stg[7][t], P.id + ii);
            cp_async4(&stg[8][t], reinterpret_cast<const unsigned *>(P.id + ii) + 1);
        }
    };
    if constexpr (STAGE) {
        const unsigned j0 = blockIdx.x * LB + threadIdx.x;
        if (j0 < n) stage(j0);
        cp_async_commit();
    }

    // One loop with one call of stack_round: the next tile is taken while the
    // stack holds less than a round, the stack is drained at the end.  The
    // round (and the event arithmetic in it) then has a single inlined copy,
    // so which round processes a particle, which depends on the order of the
    // arrays, cannot change how its results are rounded.
    unsigned base = blockIdx.x * LB;
    for (;;) {
        if (base < n && q.n < LB) {
            const unsigned j = base + threadIdx.x;
            T w = (T)0, x[3], p[3];
            unsigned long long id = 0;
            if constexpr (STAGE) {
                // this thread's staged particle, then the next tile's copies in
                // flight (the slots are free once read)
                cp_async_wait_all();
                if (j < n) {
                    const int t = threadIdx.x;
                    w = stg[0][t];
                    x[0] = stg[1][t]; x[1] = stg[2][t]; x[2] = stg[3][t];
                    p[0] = stg[4][t]; p[1] = stg[5][t]; p[2] = stg[6][t];
                    id = (unsigned long long)__float_as_uint(stg[7][t]) |
                         ((unsigned long long)__float_as_uint(stg[8][t]) << 32);
                }
                if (j + stride < n) stage(j + stride);
                cp_async_commit();
            }
            if (j < n) {
                const int s = j < n0 ? 0 : 1;
                const unsigned i = s == 0 ? b0 + j : b1 + (j - n0);
                const SpeciesDev &S = a.sp[s];
                if constexpr (!STAGE) {
                    w = ld<T>(S.w, i);
                    x[0] = ld<T>(S.x, i); x[1] = ld<T>(S.y, i); x[2] = ld<T>(S.z, i);
                    p[0] = ld<T>(S.px, i); p[1] = ld<T>(S.py, i); p[2] = ld<T>(S.pz, i);
                    id = __ldg(S.id + i);
                }
                if (w > (T)0) {
                    double tau = FRESH ? 0.0 : S.tau[i];
                    const unsigned idx = i | ((unsigned)s << 31);
                    ++my_steps;
                    uint2 rz = make_uint2(0, 0);
                    const T qch = s == 0 ? (T)-1 : (T)1;
                    bool event;
                    if constexpr (FRESH) event = advance<T, true>(c, x, p, qch, tau, id, 0u, rz, n64);
                    else event = before_step_end(tau, a.dt) && advance<T, false>(c, x, p, qch, tau, id, 0u, rz, n64);
                    if (event) {
                        stack_push<T>(q, x, p, tau, id, w, idx, 0u, rz);
                    } else {
                        finish<T>(a, idx, x, p, 0u);
                    }
                }
            }
            base += stride;
            __syncthreads();
            continue;
        }
        if (q.n == 0) break;
        stack_round<T, MLP>(c, q, my_ev, my_max, n64, ms);
    }
    __syncwarp();
    flush_stats(ctl, my_steps, my_ev, my_max, false, n64);
}

// Pair creation at a photon's event point x at clock tau (Sec. 3): chi there,
// electron fraction from the inverse CDF with the draw words rz, both leptons
// along the photon's direction with energy-conserving momenta, appended with
// their ids and birth clock.  The caller removes the photon.
template <class T>
__device__ __forceinline__ void pair_create(const PassArgs &a, const StepTime &tm, const T *icdf, const T x[3],
                                            const T kv[3], T k0, T nx, T ny, T nz, double tau, T w,
                                            unsigned long long id, unsigned k, uint2 rz, unsigned &n64) {
    DevCtl *ctl = a.ctl;
    T E[3], B[3];
    field_tau<T>(a, tm, x, tau, E, B);
    const T chi = photon_chi<T>(k0, kv, E, B, n64, a.field_zero);
    T om, ue, ve;
    Uniform<T>::draw(rz.x, rz.y, ue, ve);
    const T delta = sample_pair<T>(icdf, chi, ue, ve, &om);
    T em = delta * k0, ep = om * k0;
    em = em < (T)1 ? (T)1 : em;
    ep = ep < (T)1 ? (T)1 : ep;
    const T pm = f_sqrt((em - (T)1) * (em + (T)1)), pp = f_sqrt((ep - (T)1) * (ep + (T)1));
    const uint4 rid = event_draw(a.seed ^ CHILD_KEY_XOR, id, tm.step, k);
    const unsigned long long se = warp_append(&ctl->count[0], 1);
    const unsigned long long sp = warp_append(&ctl->count[1], 1);
    if (se < ctl->capacity[0]) {
        const SpeciesDev &P = a.sp[0];
        st<T>(P.x, se, x[0]); st<T>(P.y, se, x[1]); st<T>(P.z, se, x[2]);
        st<T>(P.px, se, pm * nx); st<T>(P.py, se, pm * ny); st<T>(P.pz, se, pm * nz);
        st<T>(P.w, se, w);
        P.id[se] = (unsigned long long)rid.x | ((unsigned long long)rid.y << 32);
        P.nev[se] = 0u;
        P.tau[se] = tau;
        if (P.od) st<T>(P.od, se, (T)0);
    } else {
        note_overflow(ctl, 0, se);
    }
    if (sp < ctl->capacity[1]) {
        const SpeciesDev &P = a.sp[1];
        st<T>(P.x, sp, x[0]); st<T>(P.y, sp, x[1]); st<T>(P.z, sp, x[2]);
        st<T>(P.px, sp, pp * nx); st<T>(P.py, sp, pp * ny); st<T>(P.pz, sp, pp * nz);
        st<T>(P.w, sp, w);
        P.id[sp] = (unsigned long long)rid.z | ((unsigned long long)rid.w << 32);
        P.nev[sp] = 0u;
        P.tau[sp] = tau;
        if (P.od) st<T>(P.od, sp, (T)0);
    } else {
        note_overflow(ctl, 1, sp);
    }
}

// One photon of a pass from its loaded state (index i, weight w, position x,
// momentum k, id): straight flight, pair creation at the event (the photon
// is removed: weight 0 and its event count stored here).  Returns false for
// a dead photon (weight 0: nothing to do and nothing to store); otherwise x
// holds the new position, which the caller stores, and k the events.
template <class T, bool FRESH>
__device__ __forceinline__ bool photon_step(const PassArgs &a, const StepTime &tm, const T *s_coef, const T *icdf,
                                            const Phase<T> &ph0, const SpeciesDev &S, unsigned i, T w, T x[3],
                                            T kx, T ky, T kz, unsigned long long id, unsigned &k, unsigned &n64) {
    k = 0;
    if (!(w > (T)0)) return false;
    const T alpha_r = (T)(ALPHA * RS);
    double tau = FRESH ? 0.0 : S.tau[i];
    const T kv[3] = {kx, ky, kz};
    const T k0 = f_sqrt(kx * kx + ky * ky + kz * kz);
    if (k0 > (T)0) {
        const T inv = f_div((T)1, k0);
        const T nx = kx * inv, ny = ky * inv, nz = kz * inv;
        // one waiting time: the photon either reaches the step end or converts
        if (FRESH || before_step_end(tau, a.dt)) {
            T E[3], B[3];
            if constexpr (FRESH) field_at<T>(a, x, ph0, E, B);
            else field_tau<T>(a, tm, x, tau, E, B);
            T chi = photon_chi<T>(k0, kv, E, B, n64, a.field_zero);
            T lam;
            if constexpr (sizeof(T) == 4) lam = alpha_r * inv * rate_pair<T>(s_coef, chi);
            else lam = alpha_r / k0 * rate_pair<T>(s_coef, chi);     // the oracle's rounding
            uint4 r = make_uint4(0, 0, 0, 0);
            T dth = t_inf<T>();
            if (lam > lam_skip<T>(a)) {
                r = event_draw(a.keys, id, tm.step, k);
                T uw, vw;
                Uniform<T>::draw(r.x, r.y, uw, vw);
                dth = f_div(Uniform<T>::neglog(uw, vw), lam);
            }
            bool no_event;
            T h;
            if constexpr (FRESH && sizeof(T) == 4) { no_event = dth >= a.dt_f_gt; h = a.dt_f; }
            else if constexpr (FRESH) { no_event = dth > a.dt; h = a.dt; }
            else if constexpr (sizeof(T) == 4) {
                // as in the lepton pass: the FP64 test decided in FP32 outside a margin
                const float rf = __double2float_rn(a.dt - tau);
                const float marg = fmaf(rf, 0x1p-20f, a.dt_f * 0x1p-40f);
                if (dth > rf + marg) no_event = true;
                else if (dth < rf - marg) no_event = false;
                else no_event = tau + (double)dth > a.dt;
                h = rf;
            } else { no_event = tau + (double)dth > a.dt; h = (T)(a.dt - tau); }
            if (no_event) {
                x[0] += nx * h; x[1] += ny * h; x[2] += nz * h;
            } else {
                x[0] += nx * dth; x[1] += ny * dth; x[2] += nz * dth;
                if constexpr (FRESH) tau = (double)dth;
                else tau += (double)dth;
                pair_create<T>(a, tm, icdf, x, kv, k0, nx, ny, nz, tau, w, id, k, make_uint2(r.z, r.w), n64);
                k = 1;
                st<T>(S.w, i, (T)0);       // the photon is eliminated
                S.nev[i] += k;
            }
        }
    }
    return true;
}

// Photon push: straight flight, pair creation at the event, the photon is
// removed (weight 0) and the pair appended.
template <class T, bool FRESH>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 4 : 1)) k_photon_pass(PassArgs a) {
    if ((unsigned long long)blockIdx.x * blockDim.x >= a.ctl->end[2] - a.ctl->begin[2]) return;   // no photon here
    __shared__ __align__(16) T s_coef[RateWords<T>::N];
    __shared__ StepTime s_tm;
    for (int i = threadIdx.x; i < RateWords<T>::N; i += blockDim.x) s_coef[i] = reinterpret_cast<const T *>(a.coef)[i];
    if (threadIdx.x == 0) s_tm = load_step_time(a);
    __syncthreads();
    const StepTime &tm = s_tm;
    DevCtl *ctl = a.ctl;
    // 32-bit indices (a species holds fewer than 2^31 entries)
    const unsigned b = (unsigned)ctl->begin[2], n = (unsigned)(ctl->end[2] - ctl->begin[2]);
    const T *icdf = reinterpret_cast<const T *>(a.icdf_pair);
    const SpeciesDev &S = a.sp[2];
    unsigned long long my_steps = 0, my_ev = 0;
    unsigned my_max = 0, n64 = 0;
    const Phase<T> ph0 = time_phase<T, StepTime>(tm, 0.0);
    // FP32 step-start pass: each thread stages its next photon in shared
    // memory (two buffers) while it works on the current one
    constexpr bool STAGE = FRESH && sizeof(T) == 4;
    constexpr int NB = STAGE ? 2 : 1, NF = STAGE ? 9 : 1, NT = STAGE ? LB : 1;
    __shared__ __align__(16) float stg[NB][NF][NT];       // w x y z kx ky kz id(2 words)
    const unsigned stride = gridDim.x * blockDim.x;
    auto stage = [&](unsigned jj, int buf) {
        if constexpr (STAGE) {
            const unsigned ii = b + jj;
            const int t = threadIdx.x;
            cp_async4(&stg[buf][0][t], reinterpret_cast<const float *>(S.w) + ii);
            cp_async4(&stg[buf][1][t], reinterpret_cast<const float *>(S.x) + ii);
            cp_async4(&stg[buf][2][t], reinterpret_cast<const float *>(S.y) + ii);
            cp_async4(&stg[buf][3][t], reinterpret_cast<const float *>(S.z) + ii);
            cp_async4(&stg[buf][4][t], reinterpret_cast<const float *>(S.px) + ii);
            cp_async4(&stg[buf][5][t], reinterpret_cast<const float *>(S.py) + ii);
            cp_async4(&stg[buf][6][t], reinterpret_cast<const float *>(S.pz) + ii);
            cp_async4(&stg[buf][7][t], S.id + ii);          // id: two 4-byte halves
            cp_async4(&stg[buf][8][t], reinterpret_cast<const unsigned *>(S.id + ii) + 1);
        }
    };
    const unsigned j0 = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (STAGE) {
        if (j0 < n) stage(j0, 0);
        cp_async_commit();
    }
    int buf = 0;
    for (unsigned j = j0; j < n; j += stride, buf ^= 1) {
        const unsigned i = b + j;
        T w, x[3], kx, ky, kz;
        unsigned long long id;
        if constexpr (STAGE) {
            if (j + stride < n) stage(j + stride, buf ^ 1);
            cp_async_commit();
            cp_async_wait_prev();                // this thread's copies of photon j have landed
            const int t = threadIdx.x;
            w = stg[buf][0][t];
            x[0] = stg[buf][1][t]; x[1] = stg[buf][2][t]; x[2] = stg[buf][3][t];
            kx = stg[buf][4][t]; ky = stg[buf][5][t]; kz = stg[buf][6][t];
            id = (unsigned long long)__float_as_uint(stg[buf][7][t]) |
                 ((unsigned long long)__float_as_uint(stg[buf][8][t]) << 32);
        } else {
            // all loads issued together (live photons are the rule: the photons
            // that converted were removed at the end of the previous step)
            w = ld<T>(S.w, i);
            x[0] = ld<T>(S.x, i); x[1] = ld<T>(S.y, i); x[2] = ld<T>(S.z, i);
            kx = ld<T>(S.px, i); ky = ld<T>(S.py, i); kz = ld<T>(S.pz, i);
            id = __ldg(S.id + i);
        }
        unsigned k;
        if (!photon_step<T, FRESH>(a, tm, s_coef, icdf, ph0, S, i, w, x, kx, ky, kz, id, k, n64)) continue;
        st<T>(S.x, i, x[0]); st<T>(S.y, i, x[1]); st<T>(S.z, i, x[2]);
        ++my_steps;
        my_ev += k;
        my_max = max(my_max, k);
    }
    __syncwarp();
    flush_stats(ctl, my_steps, my_ev, my_max, true, n64);
}


// ---- the accumulated-optical-depth method (QED_METHOD_OPTICAL_DEPTH) ----
// Per particle and step: the rate at the step start; an optical depth not
// drawn yet (od <= 0) is drawn as -ln u from Philox(id, step, OD_DRAW); od
// decreases by lambda dt; the particle is pushed by dt; if od <= 0 the event
// happens at the end of the step (chi at the end point, energy from
// Philox(id, step, 0) words 2-3) and a fresh od = -ln u from words 0-1.  At
// most one event per particle and step; the children start at the next step.
// od is held in the context's precision: a particle that does not convert
// draws no random number and does no FP64 arithmetic in FP32 mode.
constexpr unsigned OD_DRAW = 0xFFFFFFFEu;

// -ln u from words 0-1 of a draw (the FP32 form keeps full relative precision
// for u near 1)
template <class T> __device__ __forceinline__ T od_exp1(const uint4 &r) {
    T u, v;
    Uniform<T>::draw(r.x, r.y, u, v);
    return Uniform<T>::neglog(u, v);
}

// the step in the working precision (FP32: rounded once on the host)
template <class T> __device__ __forceinline__ T dt_of(const PassArgs &a);
template <> __device__ __forceinline__ float dt_of<float>(const PassArgs &a) { return a.dt_f; }
template <> __device__ __forceinline__ double dt_of<double>(const PassArgs &a) { return a.dt; }

// od after this step's decrement, drawn first when not drawn yet.  The
// product is rounded on its own (no contraction), as in the oracle.
template <class T>
__device__ __forceinline__ T od_advance(const PassArgs &a, unsigned step, unsigned long long id, T od, T lam) {
    if (!(od > (T)0)) od = od_exp1<T>(event_draw(a.keys, id, step, OD_DRAW));
    return od - mul_rn<T>(lam, dt_of<T>(a));
}

template <class T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 4 : 1)) k_lepton_od(PassArgs a) {
    __shared__ __align__(16) T s_coef[RateWords<T>::N];
    __shared__ StepTime s_tm;
    for (int i = threadIdx.x; i < RateWords<T>::N; i += blockDim.x) s_coef[i] = reinterpret_cast<const T *>(a.coef)[i];
    if (threadIdx.x == 0) s_tm = load_step_time(a);
    __syncthreads();
    const StepTime &tm = s_tm;
    DevCtl *ctl = a.ctl;
    const unsigned long long b0 = ctl->begin[0], n0 = ctl->end[0] - b0;
    const unsigned long long b1 = ctl->begin[1], n1 = ctl->end[1] - b1;
    const unsigned long long n = n0 + n1;
    const LeptonCtx<T> c{a, ctl, s_coef, reinterpret_cast<const T *>(a.icdf_em), ctl->capacity[2], (T)(ALPHA * RS),
                         tm, time_phase<T, StepTime>(tm, 0.0)};
    unsigned long long my_steps = 0, my_ev = 0;
    unsigned my_max = 0, n64 = 0;
    for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const int s = j < n0 ? 0 : 1;
        const unsigned long long i = s == 0 ? b0 + j : b1 + (j - n0);
        const SpeciesDev &S = a.sp[s];
        const T w = ld<T>(S.w, i);
        if (!(w > (T)0)) continue;
        T x[3] = {ld<T>(S.x, i), ld<T>(S.y, i), ld<T>(S.z, i)};
        T p[3] = {ld<T>(S.px, i), ld<T>(S.py, i), ld<T>(S.pz, i)};
        const unsigned long long id = __ldg(S.id + i);
        T od = ld<T>(S.od, i);
        ++my_steps;
        T E[3], B[3];
        field_at<T>(a, x, c.ph0, E, B);
        T gam, chi, p2;
        lepton_chi<T>(p, E, B, gam, chi, p2, n64, a.field_zero);
        const T lam = p2 > (T)0 ? c.alpha_r / gam * rate_em<T>(c.coef, chi) : (T)0;
        od = od_advance<T>(a, tm.step, id, od, lam);
        const T qch = s == 0 ? (T)-1 : (T)1;
        boris<T>(x, p, qch, E, B, dt_of<T>(a), a.field_zero == 1, id, tm.step, 0u);
        unsigned k = 0;
        if (od <= (T)0) {
            // the event at the end of the step
            field_tau<T>(a, tm, x, a.dt, E, B);
            lepton_chi<T>(p, E, B, gam, chi, p2, n64, a.field_zero);
            const uint4 r = event_draw(a.keys, id, tm.step, 0u);
            T om, ue, ve;
            Uniform<T>::draw(r.z, r.w, ue, ve);
            const T delta = sample_emission<T>(c.icdf, chi, ue, ve, &om);
            emit_with<T>(c, x, p, a.dt, w, id, 0u, gam, p2, delta, om);
            od = od_exp1<T>(r);
            k = 1;
        }
        st<T>(S.x, i, x[0]); st<T>(S.y, i, x[1]); st<T>(S.z, i, x[2]);
        st<T>(S.px, i, p[0]); st<T>(S.py, i, p[1]); st<T>(S.pz, i, p[2]);
        st<T>(S.od, i, od);
        if (k) S.nev[i] += 1u;
        my_ev += k;
        my_max = max(my_max, k);
    }
    __syncwarp();
    flush_stats(ctl, my_steps, my_ev, my_max, false, n64);
}

template <class T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 ? 4 : 1)) k_photon_od(PassArgs a) {
    __shared__ __align__(16) T s_coef[RateWords<T>::N];
    __shared__ StepTime s_tm;
    for (int i = threadIdx.x; i < RateWords<T>::N; i += blockDim.x) s_coef[i] = reinterpret_cast<const T *>(a.coef)[i];
    if (threadIdx.x == 0) s_tm = load_step_time(a);
    __syncthreads();
    const StepTime &tm = s_tm;
    DevCtl *ctl = a.ctl;
    const unsigned long long b = ctl->begin[2], n = ctl->end[2] - b;
    const unsigned long long cap_e = ctl->capacity[0], cap_p = ctl->capacity[1];
    const T *icdf = reinterpret_cast<const T *>(a.icdf_pair);
    const T alpha_r = (T)(ALPHA * RS);
    const SpeciesDev &S = a.sp[2];
    unsigned long long my_steps = 0, my_ev = 0;
    unsigned my_max = 0, n64 = 0;
    const Phase<T> ph0 = time_phase<T, StepTime>(tm, 0.0);
    // FP32: each thread stages its next photon in shared memory (two
    // buffers) while it works on the current one, as in the step-start pass
    constexpr bool STAGE = sizeof(T) == 4;
    constexpr int NB = STAGE ? 2 : 1, NF = STAGE ? 10 : 1, NT = STAGE ? 256 : 1;
    __shared__ __align__(16) float stg[NB][NF][NT];       // w x y z kx ky kz id(2 words) od
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    auto stage = [&](unsigned long long jj, int buf) {
        if constexpr (STAGE) {
            const unsigned long long ii = b + jj;
            const int t = threadIdx.x;
            cp_async4(&stg[buf][0][t], reinterpret_cast<const float *>(S.w) + ii);
            cp_async4(&stg[buf][1][t], reinterpret_cast<const float *>(S.x) + ii);
            cp_async4(&stg[buf][2][t], reinterpret_cast<const float *>(S.y) + ii);
            cp_async4(&stg[buf][3][t], reinterpret_cast<const float *>(S.z) + ii);
            cp_async4(&stg[buf][4][t], reinterpret_cast<const float *>(S.px) + ii);
            cp_async4(&stg[buf][5][t], reinterpret_cast<const float *>(S.py) + ii);
            cp_async4(&stg[buf][6][t], reinterpret_cast<const float *>(S.pz) + ii);
            cp_async4(&stg[buf][7][t], S.id + ii);
            cp_async4(&stg[buf][8][t], reinterpret_cast<const unsigned *>(S.id + ii) + 1);
            cp_async4(&stg[buf][9][t], reinterpret_cast<const float *>(S.od) + ii);
        }
    };
    const unsigned long long j0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (STAGE) {
        if (j0 < n) stage(j0, 0);
        cp_async_commit();
    }
    int buf = 0;
    for (unsigned long long j = j0; j < n; j += stride, buf ^= 1) {
        const unsigned long long i = b + j;
        T w, x[3], kv[3], od;
        unsigned long long id;
        if constexpr (STAGE) {
            if (j + stride < n) stage(j + stride, buf ^ 1);
            cp_async_commit();
            cp_async_wait_prev();                // this thread's copies of photon j have landed
            const int t = threadIdx.x;
            w = stg[buf][0][t];
            x[0] = stg[buf][1][t]; x[1] = stg[buf][2][t]; x[2] = stg[buf][3][t];
            kv[0] = stg[buf][4][t]; kv[1] = stg[buf][5][t]; kv[2] = stg[buf][6][t];
            id = (unsigned long long)__float_as_uint(stg[buf][7][t]) |
                 ((unsigned long long)__float_as_uint(stg[buf][8][t]) << 32);
            od = stg[buf][9][t];
        } else {
            w = ld<T>(S.w, i);
            x[0] = ld<T>(S.x, i); x[1] = ld<T>(S.y, i); x[2] = ld<T>(S.z, i);
            kv[0] = ld<T>(S.px, i); kv[1] = ld<T>(S.py, i); kv[2] = ld<T>(S.pz, i);
            id = __ldg(S.id + i);
            od = ld<T>(S.od, i);
        }
        if (!(w > (T)0)) continue;
        ++my_steps;
        const T k0 = f_sqrt(kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
        unsigned k = 0;
        if (k0 > (T)0) {
            const T inv = f_div((T)1, k0);
            const T nx = kv[0] * inv, ny = kv[1] * inv, nz = kv[2] * inv;
            T E[3], B[3];
            field_at<T>(a, x, ph0, E, B);
            T chi = photon_chi<T>(k0, kv, E, B, n64, a.field_zero);
            const T lam = alpha_r / k0 * rate_pair<T>(s_coef, chi);
            od = od_advance<T>(a, tm.step, id, od, lam);
            const T h = dt_of<T>(a);
            x[0] += nx * h; x[1] += ny * h; x[2] += nz * h;
            if (od <= (T)0) {
                // pair creation at the end of the step
                field_tau<T>(a, tm, x, a.dt, E, B);
                chi = photon_chi<T>(k0, kv, E, B, n64, a.field_zero);
                const uint4 r = event_draw(a.keys, id, tm.step, 0u);
                T om, ue, ve;
                Uniform<T>::draw(r.z, r.w, ue, ve);
                const T delta = sample_pair<T>(icdf, chi, ue, ve, &om);
                T em = delta * k0, ep = om * k0;
                em = em < (T)1 ? (T)1 : em;
                ep = ep < (T)1 ? (T)1 : ep;
                const T pm = f_sqrt((em - (T)1) * (em + (T)1)), pp = f_sqrt((ep - (T)1) * (ep + (T)1));
                const uint4 rid = event_draw(a.seed ^ CHILD_KEY_XOR, id, tm.step, 0u);
                const unsigned long long se = warp_append(&ctl->count[0], 1);
                const unsigned long long sp = warp_append(&ctl->count[1], 1);
                if (se < cap_e) {
                    const SpeciesDev &P = a.sp[0];
                    st<T>(P.x, se, x[0]); st<T>(P.y, se, x[1]); st<T>(P.z, se, x[2]);
                    st<T>(P.px, se, pm * nx); st<T>(P.py, se, pm * ny); st<T>(P.pz, se, pm * nz);
                    st<T>(P.w, se, w);
                    P.id[se] = (unsigned long long)rid.x | ((unsigned long long)rid.y << 32);
                    P.nev[se] = 0u;
                    st<T>(P.od, se, (T)0);
                } else {
                    note_overflow(ctl, 0, se);
                }
                if (sp < cap_p) {
                    const SpeciesDev &P = a.sp[1];
                    st<T>(P.x, sp, x[0]); st<T>(P.y, sp, x[1]); st<T>(P.z, sp, x[2]);
                    st<T>(P.px, sp, pp * nx); st<T>(P.py, sp, pp * ny); st<T>(P.pz, sp, pp * nz);
                    st<T>(P.w, sp, w);
                    P.id[sp] = (unsigned long long)rid.z | ((unsigned long long)rid.w << 32);
                    P.nev[sp] = 0u;
                    st<T>(P.od, sp, (T)0);
                } else {
                    note_overflow(ctl, 1, sp);
                }
                w = (T)0;
                k = 1;
            }
        }
        st<T>(S.x, i, x[0]); st<T>(S.y, i, x[1]); st<T>(S.z, i, x[2]);
        st<T>(S.od, i, od);
        if (k) { st<T>(S.w, i, w); S.nev[i] += 1u; }
        my_ev += k;
        my_max = max(my_max, k);
    }
    __syncwarp();
    flush_stats(ctl, my_steps, my_ev, my_max, true, n64);
}

// ---- host side ----
template <class K>
inline qed_status timed_launch(qed_ctx *ctx, int which, K launch) {
    if (!ctx->cfg.profile) {
        launch();
        return QED_OK;
    }
    if (ctx->ev_used[which] == qed_ctx::EVN) {
        qed_status e = sfq_drain_events(ctx);
        if (e != QED_OK) return e;
    }
    const int i = ctx->ev_used[which]++;
    SFQ_CUDA(cudaEventRecord(ctx->ev[which][i][0], ctx->stream));
    launch();
    SFQ_CUDA(cudaEventRecord(ctx->ev[which][i][1], ctx->stream));
    return QED_OK;
}

// Persistent grids: one wave of resident blocks (SM count x blocks per SM
// from the occupancy calculator unless the configuration fixes it).
template <class K> inline int resident_blocks(const qed_ctx *ctx, K kernel, int threads) {
    int per_sm = ctx->cfg.blocks_per_sm;
    if (per_sm <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    return ctx->sm_count * per_sm;
}

// a group of launches timed as one (compaction, leveling)
template <class F> inline qed_status timed_block(qed_ctx *ctx, int which, F body) {
    if (!ctx->cfg.profile) return body();
    if (ctx->ev_used[which] == qed_ctx::EVN) {
        qed_status e = sfq_drain_events(ctx);
        if (e != QED_OK) return e;
    }
    const int i = ctx->ev_used[which]++;
    SFQ_CUDA(cudaEventRecord(ctx->ev[which][i][0], ctx->stream));
    qed_status e = body();
    SFQ_CUDA(cudaEventRecord(ctx->ev[which][i][1], ctx->stream));
    return e;
}

template <class K> inline int resident_blocks_smem(const qed_ctx *ctx, K kernel, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return ctx->sm_count * per_sm;
}

template <class T, bool FRESH>
qed_status launch_pass_t(qed_ctx *ctx, PassArgs &a, bool photons) {
    const int threads = LB;
    const int bp = resident_blocks(ctx, k_photon_pass<T, FRESH>, threads);
    cudaStream_t st = ctx->stream;
    qed_status e;
    if (a.mlp_w16) {
        static bool attr_set = false;   // the attribute is per function, set once
        if (!attr_set) {
            SFQ_CUDA(cudaFuncSetAttribute(k_lepton_pass<T, FRESH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          MLP_SMEM_BYTES));
            attr_set = true;
        }
        const int bl = resident_blocks_smem(ctx, k_lepton_pass<T, FRESH, true>, threads, MLP_SMEM_BYTES);
        e = timed_launch(ctx, 0, [&] { k_lepton_pass<T, FRESH, true><<<bl, threads, MLP_SMEM_BYTES, st>>>(a); });
    } else {
        const int bl = resident_blocks(ctx, k_lepton_pass<T, FRESH, false>, threads);
        e = timed_launch(ctx, 0, [&] { k_lepton_pass<T, FRESH, false><<<bl, threads, 0, st>>>(a); });
    }
    if (e != QED_OK) return e;
    SFQ_LAUNCHED(ctx, 1);
    if (photons) {
        e = timed_launch(ctx, 1, [&] { k_photon_pass<T, FRESH><<<bp, threads, 0, st>>>(a); });
        if (e != QED_OK) return e;
        SFQ_LAUNCHED(ctx, 1);
    }
    SFQ_CUDA(cudaGetLastError());
    return QED_OK;
}

// the optical-depth method: one launch per species kind and step
template <class T>
qed_status launch_od(qed_ctx *ctx, PassArgs &a, bool photons) {
    cudaStream_t st = ctx->stream;
    const int bl = resident_blocks(ctx, k_lepton_od<T>, 256);
    qed_status e = timed_launch(ctx, 0, [&] { k_lepton_od<T><<<bl, 256, 0, st>>>(a); });
    if (e != QED_OK) return e;
    SFQ_LAUNCHED(ctx, 1);
    if (photons) {
        const int bp = resident_blocks(ctx, k_photon_od<T>, 256);
        e = timed_launch(ctx, 1, [&] { k_photon_od<T><<<bp, 256, 0, st>>>(a); });
        if (e != QED_OK) return e;
        SFQ_LAUNCHED(ctx, 1);
    }
    SFQ_CUDA(cudaGetLastError());
    return QED_OK;
}

template <class T>
qed_status launch_pass(qed_ctx *ctx, PassArgs &a, bool photons) {
    return a.pass == 0 ? launch_pass_t<T, true>(ctx, a, photons) : launch_pass_t<T, false>(ctx, a, photons);
}


}  // namespace SFQ_PASS_NS
}  // namespace sfq
