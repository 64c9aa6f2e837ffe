// K2 / K3: the per-particle QED step (arXiv:2409.17299 Sec. 3, Algorithms 1-2).
//
// One pass kernel per particle kind.  Each thread takes one particle of the
// pass range (grid-stride), runs Algorithm 1 for it to the end of the step
// (rate -> waiting time -> Boris push -> event), and appends every particle
// it creates with a warp-aggregated atomic.  Newborns carry their birth
// clock and are pushed by the next pass (Algorithm 2): leptons and photons
// are swept alternately until a pass creates nothing.
#include <math.h>
#include <string.h>

#include <chrono>

#include "sfqed_device.cuh"
#include "sfqed_internal.h"

namespace sfq {
namespace {

// Gridded field: [6][nodes] (caller's layout) -> [nodes][8] (two pads)
template <class T>
__global__ void k_grid_interleave(const T *src, T *dst, long long nodes) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
#pragma unroll
    for (int c = 0; c < 6; ++c) dst[8 * n + c] = src[c * nodes + n];
    dst[8 * n + 6] = (T)0;
    dst[8 * n + 7] = (T)0;
}

// Newborn passes of one step after which the step gives up (QED_ERR_TIMEOUT),
// unless the configuration sets another limit.
constexpr unsigned long long PASS_LIMIT = 100000;
static unsigned long long pass_limit_of(const qed_ctx *ctx) {
    return ctx->cfg.pass_limit > 0 ? (unsigned long long)ctx->cfg.pass_limit : PASS_LIMIT;
}

__device__ __forceinline__ bool ctl_stopped(const DevCtl *ctl) {
    return ctl->overflow || ctl->timeout || ctl->bad_index;
}

// Opens the next step (index ctl->step_next): its time t_n = step dt and the
// phase reduced mod 2 pi (the pass kernels read both from the control block),
// and the pass ranges: every particle present.  After an overflow or a failed
// device check the ranges are empty, so the rest of the enqueued work does
// nothing.
__global__ void k_step_begin(DevCtl *ctl, double dt) {
    const unsigned long long step = ctl->step_next;
    ctl->step_next = step + 1;
    const double t_n = (double)step * dt;
    ctl->sv_t_n = t_n;
    ctl->sv_t_red_f = (float)fmod(t_n, 2.0 * 3.14159265358979323846);
    ctl->sv_step = (unsigned)step;
    ctl->step_passes = 0;
    const bool stop = ctl_stopped(ctl);
    for (int s = 0; s < 3; ++s) {
        ctl->begin[s] = 0;
        ctl->end[s] = stop ? 0 : min(ctl->count[s], ctl->capacity[s]);
    }
}

__global__ void k_set_step(DevCtl *ctl, unsigned long long step) { ctl->step_next = step; }

__global__ void k_set_timeout(DevCtl *ctl) { ctl->timeout = 1; }

// Pass ranges of the next newborn pass: the particles appended since the
// previous pass.  In a step graph it also sets the condition of the loop
// over passes (the only setter): another pass while one found work, at most
// ctl->pass_limit per step (then the step is marked as timed out).
__device__ __forceinline__ unsigned long long pass_setup(DevCtl *ctl) {
    unsigned long long more = 0;
    for (int s = 0; s < 3; ++s) {
        const unsigned long long e = min(ctl->count[s], ctl->capacity[s]);
        ctl->begin[s] = ctl->end[s];
        ctl->end[s] = e;
        if (e > ctl->begin[s]) more = 1;
    }
    if (ctl_stopped(ctl)) {
        more = 0;
        for (int s = 0; s < 3; ++s) ctl->begin[s] = ctl->end[s];
    }
    ctl->more = more;
    ctl->passes += more;
    ctl->step_passes += more;
    return more;
}

__global__ void k_pass_setup(DevCtl *ctl) { pass_setup(ctl); }

__global__ void k_pass_setup_cond(DevCtl *ctl, cudaGraphConditionalHandle h, int in_body) {
    unsigned long long more = pass_setup(ctl);
    const unsigned long long limit = ctl->pass_limit ? ctl->pass_limit : PASS_LIMIT;
    if (more && ctl->step_passes > limit) {
        ctl->timeout = 1;
        more = 0;
        for (int s = 0; s < 3; ++s) ctl->begin[s] = ctl->end[s];
    }
    if (in_body) ctl->graph_kernels += 3;       // the loop body: two passes and this kernel
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---- component kernels for the parity tests ----
__global__ void k_philox(const uint4 *ctr, long long n, uint2 key, uint4 *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

template <class T>
__global__ void k_eval_rate(const T *coef, int is_photon, const double *chi, long long n, double *F) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T c = (T)chi[i];
    F[i] = (double)(is_photon ? rate_pair<T>(coef, c) : rate_em<T>(coef, c));
}

// chi of n particles (p, E, B as n x 3 doubles) in the mode's precision
template <class T>
__global__ void k_eval_chi(int is_photon, const double *p, const double *E, const double *B, long long n,
                           double *chi, unsigned long long *n64_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T pv[3] = {(T)p[3 * i], (T)p[3 * i + 1], (T)p[3 * i + 2]};
    const T Ev[3] = {(T)E[3 * i], (T)E[3 * i + 1], (T)E[3 * i + 2]};
    const T Bv[3] = {(T)B[3 * i], (T)B[3 * i + 1], (T)B[3 * i + 2]};
    unsigned n64 = 0;
    T c;
    if (is_photon) {
        const T k0 = m_sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
        c = photon_chi<T>(k0, pv, Ev, Bv, n64);
    } else {
        T gam, p2;
        lepton_chi<T>(pv, Ev, Bv, gam, c, p2, n64);
    }
    chi[i] = (double)c;
    if (n64) atomicAdd(n64_out, (unsigned long long)n64);
}

template <class T>
__global__ void k_sample(const T *tab, int is_photon, const double *chi, const double *u, long long n,
                         double *delta, double *om) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T o;
    const T uu = (T)u[i], vv = (T)(1.0 - u[i]);
    const T d = is_photon ? sample_pair<T>(tab, (T)chi[i], uu, vv, &o) : sample_emission<T>(tab, (T)chi[i], uu, vv, &o);
    delta[i] = (double)d;
    if (om) om[i] = (double)o;
}

}  // namespace
}  // namespace sfq

using namespace sfq;

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static qed_status check_species(const qed_species &s) {
    const void *ptrs[] = {s.x, s.y, s.z, s.px, s.py, s.pz, s.w, s.id, s.nevents};
    if (s.capacity < 0 || s.count < 0 || s.count > s.capacity) return QED_ERR_INVALID;
    if (s.capacity >= (int64_t)1 << 31) return QED_ERR_INVALID;   // the pass kernels index in 31 bits
    if (s.capacity == 0) return QED_OK;
    for (const void *q : ptrs)
        if (!q || !aligned16(q)) return QED_ERR_INVALID;
    return QED_OK;
}

static qed_status ensure_tau(qed_ctx *ctx, int s, int64_t cap) {
    if (ctx->tau_cap[s] >= cap) return QED_OK;
    if (ctx->tau[s]) SFQ_CUDA(cudaFreeAsync(ctx->tau[s], ctx->stream));
    ctx->tau[s] = nullptr;
    ctx->tau_cap[s] = 0;
    if (cudaMallocAsync(&ctx->tau[s], sizeof(double) * (size_t)(cap > 0 ? cap : 1), ctx->stream) != cudaSuccess)
        return QED_ERR_NOMEM;
    ctx->tau_cap[s] = cap;
    return QED_OK;
}

static size_t elem_bytes(const qed_ctx *ctx) { return ctx->cfg.precision == QED_FP32 ? 4 : 8; }

// Save / restore the particle state at the start of a call (overflow replay).
static qed_status snapshot(qed_ctx *ctx, qed_particles *p, bool restore) {
    const size_t eb = elem_bytes(ctx);
    size_t need = 0;
    for (int s = 0; s < 3; ++s) need += (size_t)p->s[s].count * (7 * eb + 8 + 4 + (ctx->od[s] ? eb : 0));
    if (!restore && (int64_t)need > ctx->snap_bytes) {
        if (ctx->snap) SFQ_CUDA(cudaFreeAsync(ctx->snap, ctx->stream));
        ctx->snap = nullptr;
        ctx->snap_bytes = 0;
        if (cudaMallocAsync(&ctx->snap, need + 16, ctx->stream) != cudaSuccess) return QED_ERR_NOMEM;
        ctx->snap_bytes = (int64_t)need;
    }
    char *b = static_cast<char *>(ctx->snap);
    for (int s = 0; s < 3; ++s) {
        const qed_species &S = p->s[s];
        const size_t n = (size_t)S.count;
        if (!n) continue;
        void *arr[] = {S.x, S.y, S.z, S.px, S.py, S.pz, S.w};
        for (void *q : arr) {
            if (restore) SFQ_CUDA(cudaMemcpyAsync(q, b, n * eb, cudaMemcpyDeviceToDevice, ctx->stream));
            else SFQ_CUDA(cudaMemcpyAsync(b, q, n * eb, cudaMemcpyDeviceToDevice, ctx->stream));
            b += n * eb;
        }
        if (restore) SFQ_CUDA(cudaMemcpyAsync(S.id, b, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        else SFQ_CUDA(cudaMemcpyAsync(b, S.id, n * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        b += n * 8;
        if (restore) SFQ_CUDA(cudaMemcpyAsync(S.nevents, b, n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        else SFQ_CUDA(cudaMemcpyAsync(b, S.nevents, n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        b += n * 4;
        if (ctx->od[s]) {
            if (restore) SFQ_CUDA(cudaMemcpyAsync(ctx->od[s], b, n * eb, cudaMemcpyDeviceToDevice, ctx->stream));
            else SFQ_CUDA(cudaMemcpyAsync(b, ctx->od[s], n * eb, cudaMemcpyDeviceToDevice, ctx->stream));
            b += n * eb;
        }
    }
    return QED_OK;
}

static qed_status read_ctl(qed_ctx *ctx) {
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    const auto t0 = std::chrono::steady_clock::now();
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->sync_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return QED_OK;
}

// Profiling: event pairs around the push kernels, drained into kernel_ms.
qed_status sfq_drain_events(qed_ctx *ctx) {
    for (int k = 0; k < 4; ++k) {
        for (int i = 0; i < ctx->ev_used[k]; ++i) {
            float ms = 0.f;
            SFQ_CUDA(cudaEventSynchronize(ctx->ev[k][i][1]));
            SFQ_CUDA(cudaEventElapsedTime(&ms, ctx->ev[k][i][0], ctx->ev[k][i][1]));
            ctx->kernel_ms[k] += ms;
        }
        ctx->ev_used[k] = 0;
    }
    return QED_OK;
}

static qed_status ensure_events(qed_ctx *ctx) {
    if (ctx->ev_ready) return QED_OK;
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < qed_ctx::EVN; ++i)
            for (int j = 0; j < 2; ++j) SFQ_CUDA(cudaEventCreate(&ctx->ev[k][i][j]));
    ctx->ev_ready = true;
    return QED_OK;
}

// a group of launches timed as one (compaction, leveling)
template <class F> static qed_status timed_block(qed_ctx *ctx, int which, F body) {
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

// the pass kernels of the field's variant (analytic descriptors or grid)
template <class T>
static qed_status launch_pass(qed_ctx *ctx, PassArgs &a, bool photons) {
    if (a.field_kind == QED_FIELD_GRID) return pass_grid::launch_pass<T>(ctx, a, photons);
    return pass_analytic::launch_pass<T>(ctx, a, photons);
}

template <class T>
static qed_status launch_od(qed_ctx *ctx, PassArgs &a, bool photons) {
    if (a.field_kind == QED_FIELD_GRID) return pass_grid::launch_od<T>(ctx, a, photons);
    return pass_analytic::launch_od<T>(ctx, a, photons);
}

// ---- the captured PIC step ----
// One step as a CUDA graph: the step-begin kernel, the step-start passes,
// then (a cascade) a while node sweeping the newborns until a pass creates
// nothing (Algorithm 2), then each species' merge step (leveling and removal
// of dead entries) decided on the device.  Every kernel reads its ranges and
// the step's time from the control block, so one graph serves every step and
// no step needs the host: a batch of steps is a run of graph launches.  The
// graph is rebuilt when the bound arrays, capacities, field or step change.
struct StepGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    PassArgs args;           // the kernel arguments captured (compared byte-wise)
    int64_t cap[3];
    double dt;
    int top_kernels;         // kernel nodes outside the conditional bodies
};

void sfq_step_graph_free(qed_ctx *ctx) {
    StepGraph *G = static_cast<StepGraph *>(ctx->step_graph);
    if (!G) return;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->g) cudaGraphDestroy(G->g);
    delete G;
    ctx->step_graph = nullptr;
}

template <class T>
static qed_status build_step_graph(qed_ctx *ctx, const PassArgs &args, qed_particles *p, double dt, StepGraph *G) {
    const bool cascade = ctx->cfg.push_photons != 0;
    const bool od_method = ctx->cfg.event_method == QED_METHOD_OPTICAL_DEPTH;
    const bool loop = cascade && !od_method;
    GraphBuild gb;
    if (cudaGraphCreate(&gb.g, 0) != cudaSuccess) return QED_ERR_CUDA;
    gb.st = ctx->cap_stream;
    const cudaStream_t saved = ctx->stream;
    const int64_t launches = ctx->launches;
    ctx->stream = gb.st;                   // the launchers issue on ctx->stream
    PassArgs a = args;
    qed_status rc = QED_OK;
    cudaGraphConditionalHandle h_pass = 0;
    do {
        if (loop && cudaGraphConditionalHandleCreate(&h_pass, gb.g, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
            rc = QED_ERR_CUDA;
            break;
        }
        cudaError_t e = gb.capture(gb.g, [&] {
            k_step_begin<<<1, 1, 0, ctx->stream>>>(ctx->ctl, dt);
            a.pass = 0;
            const qed_status q = od_method ? launch_od<T>(ctx, a, cascade) : launch_pass<T>(ctx, a, cascade);
            if (q != QED_OK) return q;
            if (loop) k_pass_setup_cond<<<1, 1, 0, ctx->stream>>>(ctx->ctl, h_pass, 0);
            return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
        });
        if (e != cudaSuccess) {
            rc = QED_ERR_CUDA;
            break;
        }
        gb.top_kernels = 2 + (cascade ? 1 : 0) + (loop ? 1 : 0);
        if (loop) {
            cudaGraph_t body;
            if (gb.conditional(h_pass, cudaGraphCondTypeWhile, &body) != cudaSuccess) {
                rc = QED_ERR_CUDA;
                break;
            }
            e = gb.capture(body, [&] {
                a.pass = 1;
                const qed_status q = launch_pass<T>(ctx, a, true);
                if (q != QED_OK) return q;
                k_pass_setup_cond<<<1, 1, 0, ctx->stream>>>(ctx->ctl, h_pass, 1);
                return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
            });
            if (e != cudaSuccess) {
                rc = QED_ERR_CUDA;
                break;
            }
        }
        // merge step (Sec. 4.2): converted photons removed, each species
        // leveled when its count exceeds the cap
        if (cascade || ctx->cfg.thin_cap > 0)
            for (int s = 0; s < 3 && rc == QED_OK; ++s) rc = sfq_capture_merge(ctx, gb, &p->s[s], s, cascade && s == 2);
    } while (0);
    ctx->stream = saved;
    ctx->launches = launches;
    if (rc == QED_OK && cudaGraphInstantiate(&G->exec, gb.g, 0) != cudaSuccess) rc = QED_ERR_CUDA;
    if (rc != QED_OK) {
        cudaGraphDestroy(gb.g);
        cudaGetLastError();                        // clear a failed call's error
        return rc;
    }
    G->g = gb.g;
    G->args = args;
    for (int s = 0; s < 3; ++s) G->cap[s] = p->s[s].capacity;
    G->dt = dt;
    G->top_kernels = gb.top_kernels;
    return QED_OK;
}

// The step graph for these arguments (built or rebuilt when needed), or null
// when graphs with conditional nodes are not available (host-driven steps).
template <class T>
static StepGraph *step_graph_for(qed_ctx *ctx, const PassArgs &a, qed_particles *p, double dt) {
    if (ctx->step_graph_failed) return nullptr;
    StepGraph *G = static_cast<StepGraph *>(ctx->step_graph);
    bool same = G && G->dt == dt && memcmp(&G->args, &a, sizeof(PassArgs)) == 0;
    for (int s = 0; same && s < 3; ++s) same = G->cap[s] == p->s[s].capacity;
    if (same) return G;
    sfq_step_graph_free(ctx);
    G = new StepGraph;
    if (build_step_graph<T>(ctx, a, p, dt, G) != QED_OK) {
        delete G;
        ctx->step_graph_failed = 1;
        return nullptr;
    }
    ctx->step_graph = G;
    return G;
}

// Host-driven steps: the same kernels launched one by one, the host reading
// the control block between newborn-pass groups and before the merge step.
// Used to time the kernels individually (cfg.profile: CUDA events around
// each launch) and where graphs with conditional nodes are unavailable.
template <class T>
static qed_status host_steps(qed_ctx *ctx, qed_particles *pw, PassArgs &a, double dt, int nsteps) {
    const bool cascade = ctx->cfg.push_photons != 0;
    const bool od_method = ctx->cfg.event_method == QED_METHOD_OPTICAL_DEPTH;
    qed_particles P = *pw;                         // counts below: bounds read back from the device
    int spec_passes = ctx->spec_passes > 0 ? ctx->spec_passes : 2;
    for (int it = 0; it < nsteps; ++it) {
        a.pass = 0;
        k_step_begin<<<1, 1, 0, ctx->stream>>>(ctx->ctl, dt);
        SFQ_LAUNCHED(ctx, 1);
        qed_status e = od_method ? launch_od<T>(ctx, a, cascade) : launch_pass<T>(ctx, a, cascade);
        if (e != QED_OK) return e;
        if (cascade && !od_method) {
            // Algorithm 2: sweep the newborns until a pass creates nothing.
            // Passes are enqueued in groups (a pass over an empty range
            // returns at once), so the host reads the control block once per
            // group; the group size follows the previous step's pass count.
            int pass = 1;
            k_pass_setup<<<1, 1, 0, ctx->stream>>>(ctx->ctl);
            SFQ_LAUNCHED(ctx, 1);
            for (;;) {
                for (int g = 0; g < spec_passes; ++g, ++pass) {
                    a.pass = pass;
                    e = launch_pass<T>(ctx, a, true);
                    if (e != QED_OK) return e;
                    k_pass_setup<<<1, 1, 0, ctx->stream>>>(ctx->ctl);
                    SFQ_LAUNCHED(ctx, 1);
                }
                e = read_ctl(ctx);
                if (e != QED_OK) return e;
                if (ctx->ctl_host->overflow || !ctx->ctl_host->more) break;
                if ((unsigned long long)pass >= pass_limit_of(ctx)) {
                    // give up like the graph's loop does (the wait reports it)
                    k_set_timeout<<<1, 1, 0, ctx->stream>>>(ctx->ctl);
                    SFQ_LAUNCHED(ctx, 1);
                    break;
                }
            }
            // passes with work in this step (the control block counts them)
            const long long used = (long long)ctx->ctl_host->step_passes;
            spec_passes = used < 1 ? 1 : (used > 8 ? 8 : (int)used);
        }
        if (cascade || ctx->cfg.thin_cap > 0) {
            // merge step (Sec. 4.2): drop dead photons, then level
            if (!cascade || od_method) {
                e = read_ctl(ctx);
                if (e != QED_OK) return e;
            }
            const DevCtl &c = *ctx->ctl_host;
            if (c.overflow || c.timeout || c.bad_index) break;
            for (int s = 0; s < 3; ++s) P.s[s].count = (int64_t)c.count[s];
            // per species: leveling (it skips dead entries and compacts), else
            // removal of the photons that converted
            for (int s = 0; s < 3; ++s) {
                const bool level = ctx->cfg.thin_cap > 0 && P.s[s].count > ctx->cfg.thin_cap;
                const int64_t step = (int64_t)c.step_next - 1;
                if (level) {
                    e = timed_block(ctx, 3, [&] { return sfq_level_species(ctx, &P.s[s], s, step, true); });
                } else if (cascade && s == 2) {
                    e = timed_block(ctx, 2, [&] { return sfq_compact_species(ctx, &P.s[2], 2, true); });
                }
                if (e != QED_OK) return e;
            }
        }
    }
    ctx->spec_passes = spec_passes;
    return QED_OK;
}

// Opens a batch of steps: the counts and capacities of *p go to the device
// control block (staged in pinned memory), the context's per-particle work
// buffers grow to the capacities, and with restore_on_overflow the particle
// state is copied aside.
static qed_status open_batch(qed_ctx *ctx, qed_particles *p, int64_t step0) {
    ctx->launches = 0;
    ctx->sync_ms = 0.0;
    for (int k = 0; k < 4; ++k) ctx->kernel_ms[k] = 0.0;
    ctx->async_t0_ms = std::chrono::duration<double, std::milli>(
        std::chrono::steady_clock::now().time_since_epoch()).count();
    if (ctx->cfg.profile) {
        qed_status e = ensure_events(ctx);
        if (e != QED_OK) return e;
    }
    DevCtl &h = *ctx->ctl_up;
    memset(&h, 0, sizeof(DevCtl));
    for (int s = 0; s < 3; ++s) {
        h.count[s] = (unsigned long long)p->s[s].count;
        h.capacity[s] = (unsigned long long)p->s[s].capacity;
    }
    h.step_next = (unsigned long long)step0;
    h.pass_limit = pass_limit_of(ctx);
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl, &h, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    int64_t cap_max = 0;
    for (int s = 0; s < 3; ++s) {
        qed_status e = ensure_tau(ctx, s, p->s[s].capacity);
        if (e != QED_OK) return e;
        cap_max = p->s[s].capacity > cap_max ? p->s[s].capacity : cap_max;
    }
    // compaction work buffers sized once for the largest species
    qed_status e = sfq_ensure_work(ctx, (cap_max + 1023) / 1024 + 2, cap_max);
    if (e != QED_OK) return e;
    if (ctx->cfg.restore_on_overflow) {
        e = snapshot(ctx, p, false);
        if (e != QED_OK) return e;
    }
    ctx->async_p = *p;
    ctx->async_deferred = 0;
    for (int s = 0; s < 3; ++s) ctx->async_count0[s] = p->s[s].count;
    ctx->async_next_step = step0;
    ctx->async_open = 1;
    return QED_OK;
}

static bool same_binding(const qed_particles &a, const qed_particles &b) {
    for (int s = 0; s < 3; ++s) {
        const qed_species &x = a.s[s], &y = b.s[s];
        if (x.x != y.x || x.y != y.y || x.z != y.z || x.px != y.px || x.py != y.py || x.pz != y.pz || x.w != y.w ||
            x.id != y.id || x.nevents != y.nevents || x.capacity != y.capacity)
            return false;
    }
    return true;
}

// Enqueue nsteps steps of the open batch (no host wait on the graph path).
template <class T>
static qed_status enqueue_steps(qed_ctx *ctx, const qed_field_desc *field, double dt, int nsteps, int64_t step0) {
    qed_particles *p = &ctx->async_p;
    const bool cascade = ctx->cfg.push_photons != 0;
    if (step0 != ctx->async_next_step) {
        k_set_step<<<1, 1, 0, ctx->stream>>>(ctx->ctl, (unsigned long long)step0);
        SFQ_LAUNCHED(ctx, 1);
    }
    ctx->async_next_step = step0 + nsteps;
    if (nsteps == 0) return QED_OK;
    PassArgs a;
    memset(&a, 0, sizeof a);                       // padding included: the graph key compares bytes
    for (int s = 0; s < 3; ++s) {
        const qed_species &S = p->s[s];
        a.sp[s] = SpeciesDev{S.x, S.y, S.z, S.px, S.py, S.pz, S.w,
                             reinterpret_cast<unsigned long long *>(S.id), S.nevents, ctx->tau[s], ctx->od[s]};
    }
    a.ctl = ctx->ctl;
    const bool f32 = sizeof(T) == 4;
    a.coef = f32 ? (const void *)ctx->coef32 : (const void *)ctx->coef64;
    a.icdf_em = f32 ? (const void *)ctx->icdf_em32 : (const void *)ctx->icdf_em64;
    a.icdf_pair = f32 ? (const void *)ctx->icdf_pair32 : (const void *)ctx->icdf_pair64;
    a.mlp_w16 = ctx->cfg.sampler == QED_SAMPLER_MLP ? ctx->mlp_w16 : nullptr;
    a.field_kind = field->kind;
    if (field->kind == QED_FIELD_GRID) {
        long long nodes = 1;
        for (int d = 0; d < 3; ++d) {
            a.gn[d] = (int)field->params[d];
            a.ginv[d] = (double)a.gn[d] / field->params[3 + d];
            a.ginv_f[d] = (float)a.ginv[d];
            nodes *= a.gn[d];
        }
        // the caller's [component][node] values, interleaved per node for the
        // kernels (the grid is constant during the call)
        const size_t bytes = (size_t)nodes * 8 * sizeof(T);
        if (ctx->grid_il_bytes < bytes) {
            if (ctx->grid_il) SFQ_CUDA(cudaFreeAsync(ctx->grid_il, ctx->stream));
            ctx->grid_il = nullptr;
            ctx->grid_il_bytes = 0;
            if (cudaMallocAsync(&ctx->grid_il, bytes, ctx->stream) != cudaSuccess) return QED_ERR_NOMEM;
            ctx->grid_il_bytes = bytes;
        }
        k_grid_interleave<T><<<(unsigned)((nodes + 255) / 256), 256, 0, ctx->stream>>>(
            reinterpret_cast<const T *>(ctx->field_grid), reinterpret_cast<T *>(ctx->grid_il), nodes);
        SFQ_LAUNCHED(ctx, 1);
        SFQ_CUDA(cudaGetLastError());
        a.grid_il = ctx->grid_il;
    }
    a.field_zero = field_zero_of(*field);      // chi without its cancellation guard where allowed
    for (int i = 0; i < 6; ++i) {
        a.prm[i] = field->params[i];
        a.prm_f[i] = (float)field->params[i];
    }
    a.dt = dt;
    a.dt_f = (float)dt;
    a.lam_skip = ldexp(1.0, -54) / dt;
    a.lam_skip_f = (float)a.lam_skip;
    a.dt_f_gt = (double)a.dt_f > dt ? a.dt_f : nextafterf(a.dt_f, INFINITY);
    a.seed = ctx->cfg.seed;
    a.keys = philox_keys(ctx->cfg.seed);
    a.soft_filter = ctx->cfg.soft_photon_filter;
    a.record_newborn_tau = cascade ? 1 : 0;

    ctx->async_deferred = 1;
    StepGraph *G = ctx->cfg.profile ? nullptr : step_graph_for<T>(ctx, a, p, dt);
    if (!G) return host_steps<T>(ctx, p, a, dt, nsteps);
    for (int it = 0; it < nsteps; ++it) SFQ_CUDA(cudaGraphLaunch(G->exec, ctx->stream));
    SFQ_LAUNCHED(ctx, (int64_t)nsteps * G->top_kernels);
    return QED_OK;
}

// Ends the open batch: reads the control block back (the one wait), fills the
// statistics, updates the counts of *p (or restores the state at the batch's
// start after an overflow, with restore_on_overflow).
static qed_status wait_batch(qed_ctx *ctx, qed_particles *p, qed_stats *out) {
    if (ctx->async_deferred) {
        // the steps may have left dead entries in place: remove them, so the
        // counts returned hold live particles only (after a step that ran out
        // of capacity nothing is moved)
        ctx->async_deferred = 0;
        for (int s = 0; s < 3; ++s) {
            qed_status e = sfq_compact_pending(ctx, &ctx->async_p.s[s], s);
            if (e != QED_OK) {
                ctx->async_open = 0;
                return e;
            }
        }
    }
    qed_status e = read_ctl(ctx);
    ctx->async_open = 0;
    if (e != QED_OK) return e;
    DevCtl &c = *ctx->ctl_host;
    qed_status rc = QED_OK;
    if (c.overflow) rc = QED_ERR_CAPACITY;
    if (c.timeout) rc = QED_ERR_TIMEOUT;
    if (c.bad_index) rc = QED_ERR_STATE;
    qed_stats st{};
    st.particle_steps = (int64_t)c.particle_steps;
    st.emit_events = (int64_t)c.emit_events;
    st.pair_events = (int64_t)c.pair_events;
    for (int s = 0; s < 3; ++s) st.needed_capacity[s] = (int64_t)c.needed[s];
    st.max_subevents = (int64_t)c.max_subevents;
    st.overflow = (int64_t)c.overflow;
    st.passes = (int64_t)c.passes;
    st.thinned = (int64_t)c.thinned;
    st.moved = (int64_t)c.moved;
    st.lepton_steps = (int64_t)c.lepton_steps;
    st.chi_fp64 = (int64_t)c.chi_fp64;
    st.photon_steps = (int64_t)c.photon_steps;
    if (ctx->cfg.profile) {
        e = sfq_drain_events(ctx);
        if (e != QED_OK) return e;
    }
    for (int k = 0; k < 4; ++k) st.kernel_ms[k] = ctx->kernel_ms[k];
    st.launches = ctx->launches + (int64_t)c.graph_kernels;
    st.sync_ms = ctx->sync_ms;
    st.call_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
                     .count() - ctx->async_t0_ms;
    qed_particles &B = ctx->async_p;
    if (rc == QED_ERR_CAPACITY && ctx->cfg.restore_on_overflow) {
        for (int s = 0; s < 3; ++s) B.s[s].count = ctx->async_count0[s];
        e = snapshot(ctx, &B, true);
        if (e != QED_OK) return e;
        SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        for (int s = 0; s < 3; ++s) B.s[s].count = (int64_t)min(c.count[s], c.capacity[s]);
    }
    for (int s = 0; s < 3; ++s) p->s[s].count = B.s[s].count;
    if (out) *out = st;
    ctx->acc.particle_steps += st.particle_steps;
    ctx->acc.emit_events += st.emit_events;
    ctx->acc.pair_events += st.pair_events;
    ctx->acc.passes += st.passes;
    ctx->acc.thinned += st.thinned;
    ctx->acc.moved += st.moved;
    ctx->acc.lepton_steps += st.lepton_steps;
    ctx->acc.chi_fp64 += st.chi_fp64;
    ctx->acc.photon_steps += st.photon_steps;
    ctx->acc.launches += st.launches;
    for (int k = 0; k < 4; ++k) ctx->acc.kernel_ms[k] += st.kernel_ms[k];
    ctx->acc.sync_ms += st.sync_ms;
    ctx->acc.call_ms += st.call_ms;
    if (st.max_subevents > ctx->acc.max_subevents) ctx->acc.max_subevents = st.max_subevents;
    return rc;
}

static qed_status check_push_args(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt, int nsteps,
                                  int64_t step0) {
    if (!ctx || !p || !field || nsteps < 0 || !(dt > 0.0) || step0 < 0 || step0 + nsteps > 0xFFFFFFFFll)
        return QED_ERR_INVALID;
    if (ctx->cfg.sampler == QED_SAMPLER_MLP && !ctx->mlp_ready) return QED_ERR_STATE;
    if (field->kind < QED_FIELD_UNIFORM || field->kind > QED_FIELD_GRID) return QED_ERR_INVALID;
    if (ctx->cfg.event_method == QED_METHOD_OPTICAL_DEPTH) {
        for (int s = 0; s < 3; ++s)
            if (p->s[s].capacity > 0 && !ctx->od[s]) return QED_ERR_STATE;   // qed_set_optical_depth first
        if (ctx->cfg.sampler == QED_SAMPLER_MLP) return QED_ERR_INVALID;     // the table sampler only
    } else if (ctx->cfg.event_method != QED_METHOD_SUBSTEP) {
        return QED_ERR_INVALID;
    }
    if (field->kind == QED_FIELD_GRID) {
        if (!ctx->field_grid) return QED_ERR_STATE;
        for (int d = 0; d < 3; ++d) {
            const double n = field->params[d], len = field->params[3 + d];
            if (!(n >= 1.0 && n <= 65536.0 && n == floor(n)) || !(len > 0.0)) return QED_ERR_INVALID;
        }
    }
    if (ctx->async_open) return same_binding(ctx->async_p, *p) ? QED_OK : QED_ERR_STATE;
    for (int s = 0; s < 3; ++s) {
        qed_status e = check_species(p->s[s]);
        if (e != QED_OK) return e;
    }
    return QED_OK;
}

qed_status sfq_push_async(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt, int nsteps,
                          int64_t step0) {
    qed_status e = check_push_args(ctx, p, field, dt, nsteps, step0);
    if (e != QED_OK) return e;
    if (!ctx->async_open) {
        e = open_batch(ctx, p, step0);
        if (e != QED_OK) return e;
    }
    if (ctx->cfg.precision == QED_FP32) return enqueue_steps<float>(ctx, field, dt, nsteps, step0);
    return enqueue_steps<double>(ctx, field, dt, nsteps, step0);
}

qed_status sfq_push_wait(qed_ctx *ctx, qed_particles *p, qed_stats *out) {
    if (!ctx || !p) return QED_ERR_INVALID;
    if (!ctx->async_open) return QED_ERR_STATE;
    if (!same_binding(ctx->async_p, *p)) return QED_ERR_STATE;
    return wait_batch(ctx, p, out);
}

qed_status sfq_push(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt, int nsteps,
                    int64_t step0, qed_stats *out) {
    const bool opened = ctx && !ctx->async_open;
    qed_status e = sfq_push_async(ctx, p, field, dt, nsteps, step0);
    if (e != QED_OK) {
        // a batch this call opened is closed again (its work is drained)
        if (opened && ctx->async_open) {
            qed_stats tmp;
            wait_batch(ctx, p, &tmp);
        }
        return e;
    }
    return wait_batch(ctx, p, out);
}

qed_status sfq_philox(const uint32_t *ctr, int64_t n, uint64_t key, uint32_t *out, cudaStream_t s) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return QED_ERR_INVALID;
    if (!aligned16(ctr) || !aligned16(out)) return QED_ERR_INVALID;
    if (n == 0) return QED_OK;
    k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4 *>(ctr), n,
                                                         make_uint2((uint32_t)key, (uint32_t)(key >> 32)),
                                                         reinterpret_cast<uint4 *>(out));
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaStreamSynchronize(s));
    return QED_OK;
}

qed_status sfq_eval_rate(qed_ctx *ctx, int is_photon, const double *chi, int64_t n, double *F) {
    if (!ctx || n < 0 || (n > 0 && (!chi || !F))) return QED_ERR_INVALID;
    if (n == 0) return QED_OK;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (ctx->cfg.precision == QED_FP32) k_eval_rate<float><<<g, 256, 0, ctx->stream>>>(ctx->coef32, is_photon, chi, n, F);
    else k_eval_rate<double><<<g, 256, 0, ctx->stream>>>(ctx->coef64, is_photon, chi, n, F);
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}

qed_status sfq_eval_chi(qed_ctx *ctx, int is_photon, const double *p, const double *E, const double *B, int64_t n,
                        double *chi, int64_t *n_fp64) {
    if (!ctx || n < 0 || (n > 0 && (!p || !E || !B || !chi))) return QED_ERR_INVALID;
    if (n_fp64) *n_fp64 = 0;
    if (n == 0) return QED_OK;
    const unsigned g = (unsigned)((n + 255) / 256);
    unsigned long long *cnt = &ctx->ctl->chi_fp64;
    SFQ_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), ctx->stream));
    if (ctx->cfg.precision == QED_FP32) k_eval_chi<float><<<g, 256, 0, ctx->stream>>>(is_photon, p, E, B, n, chi, cnt);
    else k_eval_chi<double><<<g, 256, 0, ctx->stream>>>(is_photon, p, E, B, n, chi, cnt);
    SFQ_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    SFQ_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (n_fp64) *n_fp64 = (int64_t)h;
    return QED_OK;
}

qed_status sfq_sample(qed_ctx *ctx, int is_photon, const double *chi, const double *u, int64_t n, double *delta,
                      double *one_minus) {
    if (!ctx || n < 0 || (n > 0 && (!chi || !u || !delta))) return QED_ERR_INVALID;
    if (n == 0) return QED_OK;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (ctx->cfg.precision == QED_FP32)
        k_sample<float><<<g, 256, 0, ctx->stream>>>(is_photon ? ctx->icdf_pair32 : ctx->icdf_em32, is_photon, chi, u,
                                                    n, delta, one_minus);
    else
        k_sample<double><<<g, 256, 0, ctx->stream>>>(is_photon ? ctx->icdf_pair64 : ctx->icdf_em64, is_photon, chi,
                                                     u, n, delta, one_minus);
    SFQ_CUDA(cudaGetLastError());
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return QED_OK;
}
