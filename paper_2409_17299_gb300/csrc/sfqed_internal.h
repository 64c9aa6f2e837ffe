// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sfqed.h"

namespace sfq {

// Table grids (the header of the public ABI states their meaning).
constexpr int EM_NCHI = 121;     // log10 chi in [-3, 3], 20 per decade
constexpr int PAIR_NCHI = 101;   // log10 chi in [-2, 3], 20 per decade
constexpr int EM_NS = 257;       // logit u in [-16, 16]
constexpr int PAIR_NS = 129;     // logit u in [-16, 0]
constexpr int CHEB_N = 11;       // degree-10 Chebyshev interpolant per decade
constexpr int EM_NDEC = 6;
constexpr int PAIR_NDEC = 5;
constexpr int NCOEF = (EM_NDEC + PAIR_NDEC) * CHEB_N;   // 121 coefficients
// FP32 mode: the same approximant as cubic pieces, RSEG per decade of
// log10 chi, each four floats (monomial coefficients in the piece's local
// coordinate t in [0, 1)), fitted in FP64 to the Chebyshev form
constexpr int RSEG = 16;
constexpr int EM_NSEG = EM_NDEC * RSEG, PAIR_NSEG = PAIR_NDEC * RSEG;
constexpr int NRATE32 = 4 * (EM_NSEG + PAIR_NSEG);    // 704 floats
// words of the rate representation in the working precision
template <class T> struct RateWords;
template <> struct RateWords<double> { static constexpr int N = NCOEF; };
template <> struct RateWords<float> { static constexpr int N = NRATE32; };

// Device-resident control block: counts, pass ranges and statistics.  Every
// counter is 64-bit so that appends can count demand beyond capacity.
struct DevCtl {
    unsigned long long count[3];        // append cursor (may exceed capacity on overflow)
    unsigned long long capacity[3];
    unsigned long long begin[3];        // range of the current pass
    unsigned long long end[3];
    unsigned long long particle_steps;
    unsigned long long lepton_steps;
    unsigned long long photon_steps;
    unsigned long long emit_events;
    unsigned long long pair_events;
    unsigned long long max_subevents;
    unsigned long long overflow;
    unsigned long long needed[3];
    unsigned long long more;            // the last pass setup found work
    unsigned long long passes;
    unsigned long long thinned;
    unsigned long long alive[3];        // compaction: alive entries per species
    unsigned long long holes[3];        // compaction: dead entries below alive[s]
    unsigned long long bad_index;       // a bounds check failed (index recorded, access skipped)
    unsigned long long chi_fp64;        // FP32 mode: chi evaluations that fell back to FP64
    unsigned long long graph_kernels;   // kernels run inside graphs (their launches are on the device)
    unsigned long long step_next;       // index of the step the next step-begin kernel opens
    unsigned long long step_passes;     // newborn passes of the current step
    unsigned long long timeout;         // a bounded device-side loop gave up (QED_ERR_TIMEOUT)
    double sv_t_n;                      // current step: t_n = step * dt
    float sv_t_red_f;                   // current step: (t_n mod 2 pi) rounded to float
    unsigned sv_step;                   // current step index (Philox counter word 2)
    unsigned long long deferred[3];     // dead entries left in place by the last merge step
    unsigned long long moved;           // compaction: entries moved into holes
    unsigned long long pass_limit;      // newborn passes a step may run (then timeout)
    unsigned long long pad[4];
};
static_assert(sizeof(DevCtl) == 384, "control block layout");

// The current step's time as the pass kernels read it from the control
// block (written by the step-begin kernel, so a captured step graph needs no
// per-step kernel arguments); time_phase() takes it like an argument block.
struct StepTime {
    int field_kind;
    double t_n;
    float t_n_red_f;
    unsigned step;
};

// Leveling: iteration state per species and per-block partial sums.
constexpr int LEVEL_MAX_BLOCKS = 4096;
struct LevelIter {
    double lo, hi;          // bracket of w*: S(lo) > cap >= S(hi)
    double w;               // point evaluated by the next pass (+inf first)
    double wstar;           // result (0: no leveling)
    float w_up, wstar_up;   // smallest floats >= w and >= wstar (exact FP32 comparisons)
    float wstar_f;          // wstar rounded to float (the new weight in FP32 mode)
    float wstar_inv_f;      // 1 / wstar rounded to float
    unsigned long long done, iters, alive;
    unsigned long long mode;    // 0: a pass advances the iteration; 1: a pass only stores its sums
    double sumA;                // sums of the last pass in mode 1
    unsigned long long sumC, sumN, sumM;
};
struct LevelWork {
    LevelIter it[3];
    unsigned arrive[4];                         // blocks of the current pass that finished (per species)
    unsigned long long passes[4];               // passes of the current graph-driven leveling
    double prev[4];                             // last threshold found per species (the next start)
    double partA[LEVEL_MAX_BLOCKS];             // sum of weights below w (block partials)
    unsigned long long partC[LEVEL_MAX_BLOCKS]; // count at or above w
    unsigned long long partN[LEVEL_MAX_BLOCKS]; // alive count
    unsigned long long partM[LEVEL_MAX_BLOCKS]; // largest weight (double bits)
    unsigned long long partL[LEVEL_MAX_BLOCKS]; // largest weight below w (double bits; 0: none)
    unsigned long long partH[LEVEL_MAX_BLOCKS]; // smallest weight at or above w (double bits; +inf: none)
};

// Philox round keys of one seed: k[2 r], k[2 r + 1] are the key of round r
struct PhiloxKeys {
    uint32_t k[20];
};

// chi shortcut a field allows everywhere: 1 B = 0, 2 E = 0, 3 E parallel
// to B (the standing circularly polarised wave), 0 none
inline int field_zero_of(const qed_field_desc &f) {
    if (f.kind == QED_FIELD_ROTATING_E) return 1;
    if (f.kind == QED_FIELD_STANDING_CP) return 3;
    if (f.kind == QED_FIELD_UNIFORM) {
        const double *q = f.params;
        if (q[3] == 0.0 && q[4] == 0.0 && q[5] == 0.0) return 1;
        if (q[0] == 0.0 && q[1] == 0.0 && q[2] == 0.0) return 2;
    }
    return 0;
}

struct SpeciesDev {
    void *x, *y, *z, *px, *py, *pz, *w;
    unsigned long long *id;
    unsigned *nev;
    double *tau;            // birth clock of newborns (context work buffer)
    void *od;               // remaining optical depth (QED_METHOD_OPTICAL_DEPTH, T), or null
};

struct PassArgs {
    SpeciesDev sp[3];
    DevCtl *ctl;
    const void *coef;       // NCOEF coefficients (T)
    const void *icdf_em;    // EM_NCHI * EM_NS (T)
    const void *icdf_pair;  // PAIR_NCHI * PAIR_NS (T)
    const __nv_bfloat16 *mlp_w16;   // surrogate network weights, or null (table sampler)
    int field_kind;
    const void *grid_il;    // QED_FIELD_GRID: node values interleaved [nz][ny][nx][8] (T)
    int gn[3];              // grid nodes per axis
    double ginv[3];         // nodes per unit length (n / L)
    float ginv_f[3];
    int field_zero;         // chi shortcut: 1 B = 0, 2 E = 0, 3 E parallel to B (everywhere), else 0
    double prm[6];
    float prm_f[6];         // prm rounded to float once (FP32 mode)
    double dt;
    float dt_f;             // (float)dt
    double lam_skip;        // 2^-54 / dt: below this rate no event can happen in a step (see the passes)
    float lam_skip_f;
    float dt_f_gt;          // smallest float above dt (FP32 first-iteration event test)
    unsigned long long seed;
    PhiloxKeys keys;        // round keys of seed (event draws)
    int pass;               // 0: particles present at the step start (tau = 0)
    int soft_filter;
    int record_newborn_tau; // newborns get their birth clock stored (cascades)
};

}  // namespace sfq

struct qed_ctx {
    qed_config cfg;
    cudaStream_t stream;
    int device;
    int sm_count;
    // tables
    double *coef64;          // NCOEF
    float *coef32;
    double *icdf_em64, *icdf_pair64;
    float *icdf_em32, *icdf_pair32;
    double *gl;              // Gauss-Legendre nodes and weights (work)
    // control
    sfq::DevCtl *ctl;
    sfq::DevCtl *ctl_host;   // pinned mirror (read back at the end of a batch of steps)
    sfq::DevCtl *ctl_up;     // pinned staging of the upload when a batch of steps opens
    // newborn birth clocks
    double *tau[3];
    int64_t tau_cap[3];
    // compaction / leveling work buffers
    unsigned long long *blk;      // per-block counts
    int64_t blk_cap;
    unsigned long long *slots;    // hole indices
    int64_t slots_cap;
    sfq::LevelWork *lev;          // leveling work (device)
    unsigned long long *pin;      // small pinned host scratch (flags read back)
    // overflow snapshot
    void *snap;
    int64_t snap_bytes;
    qed_stats acc;           // accumulated statistics (host)
    // profiling: CUDA event pairs around the push kernels
    static constexpr int EVN = 512;
    cudaEvent_t ev[4][EVN][2];   // [lepton|photon|compaction|leveling][pair][start|stop]
    int ev_used[4];
    bool ev_ready;
    double kernel_ms[4];         // lepton, photon, compaction, leveling
    int64_t launches;            // kernels launched since the last reset
    double sync_ms;              // host time blocked in stream synchronisation
    void *batch;                 // batched-push work buffers
    void *lev_graph[3];          // per species: the graph-driven leveling iteration (or null)
    int lev_graph_failed;        // graphs with conditional nodes unavailable: host-checked passes
    cudaStream_t cap_stream;     // private stream for graph capture (the caller's may be the legacy stream)
    void *od[3];                 // caller's optical-depth arrays (QED_METHOD_OPTICAL_DEPTH, T)
    const void *field_grid;      // caller's gridded field values (QED_FIELD_GRID)
    void *grid_il;               // the same interleaved per node (8 values), refreshed each call
    size_t grid_il_bytes;
    int tuned_threads;           // block shape picked by the autotuner (0: none yet)
    int tuned_budget;            // step budget picked by the autotuner (0: none yet)
    int spec_passes;             // newborn passes enqueued per host check (from the last step)
    int lev_chunk[3];            // leveling passes enqueued per host check (from the last leveling)
    // steps enqueued without waiting (qed_push_async) until qed_push_wait:
    // the device control block holds the counts meanwhile
    int async_open;
    qed_particles async_p;       // the arrays bound by the open batch (pointers and capacities)
    int64_t async_count0[3];     // counts when the batch opened (restored on overflow)
    int64_t async_next_step;     // step index following the last enqueued step
    double async_t0_ms;          // host clock when the batch opened
    void *step_graph;            // the captured PIC step (StepGraph, sfqed_push.cu) or null
    int async_deferred;          // the open batch's steps may have left dead entries in place
    int step_graph_failed;       // conditional graph nodes unavailable: host-driven steps
    // surrogate network: FP32 master parameters, Adam moments and gradient
    // (4 x 8577 floats), BF16 copy used by the kernels, loss accumulator
    float *mlp_p;
    __nv_bfloat16 *mlp_w16;
    float *mlp_loss;
    int mlp_ready;
};

// Implemented in sfqed_tables.cu
qed_status sfq_build_tables(qed_ctx *ctx);
// Implemented in sfqed_push.cu
qed_status sfq_push(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt,
                    int nsteps, int64_t step0, qed_stats *out);
qed_status sfq_push_async(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt, int nsteps,
                          int64_t step0);
qed_status sfq_push_wait(qed_ctx *ctx, qed_particles *p, qed_stats *out);
void sfq_step_graph_free(qed_ctx *ctx);
qed_status sfq_eval_rate(qed_ctx *ctx, int is_photon, const double *chi, int64_t n, double *F);
qed_status sfq_sample(qed_ctx *ctx, int is_photon, const double *chi, const double *u, int64_t n,
                      double *delta, double *one_minus);
qed_status sfq_eval_chi(qed_ctx *ctx, int is_photon, const double *p, const double *E, const double *B, int64_t n,
                        double *chi, int64_t *n_fp64);
qed_status sfq_philox(const uint32_t *ctr, int64_t n, uint64_t key, uint32_t *out, cudaStream_t s);
// Implemented in sfqed_batch.cu
qed_status sfq_batch_push(qed_ctx *ctx, qed_particles *ens, const qed_field_desc *fields, int n_ens, double dt,
                          int nsteps, int64_t step0, qed_stats *out, int threads_override,
                          int budget_override);
qed_status sfq_batch_shape(qed_ctx *ctx, int *threads, int *budget);
qed_status sfq_batch_autotune(qed_ctx *ctx, const qed_particles *ens, const qed_field_desc *fields, int n_ens,
                              double dt, int nsteps, int *chosen, double *ms3);
void sfq_batch_free(qed_ctx *ctx);
// Implemented in sfqed_mlp.cu
qed_status sfq_mlp_set_params(qed_ctx *ctx, const float *params);
qed_status sfq_mlp_get_params(qed_ctx *ctx, float *params);
qed_status sfq_mlp_eval(qed_ctx *ctx, const float *feat, int64_t n, float *y);
qed_status sfq_mlp_grad(qed_ctx *ctx, const float *feat, const float *target, int64_t n, float *grad_host,
                        double *loss);
qed_status sfq_mlp_train(qed_ctx *ctx, int64_t n_samples, int batch, double lr, uint64_t seed, double *final_loss);
// Building a CUDA graph from captured launches: each capture appends the
// launches a function issues on `st` after the current tail of the top-level
// graph (or into a conditional node's body graph, which starts empty).
struct GraphBuild {
    cudaGraph_t g = nullptr;
    cudaStream_t st = nullptr;
    std::vector<cudaGraphNode_t> tail;   // nodes the next top-level node depends on
    int top_kernels = 0;                 // kernel nodes of the top level (run once per launch)

    template <class F> cudaError_t capture(cudaGraph_t into, F issue) {
        const bool top = into == g;
        cudaError_t e = cudaStreamBeginCaptureToGraph(st, into, top && !tail.empty() ? tail.data() : nullptr, nullptr,
                                                      top ? tail.size() : 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        const qed_status q = issue();
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        cudaError_t e2 = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        std::vector<cudaGraphNode_t> next(deps, deps + (e2 == cudaSuccess ? nd : 0));
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(st, &out);
        if (e2 != cudaSuccess) return e2;
        if (e != cudaSuccess) return e;
        if (q != QED_OK) return cudaErrorUnknown;
        if (top) tail.swap(next);
        return cudaSuccess;
    }
    // a conditional node after the tail; *body receives its (first) body graph
    cudaError_t conditional(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraph_t *body) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = type;
        cp.conditional.size = 1;
        cudaGraphNode_t n;
        cudaError_t e = cudaGraphAddNode(&n, g, tail.empty() ? nullptr : tail.data(), nullptr, tail.size(), &cp);
        if (e != cudaSuccess) return e;
        *body = cp.conditional.phGraph_out[0];
        tail.assign(1, n);
        return cudaSuccess;
    }
};

// Implemented in sfqed_compact.cu
// the merge step of species s (leveling when its count exceeds the cap, dead
// entries removed) appended to a step graph; decided on the device
qed_status sfq_capture_merge(qed_ctx *ctx, GraphBuild &gb, qed_species *sp, int s, bool always_compact);
// may_defer: the moves may be left for a later step (dead entries stay in
// place while they are few; see k_scan_tiles)
qed_status sfq_compact_species(qed_ctx *ctx, qed_species *sp, int s, bool may_defer = false);
qed_status sfq_compact_pending(qed_ctx *ctx, qed_species *sp, int s);
void sfq_level_graphs_free(qed_ctx *ctx);
qed_status sfq_level_species(qed_ctx *ctx, qed_species *sp, int s, int64_t step, bool may_defer = false);
qed_status sfq_level_eval(qed_ctx *ctx, qed_species *sp, int s, double w, double *A, int64_t *C, int64_t *N,
                          double *M);
qed_status sfq_level_apply_species(qed_ctx *ctx, qed_species *sp, int s, double wstar, int64_t step);
void sfq_level_advance(double *lo, double *hi, double *w, double *wstar, int64_t *iters, int64_t *done,
                       int64_t *alive, double A, int64_t C, int64_t N, double M, int64_t cap);
qed_status sfq_drain_events(qed_ctx *ctx);
// pass launchers, one per field variant (sfqed_pass_analytic.cu, sfqed_pass_grid.cu)
namespace sfq {
namespace pass_analytic {
template <class T> qed_status launch_pass(qed_ctx *ctx, PassArgs &a, bool photons);
template <class T> qed_status launch_od(qed_ctx *ctx, PassArgs &a, bool photons);
}
namespace pass_grid {
template <class T> qed_status launch_pass(qed_ctx *ctx, PassArgs &a, bool photons);
template <class T> qed_status launch_od(qed_ctx *ctx, PassArgs &a, bool photons);
}
}  // namespace sfq
qed_status sfq_ensure_work(qed_ctx *ctx, int64_t n_blocks, int64_t n_slots);

#define SFQ_LAUNCHED(ctx, n) ((ctx)->launches += (n))

#define SFQ_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return QED_ERR_CUDA;                     \
    } while (0)
