/*
 * sfqed.h -- C ABI of the GB300 strong-field QED event generator.
 *
 * The library implements the per-macroparticle QED step of the optimized
 * event generator of arXiv:2409.17299 (Sec. 3, Algorithms 1 and 2): chi from
 * the local fields and momentum, the Compton and Breit-Wheeler rates from an
 * approximation of precomputed rates, an exponential event clock sub-stepped
 * inside each PIC step, inverse-CDF energy sampling, and the append of the
 * new particles to the ensemble (Sec. 4.1-4.2), plus compaction and global
 * leveling (Sec. 4.2, Sec. 5.1).  All work runs in CUDA kernels for sm_103a.
 *
 * Conventions shared by every call
 *  - Units: time 1/omega, length c/omega, momentum m c, energy m c^2, fields
 *    m c omega / e, wavelength 0.8 um.  One laser period is 2 pi.
 *  - Pointers named *_dev are device pointers; everything else is host memory.
 *  - Particle memory (qed_species) is owned by the caller and is never freed,
 *    reallocated or resized by the library.  The context owns its tables,
 *    work buffers and statistics.
 *  - Every call returns a qed_status; nothing is thrown across the ABI and no
 *    kernel traps.  qed_strerror() names a status.
 *  - All device work is issued on the stream given to qed_init_tables().
 *    Calls that return host-side values (counts, statistics) synchronise
 *    that stream before returning.
 *  - Randomness is counter-based (Philox4x32-10, key = seed, counter =
 *    (id low, id high, step, k)), so a particle's draws do not depend on
 *    thread scheduling or append order, and a call can be replayed (the
 *    capacity-overflow replay relies on it).  In FP32 mode the leveling
 *    threshold's sums depend on the array order in their last bits, so a
 *    keep/drop decision lying within ~1e-15 of its boundary may differ
 *    between runs whose appends landed in another order.
 */
#ifndef SFQED_H
#define SFQED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qed_ctx qed_ctx;   /* opaque; owns tables, work buffers, statistics */

typedef enum {
    QED_OK = 0,
    QED_ERR_INVALID = 1,    /* bad argument: null pointer, unknown kind, misaligned buffer, ... */
    QED_ERR_CAPACITY = 2,   /* a species ran out of capacity; see qed_stats.needed_capacity */
    QED_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    QED_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up */
    QED_ERR_NOMEM = 5,      /* the context could not allocate its own work memory */
    QED_ERR_STATE = 6       /* call not valid in the context's current state */
} qed_status;

enum { QED_FP64 = 0,        /* all arithmetic and storage in FP64 */
       QED_FP32 = 1 };      /* FP32 storage, push, rates and sampling; chi in a
                               cancellation-free FP32 form with an FP64 fallback
                               where cancellation is detected; the event clock of
                               the sub-steps after a particle's first in FP64;
                               lepton displacements below 2^-16 |x| rounded
                               stochastically (unbiased, keyed by id and step) */
enum { QED_SAMPLER_TABLE = 0, QED_SAMPLER_MLP = 1 };
enum { QED_ELECTRON = 0, QED_POSITRON = 1, QED_PHOTON = 2 };

/* Analytic field descriptors (the device cannot call a host field_fn).
 *  QED_FIELD_UNIFORM     params[0..2] = E, params[3..5] = B (constant)
 *  QED_FIELD_ROTATING_E  params[0] = a0:  E = a0 (cos t, sin t, 0), B = 0
 *  QED_FIELD_STANDING_CP params[0] = a0:  standing circularly polarised wave
 *                        E = a0 cos x (0, cos t, sin t), B = a0 sin x (0, cos t, sin t)
 *                        (electric antinode at x = 0; Sec. 5.1 test problem) */
/*  QED_FIELD_GRID        a PIC step's fields on a periodic node grid, held
 *                        constant during the step: params = (nx, ny, nz, Lx,
 *                        Ly, Lz); node (i, j, k) at (i Lx/nx, j Ly/ny, k Lz/nz);
 *                        values from qed_set_field_grid; trilinear
 *                        interpolation (lerp in x, then y, then z) */
enum { QED_FIELD_UNIFORM = 0, QED_FIELD_ROTATING_E = 1, QED_FIELD_STANDING_CP = 2, QED_FIELD_GRID = 3 };

typedef struct {
    int precision;            /* QED_FP64 or QED_FP32 */
    int sampler;              /* QED_SAMPLER_TABLE (QED_SAMPLER_MLP once trained) */
    uint64_t seed;            /* Philox key */
    int push_photons;         /* 1: photons are pushed and may create pairs;
                                 0: emitted photons are recorded, not pushed */
    int soft_photon_filter;   /* 1: emitted photons below 2 m c^2 are dropped (Sec. 4.2) */
    int64_t thin_cap;         /* global leveling cap per species; 0 = off (Sec. 5.1) */
    int restore_on_overflow;  /* 1: on QED_ERR_CAPACITY the particle buffers are put
                                 back to their state at the start of the call */
    int block_threads;        /* threads per block of the push kernels; 0 = default */
    int blocks_per_sm;        /* resident blocks per SM of the push kernels; 0 = default */
    int profile;              /* 1: time the push kernels with CUDA events on the context's
                                 stream (qed_stats.kernel_ms) */
    int batch_step_budget;    /* qed_batch_push: waiting-time iterations a lepton runs before
                                 it rejoins its block's queue (1..64); 0 = the autotuner's
                                 choice, else 4 */
    int event_method;         /* QED_METHOD_SUBSTEP (Algorithm 1, default) or
                                 QED_METHOD_OPTICAL_DEPTH (see below) */
    int pass_limit;           /* newborn passes (Algorithm 2 sweeps) a step may run; a
                                 step that needs more stops there and the call returns
                                 QED_ERR_TIMEOUT; 0 = 100000 */
    int wait_polls;           /* polls of each grid barrier inside qed_train_surrogate
                                 before the launch gives up (QED_ERR_TIMEOUT); 0 = 2^24 */
    int reserved[1];
} qed_config;

/* Event methods of qed_push_and_generate.
 *  QED_METHOD_SUBSTEP        Algorithm 1 (Sec. 3): waiting times drawn inside the
 *                            step, any number of events per step, newborns pushed
 *                            to the step end (Algorithm 2).
 *  QED_METHOD_OPTICAL_DEPTH  the inverse-sampling scheme of other PIC codes that
 *                            Sec. 3 describes (accumulated optical depth, no
 *                            sub-cycling): each particle carries its remaining
 *                            optical depth od (the context's precision, arrays
 *                            from qed_set_optical_depth).  Per step:
 *                            the rate lambda at the step start; od <= 0 means "not
 *                            drawn yet" and draws od = -ln u, u from Philox(id, step,
 *                            0xFFFFFFFE) words 0-1; od -= lambda dt; push by dt; if
 *                            od <= 0 the event happens at the end of the step (chi
 *                            at the end point, energy from Philox(id, step, 0) words
 *                            2-3) and od = -ln u with words 0-1.  At most one event
 *                            per particle and step; newborns (od = 0) start at the
 *                            next step. */
enum { QED_METHOD_SUBSTEP = 0, QED_METHOD_OPTICAL_DEPTH = 1 };

/* One species: structure of arrays (Sec. 4.1), one array set per particle
 * type.  x..w are double (QED_FP64) or float (QED_FP32) device arrays of
 * `capacity` elements, each 16-byte aligned; id and nevents likewise.
 * `count` is read on entry and updated on return. */
typedef struct {
    void *x, *y, *z, *px, *py, *pz, *w;
    uint64_t *id;             /* unique 64-bit particle id (keys the random streams) */
    uint32_t *nevents;        /* cumulative number of QED events of this particle */
    int64_t count, capacity;
} qed_species;

typedef struct { qed_species s[3]; } qed_particles;  /* e-, e+, photon */

typedef struct { int kind; double params[16]; } qed_field_desc;

typedef struct {
    int64_t particle_steps;   /* sum over steps of particles pushed (newborns included) */
    int64_t emit_events;      /* photon emissions (nonlinear Compton) */
    int64_t pair_events;      /* pair creations (nonlinear Breit-Wheeler) */
    int64_t needed_capacity[3];
    int64_t max_subevents;    /* largest number of events of one particle in one step */
    int64_t overflow;         /* 1 if a species ran out of capacity */
    int64_t passes;           /* newborn passes run (Algorithm 2 sweeps) */
    int64_t thinned;          /* particles removed by leveling */
    int64_t lepton_steps;     /* particle-steps done by the lepton kernel */
    int64_t photon_steps;     /* particle-steps done by the photon kernel */
    int64_t launches;         /* kernels launched by the call */
    int64_t chi_fp64;         /* FP32 mode: chi evaluations whose cancellation test sent
                                 them to the FP64 form */
    double kernel_ms[4];      /* with cfg.profile: summed device time (CUDA events on the
                                 context's stream) of the lepton push kernels, the photon
                                 push kernels, the dead-photon compaction, and leveling */
    double sync_ms;           /* host time spent waiting in stream synchronisation */
    double call_ms;           /* host wall time of the call (of a batch: from its opening
                                 qed_push_async to the end of qed_push_wait) */
    int64_t moved;            /* entries moved into holes by the merge step (Sec. 4.2);
                                 holes left in place (deferred) are counted when filled */
} qed_stats;

/* Create a context and build its rate approximant and inverse-CDF tables on
 * the device (Sec. 3: "polynomial approximations" of precomputed rates and
 * 2-D inverse-CDF tables over chi and energy).
 *  ctx          out: new context (host pointer to opaque handle)
 *  cfg          in: configuration (copied)
 *  cuda_stream  in: cudaStream_t for all work of this context (NULL = default stream)
 * Tables: rate = Chebyshev interpolant of degree 10 per decade of log10 chi
 * (emission F/chi on [1e-3,1e3], pair ln F + 8/(3 chi) on [1e-2,1e3]);
 * inverse CDF bilinear in (log10 chi, logit u) on 121 x 257 (emission,
 * stores ln y, y = 2 delta/(3 chi (1-delta))) and 101 x 129 (pair, u <= 1/2,
 * stores ln delta) nodes, each node the root of the exact LCFA CDF. */
qed_status qed_init_tables(qed_ctx **ctx, const qed_config *cfg, void *cuda_stream);

/* Push every particle through `nsteps` PIC steps of length dt, starting at
 * step index step0 (time t = step * dt), generating photons and pairs
 * (Sec. 3, Algorithm 1 per particle, Algorithm 2 for the avalanche: every
 * particle born inside a step is pushed to the end of that step).  Dead
 * photons are removed and, with thin_cap > 0, each species is leveled after
 * every step.  Counts in *p are updated.  On QED_ERR_CAPACITY the demand is in
 * out->needed_capacity and, with restore_on_overflow, *p is as on entry; grow
 * the buffers and call again to obtain the identical result.
 *  out may be NULL. */
qed_status qed_push_and_generate(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field,
                                 double dt, int nsteps, int64_t step0, qed_stats *out);

/* The same steps without waiting for the GPU: qed_push_async enqueues them
 * and returns; qed_push_wait waits for everything enqueued since the batch
 * opened and reports it.  qed_push_and_generate is qed_push_async followed
 * by qed_push_wait.
 *
 * A batch opens with the first qed_push_async after a wait (or after the
 * context was created): the counts and capacities of *p go to the device,
 * and with restore_on_overflow the particle state is copied aside.  Later
 * calls of the batch must pass the same arrays and capacities (else
 * QED_ERR_STATE); their counts are not read, because the device holds the
 * current counts until qed_push_wait writes them into *p.  step0 may jump
 * (the steps run in call order with the indices given).
 *
 * Each step runs as one CUDA graph launch (Sec. 3, Algorithms 1-2): the
 * step-start passes, a device-side loop over newborn passes (bounded by
 * 100000 passes per step, QED_ERR_TIMEOUT beyond), and per species the merge
 * step -- leveling when the count exceeds thin_cap, converted photons removed
 * -- decided by the device.  The host never waits inside a batch.  With
 * cfg.profile (per-kernel events) or without conditional graph nodes, the
 * steps are driven from the host instead (the same kernels; the host reads
 * the control block between passes).
 *
 * After a species runs out of capacity, every later step of the batch does
 * nothing; qed_push_wait returns QED_ERR_CAPACITY with the demand in
 * out->needed_capacity and, with restore_on_overflow, *p back at its state
 * when the batch opened (grow and replay the whole batch).
 * While a batch is open, qed_compact, qed_level_eval, qed_level_apply,
 * qed_batch_push, qed_autotune_batch, qed_eval_chi and qed_set_optical_depth
 * return QED_ERR_STATE.
 *  qed_push_async: QED_OK, or an argument / state error (nothing enqueued).
 *  qed_push_wait: the status of the batch; QED_ERR_STATE when none is open
 *                 or *p holds other arrays.  out may be NULL. */
qed_status qed_push_async(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt, int nsteps,
                          int64_t step0);
qed_status qed_push_wait(qed_ctx *ctx, qed_particles *p, qed_stats *out);

/* Remove dead particles (weight 0) from every species, then, with thin_cap > 0,
 * apply global leveling at step index `step` (Sec. 4.2 merge step, Sec. 5.1).
 * Leveling: threshold w* with sum_i min(1, w_i/w*) = cap; particle i kept with
 * probability min(1, w_i/w*) (Philox counter word 3 = 0xFFFFFFFF); kept
 * particles below w* get weight w*.  Counts in *p are updated. */
qed_status qed_compact(qed_ctx *ctx, qed_particles *p, int64_t step);

/* Push n_ens independent ensembles (ens[k] in the field fields[k]) through
 * nsteps steps in one persistent launch (replayed from a CUDA graph): the
 * emission step of Sec. 3 / Algorithm 1 for every lepton, photons recorded
 * and not pushed.  With photons not pushed and no leveling nothing couples
 * particles across steps, so each lepton is carried through all steps in
 * registers (read and written once); tiles of all ensembles are scheduled
 * by a device work counter.  Results equal nsteps calls of
 * qed_push_and_generate.  Requires cfg.push_photons == 0 and thin_cap == 0
 * (else QED_ERR_INVALID).  ens: n_ens host structs of caller-owned device
 * arrays; photon counts are updated; on QED_ERR_CAPACITY (a photon buffer
 * too small) out->needed_capacity[2] holds the largest demand and the
 * lepton arrays have been advanced (not restored): replay from a copy.
 * Block shape: cfg.block_threads if 128, 256 or 512, else the autotuner's
 * choice (qed_autotune_batch), else 256. */
qed_status qed_batch_push(qed_ctx *ctx, qed_particles *ens, const qed_field_desc *fields, int n_ens,
                          double dt, int nsteps, int64_t step0, qed_stats *out);

/* Autotuner of qed_batch_push: times block shapes of 128, 256 and 512
 * threads (one tile of particles per block), each with step budgets of 1, 2
 * and 4 (cfg.batch_step_budget), for nsteps steps on scratch copies of up to
 * 2^20 leptons sampled from ens (the caller's buffers are not modified) and
 * keeps the fastest pair for this context.  *chosen_threads and ms3[3]
 * (device ms per block shape, at its best budget) may be NULL. */
qed_status qed_autotune_batch(qed_ctx *ctx, const qed_particles *ens, const qed_field_desc *fields,
                              int n_ens, double dt, int nsteps, int *chosen_threads, double *ms3);

/* The block shape and step budget qed_batch_push uses in this context (the
 * configured ones, else the autotuner's, else 256 and 4).  Host only. */
qed_status qed_batch_shape(qed_ctx *ctx, int *threads, int *step_budget);

/* ---- learned surrogate of the emission sampler ------------------------
 * An extension of the method (the paper samples from tables only): a network
 * 2 -> 64 -> 64 -> 64 -> 1 with SiLU hidden layers, BF16 weights and FP32
 * accumulation, maps features (log10(chi)/3, logit(u)/16) to zeta/16 + 1/2,
 * zeta = ln y, y = 2 delta / (3 chi (1 - delta)) (the quantity the emission
 * table stores).  Parameter layout (8577 floats, W[out][in] row-major):
 * W1[64][2], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4.
 * With cfg.sampler == QED_SAMPLER_MLP the lepton push draws photon energies
 * from the network for chi in [1e-3, 1e3] and |logit u| < 16, and from the
 * table elsewhere. */

/* Train on n_samples draws (log10 chi uniform on [-3, 3], u uniform) labelled
 * by the emission table, in batches of `batch` (a multiple of 128): forward
 * and backward passes on the tensor cores (tcgen05, accumulators in tensor
 * memory), Adam, learning rate decaying from lr to lr/100 (cosine).  Every
 * step runs inside one cooperative launch (one CTA per SM at most, a grid
 * barrier per step); the call allocates its scratch, blocks until the
 * launch ends and frees it.  *final_loss (may be NULL): mean squared error
 * over the last 16 batches.  QED_ERR_TIMEOUT if a grid barrier or a
 * tensor-core wait inside the launch ran out (bounded waits); the
 * parameters are then left as they were before the call's first step
 * (the freshly initialised network). */
qed_status qed_train_surrogate(qed_ctx *ctx, int64_t n_samples, int batch, double lr, uint64_t seed,
                               double *final_loss);

/* Load / read the FP32 master parameters (host arrays of 8577 floats). */
qed_status qed_mlp_set_params(qed_ctx *ctx, const float *params);
qed_status qed_mlp_get_params(qed_ctx *ctx, float *params);

/* Network output for n feature pairs (feat_dev: n x 2 floats, y_dev: n
 * floats, both on the device), with the BF16 weights. */
qed_status qed_mlp_forward(qed_ctx *ctx, const float *feat_dev, int64_t n, float *y_dev);

/* Gradient of the mean squared error (1/n) sum (y - target)^2 over n given
 * samples, without updating anything (grad: host array of 8577 floats;
 * *loss may be NULL).  Same kernel as the training, one pass over the
 * samples; activations and deltas are rounded to BF16 where the products
 * read them, as in the training. */
qed_status qed_mlp_grad(qed_ctx *ctx, const float *feat_dev, const float *target_dev, int64_t n,
                        float *grad, double *loss);

/* ---- leveling of one species split over several processes ------------
 * Global leveling (Sec. 5.1) when a species is sharded across GPUs (one
 * process each): the threshold w* solves sum_i min(1, w_i/w*) = cap over ALL
 * shards, so each iteration needs the shards' sums added together (an
 * all-reduce, done by the caller).  Protocol, identical on every rank:
 *     qed_level_begin(&st);
 *     while (!st.done) {
 *         qed_level_eval(ctx, &my_species, s, st.w, &A, &C, &N, &M);
 *         all-reduce: A, C, N summed, M maximum over the ranks;
 *         qed_level_advance(&st, A, C, N, M, cap);
 *     }
 *     qed_level_apply(ctx, &my_particles, s, st.wstar, step);
 * The iteration is the one a single GPU runs on the device (piecewise-exact
 * Newton steps inside a bisection bracket), so every rank holds the same
 * state after each advance.  (The device iteration also reduces the bounds
 * of the evaluated piece and stops one pass early when the Newton point
 * lies between them; the threshold is the same.)  Keep/drop draws are keyed on particle id and
 * step, so the survivors do not depend on how the species is split. */
typedef struct {
    double lo, hi;      /* bracket of w*: S(lo) > cap >= S(hi) */
    double w;           /* point to evaluate next (+inf before the first pass) */
    double wstar;       /* threshold once done (0: the species fits, no thinning) */
    int64_t iters;      /* passes taken */
    int64_t done;       /* nonzero once wstar is final */
    int64_t alive;      /* alive particles over all shards (set by the first pass) */
} qed_level_state;

/* Start an iteration (w = +inf, not done).  Host only.  The caller may set
 * st->w to a finite warm start (for example the previous step's wstar)
 * before the first advance: the first sums are then taken there, which
 * changes the number of passes, not the threshold.  The single-GPU leveling
 * starts each species at its previous threshold in this way. */
void qed_level_begin(qed_level_state *st);

/* Advance with the summed shard values at st->w: A = sum of alive weights
 * below w, C = alive count at or above w, N = alive count, max_w = largest
 * alive weight.  Host only (no GPU work).  QED_ERR_INVALID for negative
 * inputs or cap <= 0. */
qed_status qed_level_advance(qed_level_state *st, double A, int64_t C, int64_t N, double max_w, int64_t cap);

/* This shard's sums at point w (w > 0, +inf allowed) for species `species`
 * of the context's precision: one device pass over sp->w (caller-owned).
 * Synchronises the context's stream. */
qed_status qed_level_eval(qed_ctx *ctx, const qed_species *sp, int species, double w, double *A, int64_t *C,
                          int64_t *N, double *max_w);

/* Apply threshold wstar to species `species` of this shard at step index
 * `step` (keep with probability min(1, w_i/wstar), survivors below wstar get
 * wstar; wstar = 0: compaction only), then remove dead entries; count in *p
 * is updated. */
qed_status qed_level_apply(qed_ctx *ctx, qed_particles *p, int species, double wstar, int64_t step);

/* Node values of the gridded field (QED_FIELD_GRID) for the following calls:
 * grid_dev holds 6 * nz * ny * nx values of the context's precision (double
 * for QED_FP64, float for QED_FP32), layout [component][k][j][i] with the
 * components E_x, E_y, E_z, B_x, B_y, B_z.  Caller-owned device memory,
 * read (not copied) by every push with a QED_FIELD_GRID descriptor; the
 * caller may rewrite it between calls (a PIC code's new fields each step).
 * NULL detaches it.  The batched push does not take gridded fields. */
qed_status qed_set_field_grid(qed_ctx *ctx, const void *grid_dev);

/* Optical-depth arrays for QED_METHOD_OPTICAL_DEPTH: od_dev[s] holds one value
 * of the context's precision (double for QED_FP64, float for QED_FP32) per
 * particle of species s (caller-owned device memory, at least the species'
 * capacity, aligned to the element size), parallel to the species arrays: the
 * library reads and writes it in the pushes, moves it with the particles in
 * compaction and leveling, and writes 0 for every particle it appends.
 * Rebind after reallocating.  NULL entries detach.  QED_ERR_INVALID for a
 * misaligned pointer. */
qed_status qed_set_optical_depth(qed_ctx *ctx, void *const od_dev[3]);

/* Statistics accumulated since the context was created or last reset. */
qed_status qed_get_stats(qed_ctx *ctx, qed_stats *out, int reset);

const char *qed_strerror(qed_status s);
void qed_destroy(qed_ctx *ctx);

/* ---- component entry points, used by the parity tests ---------------- */

/* Philox4x32-10 on the device: out_dev[4i..4i+3] = Philox(ctr_dev[4i..4i+3], key)
 * with key words (key low, key high).  n counters; both arrays 4n uint32. */
qed_status qed_philox(const uint32_t *ctr_dev, int64_t n, uint64_t key, uint32_t *out_dev,
                      void *cuda_stream);

/* Copy the context's FP64 tables to host arrays of 66, 55, 121*257 and
 * 101*129 doubles (any pointer may be NULL). */
qed_status qed_get_tables(qed_ctx *ctx, double *cheb_em, double *cheb_pair,
                          double *icdf_em, double *icdf_pair);

/* Rate approximant F(chi) at n points, in the context's precision
 * (chi_dev, F_dev: n doubles on the device).  is_photon selects the pair rate. */
qed_status qed_eval_rate(qed_ctx *ctx, int is_photon, const double *chi_dev, int64_t n, double *F_dev);

/* Quantum parameter chi = sqrt((e0 E + p x B)^2 - (p.E)^2) / R (Algorithm 1,
 * Calculate chi) of n particles, in the context's precision: FP64 mode the
 * direct form in FP64; FP32 mode the inputs rounded to FP32 and the
 * cancellation-free split S + T (Lagrange's identity) in FP32, with the direct
 * FP64 form where the cancellation test fails.  e0 = sqrt(1 + p^2) (lepton) or
 * |k| (photon).  p_dev, E_dev, B_dev: n x 3 doubles on the device; chi_dev: n
 * doubles on the device; *n_fp64 (host, may be NULL): how many took the FP64 form. */
qed_status qed_eval_chi(qed_ctx *ctx, int is_photon, const double *p_dev, const double *E_dev,
                        const double *B_dev, int64_t n, double *chi_dev, int64_t *n_fp64);

/* Energy fraction delta (and 1 - delta) drawn by inverse CDF at (chi, u), in
 * the context's precision: emission (photon fraction) or pair (electron
 * fraction).  All arrays n doubles on the device. */
qed_status qed_sample(qed_ctx *ctx, int is_photon, const double *chi_dev, const double *u_dev,
                      int64_t n, double *delta_dev, double *one_minus_dev);

/* ---- measurement ------------------------------------------------------
 * FP64 arithmetic rate of the current device, the roofline denominator of the
 * FP64 mode (every step of Algorithm 1 in FP64): one wave of resident blocks,
 * each thread running eight independent FP64 fused multiply-add chains of
 * `iters` steps (2 FLOPs each), timed with CUDA events on cuda_stream (NULL =
 * default stream); best of three launches after a warm-up.  *flops_per_s
 * receives the rate, *ms (may be NULL) the best launch's duration.
 * QED_ERR_INVALID for iters <= 0 or a null flops_per_s; synchronises the
 * stream. */
qed_status qed_measure_fp64_peak(int iters, double *flops_per_s, double *ms, void *cuda_stream);

/* ---- compaction for callers that cannot allocate --------------------- */

/* Largest species count qed_compact_species_noalloc() accepts. */
#define QED_NOALLOC_MAX_ENTRIES (1 << 20)

/* Remove dead entries (weight 0) from one species without allocating any
 * memory.  The paper has no counterpart: this exists for callers that cannot
 * call cudaMalloc, such as a host code whose device memory belongs entirely
 * to its own pool allocator, or a time loop that cannot accept the
 * device-wide synchronisation cudaMalloc / cudaFree may cause.
 *  sp           in/out: caller-owned device arrays (16-byte aligned); count is
 *               read and updated (alive entries end up in [0, count))
 *  od_dev       the species' optical-depth array (QED_METHOD_OPTICAL_DEPTH: one
 *               value of the precision's type per particle, caller-owned,
 *               aligned to the element size), moved with the particles like
 *               the arrays of *sp; NULL when there is none (the sub-step method)
 *  precision    QED_FP64 (double arrays) or QED_FP32 (float arrays)
 *  cuda_stream  stream for the work (NULL = default stream); synchronised
 *               before returning
 * Same result as the compaction inside qed_compact() with the same
 * optical-depth array bound: the r-th dead slot below the new count receives
 * the r-th alive entry at or above it.
 * Scratch: one file-scope device array of about 8 MB holding control words,
 * per-block counts and hole ranks, kept by every GPU that loads the library
 * until the process exits.  No context is needed and nothing is allocated:
 * no cudaMalloc, cudaFree or allocating library routine.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents (each call
 * resets the words it needs), so calls that overlap on the GPU -- from
 * several threads or streams at once -- race and corrupt each other.
 * Errors: QED_ERR_INVALID for a null or misaligned array, an unknown
 * precision, count < 0 or > capacity, or count > QED_NOALLOC_MAX_ENTRIES;
 * QED_ERR_STATE if a bounds check inside the kernels failed; QED_ERR_CUDA. */
qed_status qed_compact_species_noalloc(qed_species *sp, void *od_dev, int precision, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SFQED_H */
