// C-ABI entry points (declared and documented in include/sfqed.h).
#include <stdlib.h>
#include <string.h>

#include "sfqed_internal.h"

using namespace sfq;

static void free_ctx(qed_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    sfq_batch_free(c);
    sfq_level_graphs_free(c);
    sfq_step_graph_free(c);
    void *dev[] = {c->coef64, c->coef32, c->icdf_em64, c->icdf_pair64, c->icdf_em32, c->icdf_pair32, c->gl,
                   c->ctl, c->tau[0], c->tau[1], c->tau[2], c->blk, c->slots, c->snap, c->lev,
                   c->mlp_p, c->mlp_w16, c->mlp_loss};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    if (c->ctl_up) cudaFreeHost(c->ctl_up);
    if (c->pin) cudaFreeHost(c->pin);
    if (c->grid_il) cudaFree(c->grid_il);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->ev_ready)
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < qed_ctx::EVN; ++i)
                for (int j = 0; j < 2; ++j) cudaEventDestroy(c->ev[k][i][j]);
    free(c);
}

extern "C" qed_status qed_init_tables(qed_ctx **out, const qed_config *cfg, void *cuda_stream) {
    if (!out || !cfg) return QED_ERR_INVALID;
    *out = nullptr;
    if (cfg->precision != QED_FP64 && cfg->precision != QED_FP32) return QED_ERR_INVALID;
    if (cfg->sampler != QED_SAMPLER_TABLE && cfg->sampler != QED_SAMPLER_MLP) return QED_ERR_INVALID;
    if (cfg->thin_cap < 0 || cfg->block_threads < 0 || cfg->block_threads > 1024 || cfg->block_threads % 32 ||
        cfg->blocks_per_sm < 0)
        return QED_ERR_INVALID;
    qed_ctx *c = static_cast<qed_ctx *>(calloc(1, sizeof(qed_ctx)));
    if (!c) return QED_ERR_NOMEM;
    c->cfg = *cfg;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        free(c);
        return QED_ERR_CUDA;
    }
    bool ok = cudaMalloc(&c->coef64, sizeof(double) * NCOEF) == cudaSuccess &&
              cudaMalloc(&c->coef32, sizeof(float) * NRATE32) == cudaSuccess &&
              cudaMalloc(&c->icdf_em64, sizeof(double) * EM_NCHI * EM_NS) == cudaSuccess &&
              cudaMalloc(&c->icdf_pair64, sizeof(double) * PAIR_NCHI * PAIR_NS) == cudaSuccess &&
              cudaMalloc(&c->icdf_em32, sizeof(float) * EM_NCHI * EM_NS) == cudaSuccess &&
              cudaMalloc(&c->icdf_pair32, sizeof(float) * PAIR_NCHI * PAIR_NS) == cudaSuccess &&
              cudaMalloc(&c->gl, sizeof(double) * 64) == cudaSuccess &&
              cudaMalloc(&c->ctl, sizeof(DevCtl)) == cudaSuccess &&
              cudaMalloc(&c->lev, sizeof(LevelWork)) == cudaSuccess &&
              cudaHostAlloc(&c->ctl_host, sizeof(DevCtl), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&c->ctl_up, sizeof(DevCtl), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(&c->pin, 64, cudaHostAllocDefault) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        free_ctx(c);
        return QED_ERR_NOMEM;
    }
    if (cudaMemsetAsync(c->ctl, 0, sizeof(DevCtl), c->stream) != cudaSuccess) {
        free_ctx(c);
        return QED_ERR_CUDA;
    }
    qed_status e = sfq_build_tables(c);
    if (e != QED_OK) {
        free_ctx(c);
        return e;
    }
    *out = c;
    return QED_OK;
}

extern "C" void qed_destroy(qed_ctx *ctx) { free_ctx(ctx); }

extern "C" qed_status qed_push_and_generate(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field,
                                            double dt, int nsteps, int64_t step0, qed_stats *out) {
    return sfq_push(ctx, p, field, dt, nsteps, step0, out);
}

extern "C" qed_status qed_push_async(qed_ctx *ctx, qed_particles *p, const qed_field_desc *field, double dt,
                                     int nsteps, int64_t step0) {
    return sfq_push_async(ctx, p, field, dt, nsteps, step0);
}

extern "C" qed_status qed_push_wait(qed_ctx *ctx, qed_particles *p, qed_stats *out) {
    return sfq_push_wait(ctx, p, out);
}

extern "C" qed_status qed_batch_push(qed_ctx *ctx, qed_particles *ens, const qed_field_desc *fields, int n_ens,
                                     double dt, int nsteps, int64_t step0, qed_stats *out) {
    if (ctx && ctx->async_open) return QED_ERR_STATE;
    return sfq_batch_push(ctx, ens, fields, n_ens, dt, nsteps, step0, out, 0, 0);
}

extern "C" qed_status qed_set_optical_depth(qed_ctx *ctx, void *const od_dev[3]) {
    if (!ctx || !od_dev) return QED_ERR_INVALID;
    if (ctx->async_open) return QED_ERR_STATE;
    const uintptr_t align = ctx->cfg.precision == QED_FP32 ? 4u : 8u;
    for (int s = 0; s < 3; ++s) {
        if (od_dev[s] && (reinterpret_cast<uintptr_t>(od_dev[s]) % align)) return QED_ERR_INVALID;
        ctx->od[s] = od_dev[s];
    }
    return QED_OK;
}

extern "C" qed_status qed_set_field_grid(qed_ctx *ctx, const void *grid_dev) {
    if (!ctx) return QED_ERR_INVALID;
    if (grid_dev && (reinterpret_cast<uintptr_t>(grid_dev) % (ctx->cfg.precision == QED_FP32 ? 4 : 8)))
        return QED_ERR_INVALID;
    ctx->field_grid = grid_dev;
    return QED_OK;
}

extern "C" qed_status qed_batch_shape(qed_ctx *ctx, int *threads, int *step_budget) {
    return sfq_batch_shape(ctx, threads, step_budget);
}

extern "C" qed_status qed_autotune_batch(qed_ctx *ctx, const qed_particles *ens, const qed_field_desc *fields,
                                         int n_ens, double dt, int nsteps, int *chosen_threads, double *ms3) {
    if (ctx && ctx->async_open) return QED_ERR_STATE;
    return sfq_batch_autotune(ctx, ens, fields, n_ens, dt, nsteps, chosen_threads, ms3);
}

extern "C" qed_status qed_compact(qed_ctx *ctx, qed_particles *p, int64_t step) {
    if (!ctx || !p || step < 0 || step > 0xFFFFFFFFll) return QED_ERR_INVALID;
    if (ctx->async_open) return QED_ERR_STATE;
    for (int s = 0; s < 3; ++s)
        if (p->s[s].count < 0 || p->s[s].count > p->s[s].capacity) return QED_ERR_INVALID;
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    DevCtl &h = *ctx->ctl_host;                 // pinned staging
    memset(&h, 0, sizeof(DevCtl));
    for (int s = 0; s < 3; ++s) {
        h.count[s] = (unsigned long long)p->s[s].count;
        h.capacity[s] = (unsigned long long)p->s[s].capacity;
    }
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl, &h, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    for (int s = 0; s < 3; ++s) {
        // leveling skips dead entries and compacts; otherwise compaction only
        const bool level = ctx->cfg.thin_cap > 0 && p->s[s].count > ctx->cfg.thin_cap;
        qed_status e = level ? sfq_level_species(ctx, &p->s[s], s, step) : sfq_compact_species(ctx, &p->s[s], s);
        if (e != QED_OK) return e;
    }
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->ctl_host->bad_index) return QED_ERR_STATE;
    for (int s = 0; s < 3; ++s) p->s[s].count = (int64_t)ctx->ctl_host->count[s];
    ctx->acc.thinned += (int64_t)ctx->ctl_host->thinned;
    ctx->acc.moved += (int64_t)ctx->ctl_host->moved;
    return QED_OK;
}

extern "C" void qed_level_begin(qed_level_state *st) {
    if (!st) return;
    memset(st, 0, sizeof *st);
    st->hi = INFINITY;
    st->w = INFINITY;
}

extern "C" qed_status qed_level_advance(qed_level_state *st, double A, int64_t C, int64_t N, double max_w,
                                        int64_t cap) {
    if (!st || cap <= 0 || C < 0 || N < 0 || !(A >= 0.0) || !(max_w >= 0.0)) return QED_ERR_INVALID;
    if (st->done) return QED_OK;
    sfq_level_advance(&st->lo, &st->hi, &st->w, &st->wstar, &st->iters, &st->done, &st->alive, A, C, N, max_w, cap);
    return QED_OK;
}

extern "C" qed_status qed_level_eval(qed_ctx *ctx, const qed_species *sp, int species, double w, double *A,
                                     int64_t *C, int64_t *N, double *max_w) {
    if (!ctx || !sp || !A || !C || !N || !max_w || species < 0 || species > 2 || !(w > 0.0)) return QED_ERR_INVALID;
    if (sp->count < 0 || sp->count > sp->capacity || (sp->count > 0 && !sp->w)) return QED_ERR_INVALID;
    if (ctx->async_open) return QED_ERR_STATE;
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    qed_species copy = *sp;
    return sfq_level_eval(ctx, &copy, species, w, A, C, N, max_w);
}

extern "C" qed_status qed_level_apply(qed_ctx *ctx, qed_particles *p, int species, double wstar, int64_t step) {
    if (!ctx || !p || species < 0 || species > 2 || !(wstar >= 0.0) || step < 0 || step > 0xFFFFFFFFll)
        return QED_ERR_INVALID;
    if (ctx->async_open) return QED_ERR_STATE;
    for (int s = 0; s < 3; ++s)
        if (p->s[s].count < 0 || p->s[s].count > p->s[s].capacity) return QED_ERR_INVALID;
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    DevCtl &h = *ctx->ctl_host;                 // pinned staging
    memset(&h, 0, sizeof(DevCtl));
    for (int s = 0; s < 3; ++s) {
        h.count[s] = (unsigned long long)p->s[s].count;
        h.capacity[s] = (unsigned long long)p->s[s].capacity;
    }
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl, &h, sizeof(DevCtl), cudaMemcpyHostToDevice, ctx->stream));
    qed_status e = sfq_level_apply_species(ctx, &p->s[species], species, wstar, step);
    if (e != QED_OK) return e;
    SFQ_CUDA(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, ctx->stream));
    SFQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->ctl_host->bad_index) return QED_ERR_STATE;
    p->s[species].count = (int64_t)ctx->ctl_host->count[species];
    ctx->acc.thinned += (int64_t)ctx->ctl_host->thinned;
    ctx->acc.moved += (int64_t)ctx->ctl_host->moved;
    return QED_OK;
}

extern "C" qed_status qed_get_stats(qed_ctx *ctx, qed_stats *out, int reset) {
    if (!ctx || !out) return QED_ERR_INVALID;
    *out = ctx->acc;
    if (reset) memset(&ctx->acc, 0, sizeof(ctx->acc));
    return QED_OK;
}

extern "C" const char *qed_strerror(qed_status s) {
    switch (s) {
    case QED_OK: return "ok";
    case QED_ERR_INVALID: return "invalid argument";
    case QED_ERR_CAPACITY: return "particle buffer capacity exceeded";
    case QED_ERR_CUDA: return "CUDA runtime error";
    case QED_ERR_TIMEOUT: return "bounded device wait gave up";
    case QED_ERR_NOMEM: return "out of device memory";
    case QED_ERR_STATE: return "invalid state";
    default: return "unknown status";
    }
}

extern "C" qed_status qed_philox(const uint32_t *ctr_dev, int64_t n, uint64_t key, uint32_t *out_dev,
                                 void *cuda_stream) {
    return sfq_philox(ctr_dev, n, key, out_dev, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" qed_status qed_get_tables(qed_ctx *ctx, double *cheb_em, double *cheb_pair, double *icdf_em,
                                     double *icdf_pair) {
    if (!ctx) return QED_ERR_INVALID;
    cudaStream_t st = ctx->stream;
    if (cheb_em) SFQ_CUDA(cudaMemcpyAsync(cheb_em, ctx->coef64, sizeof(double) * EM_NDEC * CHEB_N, cudaMemcpyDeviceToHost, st));
    if (cheb_pair)
        SFQ_CUDA(cudaMemcpyAsync(cheb_pair, ctx->coef64 + EM_NDEC * CHEB_N, sizeof(double) * PAIR_NDEC * CHEB_N,
                                 cudaMemcpyDeviceToHost, st));
    if (icdf_em) SFQ_CUDA(cudaMemcpyAsync(icdf_em, ctx->icdf_em64, sizeof(double) * EM_NCHI * EM_NS, cudaMemcpyDeviceToHost, st));
    if (icdf_pair)
        SFQ_CUDA(cudaMemcpyAsync(icdf_pair, ctx->icdf_pair64, sizeof(double) * PAIR_NCHI * PAIR_NS, cudaMemcpyDeviceToHost, st));
    SFQ_CUDA(cudaStreamSynchronize(st));
    return QED_OK;
}

extern "C" qed_status qed_eval_rate(qed_ctx *ctx, int is_photon, const double *chi_dev, int64_t n, double *F_dev) {
    return sfq_eval_rate(ctx, is_photon, chi_dev, n, F_dev);
}

extern "C" qed_status qed_eval_chi(qed_ctx *ctx, int is_photon, const double *p_dev, const double *E_dev,
                                   const double *B_dev, int64_t n, double *chi_dev, int64_t *n_fp64) {
    if (ctx && ctx->async_open) return QED_ERR_STATE;
    return sfq_eval_chi(ctx, is_photon, p_dev, E_dev, B_dev, n, chi_dev, n_fp64);
}

extern "C" qed_status qed_sample(qed_ctx *ctx, int is_photon, const double *chi_dev, const double *u_dev, int64_t n,
                                 double *delta_dev, double *one_minus_dev) {
    return sfq_sample(ctx, is_photon, chi_dev, u_dev, n, delta_dev, one_minus_dev);
}

extern "C" qed_status qed_train_surrogate(qed_ctx *ctx, int64_t n_samples, int batch, double lr, uint64_t seed,
                                          double *final_loss) {
    return sfq_mlp_train(ctx, n_samples, batch, lr, seed, final_loss);
}

extern "C" qed_status qed_mlp_set_params(qed_ctx *ctx, const float *params) { return sfq_mlp_set_params(ctx, params); }

extern "C" qed_status qed_mlp_get_params(qed_ctx *ctx, float *params) { return sfq_mlp_get_params(ctx, params); }

extern "C" qed_status qed_mlp_forward(qed_ctx *ctx, const float *feat_dev, int64_t n, float *y_dev) {
    return sfq_mlp_eval(ctx, feat_dev, n, y_dev);
}

extern "C" qed_status qed_mlp_grad(qed_ctx *ctx, const float *feat_dev, const float *target_dev, int64_t n,
                                   float *grad, double *loss) {
    return sfq_mlp_grad(ctx, feat_dev, target_dev, n, grad, loss);
}
