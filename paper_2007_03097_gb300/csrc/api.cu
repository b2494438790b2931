// C ABI of the library (include/sph.h): context life cycle, argument checks,
// and the orchestration of the hot path on the caller's stream.
#include <cmath>
#include <cstring>

#include <algorithm>
#include <climits>

#include "sph_internal.cuh"

int hnet_refresh_bf16(sph_ctx *ctx, cudaStream_t s);

namespace {

template <typename T>
int alloc(sph_ctx *ctx, T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        *p = nullptr;
        return SPH_ERR_CUDA;
    }
    return SPH_OK;
}

int check_params(const sph_params *q, std::string &why)
{
    if (!q) { why = "params is NULL"; return SPH_ERR_ARG; }
    if (q->kernel < 0 || q->kernel > 2) { why = "kernel must be 0 (M4), 1 (WC2) or 2 (WC4)"; return SPH_ERR_ARG; }
    if (q->precision != SPH_FP64 && q->precision != SPH_MIXED) { why = "precision must be 0 or 1"; return SPH_ERR_ARG; }
    if (!(q->gamma > 1.0)) { why = "gamma must exceed 1"; return SPH_ERR_ARG; }
    if (!(q->eta > 0.0)) { why = "eta must be positive"; return SPH_ERR_ARG; }
    if (!(q->alpha >= 0.0) || !(q->beta >= 0.0) || !(q->eps_visc > 0.0)) { why = "viscosity parameters out of range"; return SPH_ERR_ARG; }
    if (!(q->cfl > 0.0)) { why = "cfl must be positive"; return SPH_ERR_ARG; }
    if (!(q->h_tol > 0.0)) { why = "h_tol must be positive"; return SPH_ERR_ARG; }
    if (q->max_sweeps < 1 || q->max_sweeps > 1000) { why = "max_sweeps must be in [1, 1000]"; return SPH_ERR_ARG; }
    if (q->leaf_size < 1 || q->leaf_size > 32) { why = "leaf_size must be in [1, 32]"; return SPH_ERR_ARG; }
    if (!(q->h_min > 0.0) || !(q->h_max > q->h_min)) { why = "need 0 < h_min < h_max"; return SPH_ERR_ARG; }
    if (!(q->skin >= 0.0) || q->skin > 1.0) { why = "skin must be in [0, 1]"; return SPH_ERR_ARG; }
    if (!(q->rho_ref > 0.0)) { why = "rho_ref must be positive"; return SPH_ERR_ARG; }
    if (q->nb_capacity < 0) { why = "nb_capacity must be >= 0"; return SPH_ERR_ARG; }
    if (q->energy != SPH_ENERGY_INTERNAL && q->energy != SPH_ENERGY_TOTAL) { why = "energy must be an sph_energy"; return SPH_ERR_ARG; }
    if (q->curve != SPH_CURVE_MORTON && q->curve != SPH_CURVE_HILBERT) { why = "curve must be an sph_curve"; return SPH_ERR_ARG; }
    if (q->dim != 1 && q->dim != 3) { why = "dim must be 1 or 3"; return SPH_ERR_ARG; }
    if (!(q->hnet_lr > 0.0) || q->hnet_batch < 1 || q->hnet_iters < 0 || q->hnet_iters > 10000) {
        why = "need hnet_lr > 0, hnet_batch >= 1, 0 <= hnet_iters <= 10000";
        return SPH_ERR_ARG;
    }
    if (q->periodic) {
        const double L = q->box_hi[0] - q->box_lo[0];
        if (!(L > 0.0) || q->box_hi[1] - q->box_lo[1] != L || q->box_hi[2] - q->box_lo[2] != L) {
            why = "a periodic box must be a cube with positive side";
            return SPH_ERR_ARG;
        }
        if (q->h_max > 0.25 * L) { why = "periodic box: h_max must not exceed a quarter of the side"; return SPH_ERR_ARG; }
    }
    return SPH_OK;
}

template <typename T>
bool aligned(const void *p)
{
    return p && ((uintptr_t)p % sizeof(T)) == 0;
}

int check_particles(sph_ctx *ctx, const sph_particles *p, bool need_tree)
{
    if (!ctx) return SPH_ERR_ARG;
    if (!p) return sph_fail(ctx, SPH_ERR_ARG, "particles is NULL");
    if (p->n < 1 || p->n > ctx->n_max) return sph_fail(ctx, SPH_ERR_ARG, "n must be in [1, n_max]");
    const void *dbl[] = {p->x, p->y, p->z};
    for (const void *a : dbl)
        if (!aligned<double>(a)) return sph_fail(ctx, SPH_ERR_ARG, "x, y, z must be non-NULL 8-byte aligned device arrays");
    const void *fl[] = {p->vx, p->vy, p->vz, p->m, p->h, p->u, p->hprev, p->rho, p->omega, p->P, p->c,
                        p->ax, p->ay, p->az, p->dudt, p->divv, p->vsig};
    for (const void *a : fl) {
        bool ok = ctx->fp64 ? aligned<double>(a) : aligned<float>(a);
        if (!ok) return sph_fail(ctx, SPH_ERR_ARG, "every particle array must be non-NULL and naturally aligned");
    }
    if (!aligned<int32_t>(p->nnb) || !aligned<uint32_t>(p->id))
        return sph_fail(ctx, SPH_ERR_ARG, "nnb and id must be non-NULL 4-byte aligned device arrays");
    if (need_tree && (!ctx->tree_valid || ctx->n != p->n))
        return sph_fail(ctx, SPH_ERR_STATE, "no tree for this particle set: call sph_build_tree first");
    return SPH_OK;
}

int elapsed(sph_ctx *ctx, cudaEvent_t a, cudaEvent_t b, double *ms)
{
    float f = 0.f;
    SPH_CUDA(cudaEventElapsedTime(&f, a, b));
    *ms = f;
    return SPH_OK;
}

int allocate(sph_ctx *c, int64_t N)
{
    sph_ctx *ctx = c;   // for SPH_CUDA
    const int64_t tiles = (N + 4095) / 4096;
    c->hist_cap = 256 * tiles;
    SPH_TRY(alloc(c, &c->key_a, N));
    SPH_TRY(alloc(c, &c->key_b, N));
    SPH_TRY(alloc(c, &c->val_a, N));
    SPH_TRY(alloc(c, &c->val_b, N));
    SPH_TRY(alloc(c, &c->hist, (size_t)c->hist_cap));
    SPH_TRY(alloc(c, &c->ns_tiles, (size_t)(N / 1024 + 2)));
    SPH_TRY(alloc(c, &c->dlev, N));
    SPH_TRY(alloc(c, &c->plev, N));
    SPH_TRY(alloc(c, &c->itmp0, N + 1));
    SPH_TRY(alloc(c, &c->itmp1, N + 1));
    SPH_TRY(alloc(c, &c->itmp2, N + 1));
    SPH_TRY(alloc(c, &c->itmp3, N + 1));
    SPH_TRY(alloc(c, &c->leaf_begin, N + 1));
    SPH_TRY(alloc(c, &c->leaf_level, N));
    SPH_TRY(alloc(c, &c->group_begin, N + 1));
    SPH_TRY(alloc(c, &c->leaf_lo, N));
    SPH_TRY(alloc(c, &c->leaf_hi, N));
    SPH_TRY(alloc(c, &c->group_lo, N));
    SPH_TRY(alloc(c, &c->group_hi, N));
    SPH_TRY(alloc(c, &c->node_child, 2 * N));
    SPH_TRY(alloc(c, &c->node_parent, N));
    SPH_TRY(alloc(c, &c->leaf_parent, N));
    SPH_TRY(alloc(c, &c->node_visit, N));
    SPH_TRY(alloc(c, &c->node_delta, N));
    SPH_TRY(alloc(c, &c->cell_table, (size_t)cell_table_size()));
    SPH_TRY(alloc(c, &c->node_lo, N));
    SPH_TRY(alloc(c, &c->node_hi, N));
    float4 **packs[] = {&c->srcA, &c->srcB, &c->srcC, &c->srcD, &c->srcE, &c->srcF};
    for (float4 **s : packs) SPH_TRY(alloc(c, s, N));
    c->nbl_cap = c->prm.nb_capacity > 0 ? c->prm.nb_capacity : 640 * N;
    SPH_TRY(alloc(c, &c->nbl, (size_t)c->nbl_cap));
    SPH_TRY(alloc(c, &c->group_width, N));
    SPH_TRY(alloc(c, &c->group_off, N + 1));
    // union slots: exact unions never exceed the exact lists; the leaf-bound
    // sizing needs about 30 per particle at ~100 neighbours
    c->uni_cap = c->prm.nb_capacity > 0 ? c->prm.nb_capacity : 64 * N;
    SPH_TRY(alloc(c, &c->uni, (size_t)c->uni_cap));
    if (!c->fp64) SPH_TRY(alloc(c, &c->urec, (size_t)c->uni_cap));
    SPH_TRY(alloc(c, &c->group_ubound, N));
    SPH_TRY(alloc(c, &c->union_off, N + 1));
    SPH_TRY(alloc(c, &c->group_union, N));
    SPH_TRY(alloc(c, &c->group_img, N));
    SPH_CUDA(cudaMemset(c->group_img, 0, sizeof(int32_t) * (size_t)N));
    SPH_TRY(alloc(c, &c->group_mark, N));
    SPH_CUDA(cudaMemset(c->group_mark, 0, sizeof(int32_t) * (size_t)N));
    c->kept_cap = 8 * N;
    SPH_TRY(alloc(c, &c->kept, (size_t)c->kept_cap));
    SPH_TRY(alloc(c, &c->kept_count, N));
    SPH_TRY(alloc(c, &c->it_lo, N));
    SPH_TRY(alloc(c, &c->it_hi, N));
    SPH_TRY(alloc(c, &c->it_flags, N));
    SPH_TRY(alloc(c, &c->it_sweeps, N));
    SPH_TRY(alloc(c, &c->cov, N));
    SPH_TRY(alloc(c, &c->lcount, N));
    SPH_TRY(alloc(c, &c->act_groups[0], N));
    SPH_TRY(alloc(c, &c->act_groups[1], N));
    double **d8[] = {(double **)&c->vpx, (double **)&c->vpy, (double **)&c->vpz, (double **)&c->upred,
                     (double **)&c->hold, (double **)&c->hseed,
                     (double **)&c->hstart};
    for (double **d : d8) SPH_TRY(alloc(c, d, N));
    c->gbuf_bytes = 24 * (((size_t)N * 8 + 255) & ~(size_t)255);
    SPH_TRY(alloc(c, &c->gbuf, c->gbuf_bytes));
    const int64_t scan_n = N > c->hist_cap ? N : c->hist_cap;
    c->scan_tmp_bytes = scan_tmp_bytes(scan_n);
    SPH_TRY(alloc(c, (unsigned char **)&c->scan_tmp, c->scan_tmp_bytes));
    c->red_blocks = 8 * c->num_sms;
    SPH_TRY(alloc(c, &c->red, (size_t)c->red_blocks * 16));
    SPH_TRY(alloc(c, &c->dcnt, 1));
    SPH_CUDA(cudaMallocHost((void **)&c->hcnt, sizeof(DevCounters)));
    std::memset(c->hcnt, 0, sizeof(DevCounters));
    SPH_CUDA(cudaMemset(c->dcnt, 0, sizeof(DevCounters)));
    // h-predictor
    SPH_TRY(alloc(c, &c->hn_master, SPH_HNET_NPARAM));
    SPH_TRY(alloc(c, &c->hn_bf16, SPH_HNET_NPARAM));
    SPH_TRY(alloc(c, &c->hn_m, SPH_HNET_NPARAM));
    SPH_TRY(alloc(c, &c->hn_v, SPH_HNET_NPARAM));
    SPH_TRY(alloc(c, &c->hn_grad, SPH_HNET_NPARAM));
    c->hn_part_blocks = 4 * c->num_sms;
    SPH_TRY(alloc(c, &c->hn_part, (size_t)c->hn_part_blocks * (SPH_HNET_NPARAM + 1)));
    SPH_TRY(alloc(c, &c->hn_sample, 6 * (size_t)c->prm.hnet_batch));
    SPH_CUDA(cudaMemset(c->hn_master, 0, sizeof(float) * SPH_HNET_NPARAM));
    SPH_CUDA(cudaMemset(c->hn_bf16, 0, sizeof(__nv_bfloat16) * SPH_HNET_NPARAM));
    SPH_CUDA(cudaMemset(c->hn_m, 0, sizeof(float) * SPH_HNET_NPARAM));
    SPH_CUDA(cudaMemset(c->hn_v, 0, sizeof(float) * SPH_HNET_NPARAM));
    for (cudaEvent_t &e : c->ev) SPH_CUDA(cudaEventCreate(&e));
    SPH_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    SPH_CUDA(cudaEventCreateWithFlags(&c->ev_dens, cudaEventDisableTiming));
    SPH_CUDA(cudaEventCreateWithFlags(&c->ev_train, cudaEventDisableTiming));
    SPH_CUDA(cudaEventCreateWithFlags(&c->ev_order, cudaEventDisableTiming));
    SPH_CUDA(cudaEventCreateWithFlags(&c->ev_seed, cudaEventDisableTiming));
    for (cudaEvent_t &e : c->kev) SPH_CUDA(cudaEventCreate(&e));
    for (cudaEvent_t &e : c->lev) SPH_CUDA(cudaEventCreate(&e));
    SPH_TRY(hnet_init(c));
    return SPH_OK;
}

void release(sph_ctx *c)
{
    void *ptrs[] = {c->key_a, c->key_b, c->val_a, c->val_b, c->hist, c->ns_tiles, c->dlev, c->plev, c->itmp0, c->itmp1,
                    c->itmp2, c->itmp3, c->leaf_begin, c->leaf_level, c->group_begin, c->leaf_lo, c->leaf_hi,
                    c->group_lo, c->group_hi, c->node_child, c->node_parent, c->leaf_parent, c->node_visit,
                    c->node_delta, c->cell_table, c->node_lo, c->node_hi, c->srcA, c->srcB,
                    c->srcC, c->srcD, c->srcE, c->srcF, c->nbl, c->group_width, c->uni, c->urec, c->group_ubound,
                    c->union_off, c->group_union, c->group_img, c->group_mark, c->kept, c->kept_count,
                    c->group_off, c->it_lo, c->it_hi, c->it_flags, c->it_sweeps, c->cov, c->lcount, c->act_groups[0],
                    c->act_groups[1], c->vpx, c->vpy, c->vpz, c->upred, c->hold, c->hseed, c->hstart, c->gbuf,
                    c->scan_tmp, c->red, c->dcnt, c->hn_master, c->hn_bf16, c->hn_m, c->hn_v, c->hn_grad,
                    c->hn_part, c->hn_sample};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_dens) cudaEventDestroy(c->ev_dens);
    if (c->ev_train) cudaEventDestroy(c->ev_train);
    if (c->ev_order) cudaEventDestroy(c->ev_order);
    if (c->ev_seed) cudaEventDestroy(c->ev_seed);
    if (c->hcnt) cudaFreeHost(c->hcnt);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->kev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->lev)
        if (e) cudaEventDestroy(e);
}

inline cudaStream_t S(void *stream) { return (cudaStream_t)stream; }

}  // namespace

int copy_field(sph_ctx *ctx, void *dst, const void *src, int64_t n, cudaStream_t s)
{
    SPH_CUDA(cudaMemcpyAsync(dst, src, (size_t)n * (ctx->fp64 ? 8 : 4), cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

int join_side(sph_ctx *ctx, cudaStream_t s, bool host)
{
    if (!ctx->side_pending) return SPH_OK;
    if (host) SPH_CUDA(cudaEventSynchronize(ctx->ev_train));
    else SPH_CUDA(cudaStreamWaitEvent(s, ctx->ev_train, 0));
    ctx->side_pending = false;
    return SPH_OK;
}

// message of the last failing context-free call of this thread
namespace {
thread_local std::string t_free_err = "no error";
}

void noalloc_fail(const std::string &msg) { t_free_err = msg; }

extern "C" {

const char *sph_version(void) { return "sph sm_103a 1.0"; }

int sph_create(const sph_params *params, int64_t n_max, sph_ctx **out)
{
    if (!out) return SPH_ERR_ARG;
    *out = nullptr;
    std::string why;
    int st = check_params(params, why);
    if (st != SPH_OK) return st;
    if (n_max < 1 || n_max > ((int64_t)1 << 31) - 64) return SPH_ERR_ARG;
    sph_ctx *c = new sph_ctx();
    c->prm = *params;
    c->n_max = n_max;
    c->fp64 = params->precision == SPH_FP64;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return SPH_ERR_CUDA;
    }
    st = allocate(c, n_max);
    if (st != SPH_OK) {
        release(c);
        delete c;
        return st;
    }
    *out = c;
    return SPH_OK;
}

void sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    release(ctx);
    delete ctx;
}

int sph_set_params(sph_ctx *ctx, const sph_params *params)
{
    if (!ctx) return SPH_ERR_ARG;
    std::string why;
    int st = check_params(params, why);
    if (st != SPH_OK) return sph_fail(ctx, st, "sph_set_params: " + why);
    if (params->precision != ctx->prm.precision) return sph_fail(ctx, SPH_ERR_ARG, "sph_set_params: precision is fixed at creation");
    if (params->hnet_batch > ctx->prm.hnet_batch)
        return sph_fail(ctx, SPH_ERR_ARG, "sph_set_params: hnet_batch cannot grow after creation");
    const int64_t cap = ctx->prm.nb_capacity;
    ctx->prm = *params;
    ctx->prm.nb_capacity = cap;
    ctx->tree_valid = false;
    return SPH_OK;
}

const char *sph_last_error(const sph_ctx *ctx) { return ctx ? ctx->err.c_str() : t_free_err.c_str(); }

int sph_build_tree(sph_ctx *ctx, sph_particles *p, void *stream)
{
    SPH_TRY(check_particles(ctx, p, false));
    SPH_TRY(join_side(ctx, S(stream)));
    return tree_build(ctx, p, S(stream));
}

int sph_density(sph_ctx *ctx, sph_particles *p, const void *h_seed, sph_density_stats *stats, void *stream)
{
    SPH_TRY(check_particles(ctx, p, true));
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    sph_density_stats local{};
    SPH_CUDA(cudaEventRecord(ctx->ev[0], s));
    int st = density_run(ctx, p, h_seed, &local, s);
    SPH_CUDA(cudaEventRecord(ctx->ev[1], s));
    SPH_CUDA(cudaEventSynchronize(ctx->ev[1]));
    SPH_TRY(elapsed(ctx, ctx->ev[0], ctx->ev[1], &local.ms));
    if (stats) *stats = local;
    return st;
}

int sph_forces(sph_ctx *ctx, sph_particles *p, sph_force_stats *stats, void *stream)
{
    SPH_TRY(check_particles(ctx, p, true));
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    sph_force_stats local{};
    SPH_CUDA(cudaEventRecord(ctx->ev[0], s));
    SPH_TRY(forces_run(ctx, p, p->vx, p->vy, p->vz, p->u, &local, false, s));
    SPH_CUDA(cudaEventRecord(ctx->ev[1], s));
    SPH_CUDA(cudaEventSynchronize(ctx->ev[1]));
    SPH_TRY(elapsed(ctx, ctx->ev[0], ctx->ev[1], &local.ms));
    if (stats) *stats = local;
    return SPH_OK;
}

int sph_step(sph_ctx *ctx, sph_particles *p, double dt, int use_hnet, sph_step_stats *stats, void *stream)
{
    SPH_TRY(check_particles(ctx, p, false));
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    if (!(dt > 0.0)) dt = ctx->dt_cfl;
    if (!(dt > 0.0) || !std::isfinite(dt))
        return sph_fail(ctx, SPH_ERR_STATE, "sph_step: dt <= 0 and no CFL step known yet (run sph_step with dt > 0 first)");
    sph_step_stats local{};
    local.dt = dt;
    const int64_t launches0 = ctx->launches;
    const bool seed_net = (use_hnet & SPH_HNET_SEED) != 0, train_net = (use_hnet & SPH_HNET_TRAIN) != 0;
    cudaEvent_t *ev = ctx->ev;
    SPH_CUDA(cudaEventRecord(ev[0], s));
    SPH_TRY(kick_drift(ctx, p, dt, s));
    // The h seed reads only particle fields, so it runs on the side stream as
    // soon as the fields exist in key order (in a full sort, on the scratch
    // copy before it is copied back), beside the copy back and the leaf
    // build (chains of small kernels that leave most of the GPU idle); the
    // density iteration waits for it.
    struct SeedHook : OrderHook {
        sph_ctx *ctx;
        double dt;
        bool train;
        int operator()(cudaStream_t ms, const sph_particles *view) override
        {
            SPH_CUDA(cudaEventRecord(ctx->ev_order, ms));
            SPH_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_order, 0));
            SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->hnet_fallback, 0, sizeof(int32_t), ctx->side));
            SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->hnet_err, 0, sizeof(uint32_t), ctx->side));
            SPH_TRY(copy_field(ctx, ctx->hold, view->h, view->n, ctx->side));   // the pre-iteration h
            SPH_TRY(hnet_seed_from_fields(ctx, view, dt, train, ctx->hseed, ctx->side));
            SPH_CUDA(cudaEventRecord(ctx->ev_seed, ctx->side));
            return SPH_OK;
        }
        int join(cudaStream_t ms) override
        {
            SPH_CUDA(cudaStreamWaitEvent(ms, ctx->ev_seed, 0));
            return SPH_OK;
        }
    } hook;
    hook.ctx = ctx;
    hook.dt = dt;
    hook.train = train_net;
    // omega, P, c and vsig are rewritten for every particle by this step's
    // density iteration and force pass before anything reads them
    const int built = tree_build(ctx, p, s, seed_net ? &hook : nullptr, false);
    // the main stream joins the seed before anything else (also on an error,
    // so that no side-stream work outlives the call)
    if (seed_net) SPH_CUDA(cudaStreamWaitEvent(s, ctx->ev_seed, 0));
    SPH_TRY(built);
    local.tree_moved = (int32_t)std::min<int64_t>(ctx->ns_moved, INT32_MAX);
    SPH_CUDA(cudaEventRecord(ev[1], s));
    const void *seed = nullptr;
    if (!seed_net) SPH_TRY(copy_field(ctx, ctx->hold, p->h, p->n, s));   // else on the side stream
    if (seed_net) {
        seed = ctx->hseed;
        local.hnet_used = 1;
    } else if (train_net) {
        SPH_TRY(hnet_sample_features(ctx, p, dt, s));
    }
    SPH_CUDA(cudaEventRecord(ev[2], s));
    int st = density_run(ctx, p, seed, &local.density, s, false);
    if (seed_net) local.hnet_fallback = ctx->hcnt->hnet_fallback;
    if (seed_net && ctx->hcnt->hnet_err)
        return sph_fail(ctx, SPH_ERR_CUDA, "sph_step: an h-predictor tensor-core MMA did not complete within 1 s");
    if (st == SPH_ERR_NOT_CONVERGED && seed_net) {
        // the plain iteration is the fallback: restart from the previous h
        local.hnet_fallback += (int32_t)local.density.n_unconverged;
        sph_density_stats again{};
        st = density_run(ctx, p, ctx->hold, &again, s, false);
        local.density.sweeps += again.sweeps;
        local.density.list_builds += again.list_builds;
        local.density.interactions += again.interactions;
        local.density.evaluations += again.evaluations;
        local.density.n_unconverged = again.n_unconverged;
        local.density.n_hbounds = again.n_hbounds;
        local.density.kernel_ms += again.kernel_ms;
        local.density.lists_ms += again.lists_ms;
        local.density.launches += again.launches;
    }
    if (st != SPH_OK && st != SPH_ERR_H_BOUNDS) return st;
    const int dens_status = st;
    if (train_net) {
        // the training round reads h and the pre-iteration h (hold), which
        // nothing writes before the next call joins it
        SPH_CUDA(cudaEventRecord(ctx->ev_dens, s));
        SPH_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_dens, 0));
        SPH_TRY(hnet_online(ctx, p, ctx->side));
        SPH_CUDA(cudaEventRecord(ctx->ev_train, ctx->side));
        ctx->side_pending = true;
    }
    SPH_CUDA(cudaEventRecord(ev[3], s));
    SPH_TRY(copy_field(ctx, p->hprev, ctx->hold, p->n, s));
    SPH_TRY(predict(ctx, p, dt, s));
    SPH_TRY(forces_run(ctx, p, ctx->vpx, ctx->vpy, ctx->vpz, ctx->upred, nullptr, true, s));
    SPH_TRY(kick(ctx, p, dt, s));
    SPH_TRY(totals_run(ctx, p, ctx->vpx, ctx->vpy, ctx->vpz, p->u, s));
    SPH_CUDA(cudaEventRecord(ev[4], s));
    SPH_TRY(sync_counters(ctx, s));
    SPH_TRY(forces_collect(ctx, &local.forces));
    const DevCounters &h = *ctx->hcnt;
    for (int k = 0; k < 3; ++k) { local.momentum[k] = h.totals[k]; local.force[k] = h.totals[3 + k]; }
    local.energy = h.totals[6];
    local.power = h.totals[7];
    local.dt_next = ctx->prm.cfl * h.min_dt;
    if (train_net) local.hnet_loss = h.loss;
    local.launches = ctx->launches - launches0;
    ctx->dt_cfl = local.dt_next;
    double t_tree = 0, t_hnet = 0, t_dens = 0, t_tot = 0;
    SPH_TRY(elapsed(ctx, ev[0], ev[1], &t_tree));
    SPH_TRY(elapsed(ctx, ev[1], ev[2], &t_hnet));
    SPH_TRY(elapsed(ctx, ev[2], ev[3], &t_dens));
    SPH_TRY(elapsed(ctx, ev[0], ev[4], &t_tot));
    local.ms_tree = t_tree;
    local.ms_hnet = t_hnet;
    local.density.ms = t_dens;
    local.forces.ms = t_tot - t_tree - t_hnet - t_dens;
    local.ms_total = t_tot;
    if (stats) *stats = local;
    return dens_status;
}

int sph_totals(sph_ctx *ctx, const sph_particles *p, double out[8], void *stream)
{
    SPH_TRY(check_particles(ctx, p, false));
    if (!out) return sph_fail(ctx, SPH_ERR_ARG, "out is NULL");
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    SPH_TRY(totals_run(ctx, p, nullptr, nullptr, nullptr, p->u, s));
    SPH_TRY(sync_counters(ctx, s));
    for (int k = 0; k < 8; ++k) out[k] = ctx->hcnt->totals[k];
    return SPH_OK;
}

int sph_morton_keys(sph_ctx *ctx, const sph_particles *p, uint64_t *keys, double dom[4], void *stream)
{
    SPH_TRY(join_side(ctx, S(stream)));
    SPH_TRY(check_particles(ctx, p, false));
    if (!keys) return sph_fail(ctx, SPH_ERR_ARG, "keys is NULL");
    SPH_TRY(tree_keys(ctx, p, keys, S(stream)));
    if (dom)
        for (int d = 0; d < 4; ++d) dom[d] = ctx->dom[d];
    return SPH_OK;
}

int sph_sort_keys(sph_ctx *ctx, int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    SPH_TRY(join_side(ctx, S(stream)));
    if (n < 1 || n > ctx->n_max) return sph_fail(ctx, SPH_ERR_ARG, "n must be in [1, n_max]");
    if (!keys || !perm) return sph_fail(ctx, SPH_ERR_ARG, "keys and perm must be device arrays");
    ctx->tree_valid = false;
    return tree_sort(ctx, n, keys, ids, perm, S(stream));
}

int sph_tree_info(sph_ctx *ctx, int64_t *n_leaves, int64_t *n_groups)
{
    if (!ctx) return SPH_ERR_ARG;
    if (!ctx->tree_valid) return sph_fail(ctx, SPH_ERR_STATE, "no tree: call sph_build_tree first");
    if (n_leaves) *n_leaves = ctx->n_leaves;
    if (n_groups) *n_groups = ctx->n_groups;
    return SPH_OK;
}

int sph_list_info(sph_ctx *ctx, int64_t *slots_reserved, int64_t *slots_used, int64_t *union_used,
                  int32_t *exact_sizing, int32_t *union_max, int32_t *predicted, int32_t *pred_failures)
{
    if (!ctx) return SPH_ERR_ARG;
    if (union_max) *union_max = ctx->hcnt->union_max;
    if (predicted) *predicted = ctx->lists_pred ? 1 : 0;
    if (pred_failures) *pred_failures = ctx->lists_pred_fail;
    if (slots_reserved) *slots_reserved = (int64_t)ctx->hcnt->list_total;
    if (slots_used) *slots_used = (int64_t)ctx->hcnt->list_used;
    if (union_used) *union_used = (int64_t)ctx->hcnt->union_used;
    if (exact_sizing) *exact_sizing = ctx->lists_exact ? 1 : 0;
    return SPH_OK;
}

int sph_export_leaves(sph_ctx *ctx, int32_t *leaf_begin, int32_t *level, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    if (!ctx->tree_valid) return sph_fail(ctx, SPH_ERR_STATE, "no tree: call sph_build_tree first");
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    if (leaf_begin)
        SPH_CUDA(cudaMemcpyAsync(leaf_begin, ctx->leaf_begin, sizeof(int32_t) * (size_t)(ctx->n_leaves + 1),
                                 cudaMemcpyDeviceToDevice, s));
    if (level)
        SPH_CUDA(cudaMemcpyAsync(level, ctx->leaf_level, sizeof(int32_t) * (size_t)ctx->n_leaves,
                                 cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    return SPH_OK;
}

int sph_neighbors(sph_ctx *ctx, const sph_particles *p, int kind, int64_t *counts, const int64_t *offsets,
                  uint32_t *idx, void *stream)
{
    SPH_TRY(join_side(ctx, S(stream)));
    SPH_TRY(check_particles(ctx, p, true));
    if (kind != 0 && kind != 1) return sph_fail(ctx, SPH_ERR_ARG, "kind must be 0 (density) or 1 (force)");
    if (!counts || (offsets && !idx)) return sph_fail(ctx, SPH_ERR_ARG, "counts (and idx with offsets) required");
    return neighbors_export(ctx, p, kind, counts, offsets, idx, S(stream));
}

int sph_hnet_set_weights(sph_ctx *ctx, const float *params_host, int64_t count)
{
    if (!ctx) return SPH_ERR_ARG;
    SPH_TRY(join_side(ctx, nullptr, true));
    if (!params_host || count != SPH_HNET_NPARAM) return sph_fail(ctx, SPH_ERR_ARG, "expected SPH_HNET_NPARAM floats");
    for (int64_t k = 0; k < count; ++k)
        if (!std::isfinite(params_host[k])) return sph_fail(ctx, SPH_ERR_NONFINITE, "non-finite network weight");
    SPH_CUDA(cudaMemcpy(ctx->hn_master, params_host, sizeof(float) * SPH_HNET_NPARAM, cudaMemcpyHostToDevice));
    SPH_CUDA(cudaMemset(ctx->hn_m, 0, sizeof(float) * SPH_HNET_NPARAM));
    SPH_CUDA(cudaMemset(ctx->hn_v, 0, sizeof(float) * SPH_HNET_NPARAM));
    ctx->hn_step = 0;
    SPH_TRY(hnet_refresh_bf16(ctx, 0));
    SPH_CUDA(cudaDeviceSynchronize());
    return SPH_OK;
}

int sph_hnet_get_weights(sph_ctx *ctx, float *params_host, int64_t count)
{
    if (!ctx) return SPH_ERR_ARG;
    SPH_TRY(join_side(ctx, nullptr, true));
    if (!params_host || count != SPH_HNET_NPARAM) return sph_fail(ctx, SPH_ERR_ARG, "expected SPH_HNET_NPARAM floats");
    SPH_CUDA(cudaDeviceSynchronize());
    SPH_CUDA(cudaMemcpy(params_host, ctx->hn_master, sizeof(float) * SPH_HNET_NPARAM, cudaMemcpyDeviceToHost));
    return SPH_OK;
}

int sph_hnet_features(sph_ctx *ctx, const sph_particles *p, double dt, float *feats, void *stream)
{
    SPH_TRY(check_particles(ctx, p, false));
    if (!feats) return sph_fail(ctx, SPH_ERR_ARG, "feats is NULL");
    SPH_TRY(join_side(ctx, S(stream)));
    return hnet_features(ctx, p, dt, feats, S(stream));
}

int sph_test_hooks(sph_ctx *ctx, int flags)
{
    if (!ctx) return SPH_ERR_ARG;
    if (flags & ~SPH_TEST_SKIP_MMA) return sph_fail(ctx, SPH_ERR_ARG, "sph_test_hooks: unknown flag");
    ctx->test_flags = flags;
    return SPH_OK;
}

int sph_hnet_infer(sph_ctx *ctx, const float *feats, int64_t nb, float *y, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    if (!feats || !y || nb < 1) return sph_fail(ctx, SPH_ERR_ARG, "feats, y and nb >= 1 required");
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->hnet_err, 0, sizeof(uint32_t), s));
    SPH_TRY(hnet_infer(ctx, feats, nb, y, s));
    SPH_TRY(sync_counters(ctx, s));
    if (ctx->hcnt->hnet_err)
        return sph_fail(ctx, SPH_ERR_CUDA, "sph_hnet_infer: a tensor-core MMA did not complete within 1 s");
    return SPH_OK;
}

int sph_hnet_seed(sph_ctx *ctx, const sph_particles *p, double dt, void *h_seed, int64_t *fallbacks, void *stream)
{
    SPH_TRY(check_particles(ctx, p, false));
    if (!h_seed) return sph_fail(ctx, SPH_ERR_ARG, "h_seed is NULL");
    if ((reinterpret_cast<uintptr_t>(h_seed) & 15u) != 0) return sph_fail(ctx, SPH_ERR_ARG, "h_seed must be 16-byte aligned");
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->hnet_fallback, 0, sizeof(int32_t), s));
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->hnet_err, 0, sizeof(uint32_t), s));
    SPH_TRY(hnet_seed_from_fields(ctx, p, dt, false, h_seed, s));
    SPH_TRY(sync_counters(ctx, s));
    if (ctx->hcnt->hnet_err)
        return sph_fail(ctx, SPH_ERR_CUDA, "sph_hnet_seed: a tensor-core MMA did not complete within 1 s");
    if (fallbacks) *fallbacks = ctx->hcnt->hnet_fallback;
    return SPH_OK;
}

int sph_hnet_grad(sph_ctx *ctx, const float *feats, const float *target, int64_t nb, float *grad_host,
                  float *loss_host, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    if (!feats || !target || nb < 1) return sph_fail(ctx, SPH_ERR_ARG, "feats, target and nb >= 1 required");
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    SPH_TRY(hnet_grad(ctx, feats, target, nb, s));
    SPH_TRY(sync_counters(ctx, s));
    if (grad_host)
        SPH_CUDA(cudaMemcpy(grad_host, ctx->hn_grad, sizeof(float) * SPH_HNET_NPARAM, cudaMemcpyDeviceToHost));
    if (loss_host) *loss_host = ctx->hcnt->loss;
    return SPH_OK;
}

int sph_hnet_train_step(sph_ctx *ctx, const float *feats, const float *target, int64_t nb, float lr,
                        float *loss_host, void *stream)
{
    if (!ctx) return SPH_ERR_ARG;
    if (!feats || !target || nb < 1 || !(lr > 0.f)) return sph_fail(ctx, SPH_ERR_ARG, "feats, target, nb >= 1, lr > 0 required");
    cudaStream_t s = S(stream);
    SPH_TRY(join_side(ctx, s));
    SPH_TRY(hnet_grad(ctx, feats, target, nb, s));
    SPH_TRY(hnet_adam(ctx, lr, s));
    if (loss_host) {
        SPH_TRY(sync_counters(ctx, s));
        *loss_host = ctx->hcnt->loss;
    }
    return SPH_OK;
}

}  // extern "C"
