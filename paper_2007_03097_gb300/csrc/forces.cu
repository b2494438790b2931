// Momentum and internal-energy equations (Eqs. 5-6, g = 0) with the Monaghan
// (1992) artificial viscosity the paper cites as its standard prescription:
//   dv_a/dt = -sum_b m_b (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) grad_a W(r_ab, h_ab)
//   du_a/dt =  sum_b m_b (P_a/rho_a^2 + Pi_ab/2) v_ab . grad_a W(r_ab, h_ab)
//   h_ab = (h_a + h_b)/2, pairs with r_ab < h_a + h_b (W_ab vanishes beyond),
//   mu_ab = h_ab v_ab.r_ab / (r_ab^2 + eps h_ab^2),
//   Pi_ab = (-alpha cbar mu + beta mu^2) / rhobar if v_ab.r_ab < 0 else 0.
// Also: div v_a = -(1/rho_a) sum_{r_ab < 2 h_a} m_b v_ab . grad_a W(r_ab, h_a)
// and the signal speed vsig_a = max_b (c_a + c_b - 3 min(0, v_ab . rhat_ab)).
// One warp per target group, one lane per target, each lane walking its own
// force list (b with r_ab <= max(2 h_a, h_a + h_b)) and testing it exactly.
#include "sph_internal.cuh"

namespace {

constexpr int FW = 4;

struct ForceArgs {
    const int32_t *group_begin;
    const int64_t *goff;
    const int32_t *gwidth;
    const uint32_t *nbl;
    int64_t cap;
    int n_groups;
    const double *x, *y, *z;
    const float *xh, *xl, *yh, *yl, *zh, *zl;
    const void *vx, *vy, *vz, *m, *h, *rho, *pr2, *c;
    void *ax, *ay, *az, *dudt, *divv, *vsig;
    int kernel, periodic;
    double L, alpha, beta, eps;
    DevCounters *cnt;
};

template <typename T, bool FP64POS>
__global__ void __launch_bounds__(FW * 32) k_forces(ForceArgs a)
{
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * FW + (threadIdx.x >> 5);
    if (g >= a.n_groups) return;
    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const bool tgt = lane < ge - gb;
    const int i = gb + (tgt ? lane : 0);
    const T *vx = (const T *)a.vx, *vy = (const T *)a.vy, *vz = (const T *)a.vz;
    const T *m = (const T *)a.m, *h = (const T *)a.h, *rho = (const T *)a.rho;
    const T *pr2 = (const T *)a.pr2, *c = (const T *)a.c;
    const T vxa = vx[i], vya = vy[i], vza = vz[i];
    const T ha = h[i], rhoa = rho[i], pra = pr2[i], ca = c[i];
    const T hainv = T(1) / ha;
    const T sig = kern_sigma<T>(a.kernel);
    const T alpha = (T)a.alpha, beta = (T)a.beta, eps = (T)a.eps;
    const int64_t off = a.goff[g];
    int width = tgt ? a.gwidth[g] : 0;
    if (off + 32 * (int64_t)width > a.cap) width = 0;    // never read past the lists

    T accx = 0, accy = 0, accz = 0, du = 0, dv = 0, vs = ca;
    int nint = 0;
    double xa = 0, ya = 0, za = 0;
    float xah = 0, xal = 0, yah = 0, yal = 0, zah = 0, zal = 0;
    if (FP64POS) { xa = a.x[i]; ya = a.y[i]; za = a.z[i]; }
    else { xah = a.xh[i]; xal = a.xl[i]; yah = a.yh[i]; yal = a.yl[i]; zah = a.zh[i]; zal = a.zl[i]; }
    const double thr_d = __dmul_rn(__dmul_rn(4.0, (double)ha), (double)ha);
    const float thr_f = __fmul_rn(__fmul_rn(4.f, (float)ha), (float)ha);

    for (int k = 0; k < width; ++k) {
        const uint32_t b = a.nbl[off + (int64_t)k * 32 + lane];
        if (b == SPH_SENTINEL) continue;
        const T hb = h[b];
        T dx, dy, dz, r2;
        bool in_f, in_d;
        if (FP64POS) {
            const double half = 0.5 * a.L;
            double ddx = sep_d(xa, a.x[b], a.periodic, a.L, half);
            double ddy = sep_d(ya, a.y[b], a.periodic, a.L, half);
            double ddz = sep_d(za, a.z[b], a.periodic, a.L, half);
            double rr = r2_d(ddx, ddy, ddz);
            double hs = __dadd_rn((double)ha, (double)hb);
            in_f = rr < __dmul_rn(hs, hs);
            in_d = rr < thr_d;
            dx = (T)ddx; dy = (T)ddy; dz = (T)ddz; r2 = (T)rr;
        } else {
            const float Lf = (float)a.L, half = 0.5f * Lf;
            float fdx = sep_f(xah, xal, a.xh[b], a.xl[b], a.periodic, Lf, half);
            float fdy = sep_f(yah, yal, a.yh[b], a.yl[b], a.periodic, Lf, half);
            float fdz = sep_f(zah, zal, a.zh[b], a.zl[b], a.periodic, Lf, half);
            float rr = __fadd_rn(__fadd_rn(__fmul_rn(fdx, fdx), __fmul_rn(fdy, fdy)), __fmul_rn(fdz, fdz));
            float hs = __fadd_rn((float)ha, (float)hb);
            in_f = rr < __fmul_rn(hs, hs);
            in_d = rr < thr_f;
            dx = (T)fdx; dy = (T)fdy; dz = (T)fdz; r2 = (T)rr;
        }
        if (!in_f && !in_d) continue;
        const T r = sqrt(r2);
        const T rinv = T(1) / r;
        const T vabx = vxa - vx[b], vaby = vya - vy[b], vabz = vza - vz[b];
        const T vdotr = (vabx * dx + vaby * dy) + vabz * dz;
        const T mb = m[b];
        if (in_d) {
            T w, dwq;
            kern_wdw<T>(a.kernel, r * hainv, w, dwq);
            const T h2 = hainv * hainv;
            dv += mb * (sig * h2 * h2 * dwq) * rinv * vdotr;
        }
        if (in_f) {
            const T hab = T(0.5) * (ha + hb);
            const T habinv = T(1) / hab;
            T w, dwq;
            kern_wdw<T>(a.kernel, r * habinv, w, dwq);
            const T h2 = habinv * habinv;
            const T gr = sig * h2 * h2 * dwq * rinv;          // grad_a W = gr * r_ab
            T Pi = T(0);
            if (vdotr < T(0)) {
                const T mu = hab * vdotr / (r2 + eps * hab * hab);
                Pi = (-alpha * T(0.5) * (ca + c[b]) * mu + beta * mu * mu) / (T(0.5) * (rhoa + rho[b]));
            }
            const T coef = mb * (pra + pr2[b] + Pi) * gr;
            accx -= coef * dx;
            accy -= coef * dy;
            accz -= coef * dz;
            du += mb * (pra + T(0.5) * Pi) * gr * vdotr;
            const T vr = vdotr * rinv;
            const T sgn = ca + c[b] - T(3) * (vr < T(0) ? vr : T(0));
            vs = sgn > vs ? sgn : vs;
            ++nint;
        }
    }
    if (tgt) {
        ((T *)a.ax)[i] = accx;
        ((T *)a.ay)[i] = accy;
        ((T *)a.az)[i] = accz;
        ((T *)a.dudt)[i] = du;
        ((T *)a.divv)[i] = -dv / rhoa;
        ((T *)a.vsig)[i] = vs;
    }
    for (int o = 16; o > 0; o >>= 1) nint += __shfl_xor_sync(0xffffffffu, nint, o);
    if (lane == 0) atomicAdd(&a.cnt->interactions, (unsigned long long)nint);
}

template <typename T>
__global__ void k_pr2(const T *__restrict__ P, const T *__restrict__ rho, int64_t n, T *__restrict__ pr2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { const T r = rho[i]; pr2[i] = P[i] / (r * r); }
}

__global__ void k_reset_inter(DevCounters *c)
{
    c->interactions = 0;
    c->err = 0;
}

template <typename T>
int run_impl(sph_ctx *ctx, sph_particles *p, const void *vx, const void *vy, const void *vz,
             sph_force_stats *st, cudaStream_t s)
{
    const int64_t launches0 = ctx->launches;
    k_reset_inter<<<1, 1, 0, s>>>(ctx->dcnt);
    k_pr2<T><<<grid_for(p->n, 256), 256, 0, s>>>((const T *)p->P, (const T *)p->rho, p->n, (T *)ctx->pr2);
    SPH_CHECK_LAUNCH();
    SPH_TRY(tree_refit_h(ctx, p, s));
    SPH_TRY(lists_build(ctx, p, 1, s));
    ForceArgs a{};
    a.group_begin = ctx->group_begin;
    a.goff = ctx->group_off;
    a.gwidth = ctx->group_width;
    a.nbl = ctx->nbl;
    a.cap = ctx->nbl_cap;
    a.n_groups = (int)ctx->n_groups;
    a.x = p->x; a.y = p->y; a.z = p->z;
    a.xh = ctx->xh; a.xl = ctx->xl; a.yh = ctx->yh; a.yl = ctx->yl; a.zh = ctx->zh; a.zl = ctx->zl;
    a.vx = vx; a.vy = vy; a.vz = vz; a.m = p->m; a.h = p->h; a.rho = p->rho; a.pr2 = ctx->pr2; a.c = p->c;
    a.ax = p->ax; a.ay = p->ay; a.az = p->az; a.dudt = p->dudt; a.divv = p->divv; a.vsig = p->vsig;
    a.kernel = ctx->prm.kernel;
    a.periodic = ctx->prm.periodic;
    a.L = ctx->dom[3];
    a.alpha = ctx->prm.alpha; a.beta = ctx->prm.beta; a.eps = ctx->prm.eps_visc;
    a.cnt = ctx->dcnt;
    SPH_CUDA(cudaEventRecord(ctx->kev[2], s));
    if (ctx->fp64) k_forces<T, true><<<grid_for(ctx->n_groups, FW), FW * 32, 0, s>>>(a);
    else k_forces<T, false><<<grid_for(ctx->n_groups, FW), FW * 32, 0, s>>>(a);
    SPH_CHECK_LAUNCH();
    SPH_CUDA(cudaEventRecord(ctx->kev[3], s));
    if (st) {
        SPH_TRY(sync_counters(ctx, s));
        float f = 0.f;
        SPH_CUDA(cudaEventElapsedTime(&f, ctx->kev[2], ctx->kev[3]));
        st->kernel_ms = f;
        st->launches = ctx->launches - launches0;
        st->interactions = (int64_t)ctx->hcnt->interactions;
        st->list_entries = (int64_t)ctx->hcnt->list_total;
        if (ctx->hcnt->err & (ERRB_LIST_CAPACITY | ERRB_STACK))
            return sph_fail(ctx, SPH_ERR_CAPACITY, "sph_forces: neighbour-list capacity exceeded");
    }
    return SPH_OK;
}

}  // namespace

int forces_run(sph_ctx *ctx, sph_particles *p, const void *vx, const void *vy, const void *vz,
               sph_force_stats *st, cudaStream_t s)
{
    return ctx->fp64 ? run_impl<double>(ctx, p, vx, vy, vz, st, s) : run_impl<float>(ctx, p, vx, vy, vz, st, s);
}
