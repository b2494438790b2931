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
// neighbour list and testing every entry exactly.
// SPH_MIXED: FP32 throughout (reciprocal square root for 1/r).  SPH_FP64: pair terms in double-float on the
// FP32 pipes, membership decided in FP32 outside a 1e-5 relative band around
// each threshold and by the exact FP64 r^2 inside it.
#include "dfloat.cuh"
#include "sph_internal.cuh"

namespace {

constexpr int FW = 4;

struct ForceArgs {
    const int32_t *group_begin;
    const int64_t *goff;
    const int32_t *gwidth;
    const uint16_t *nbl;
    int64_t cap;
    const uint32_t *uni;           // group source unions
    const int64_t *uoff;
    const int32_t *group_img;      // 1: the group's sources include periodic images
    int n_groups;
    const double *x, *y, *z;
    const float4 *srcA, *srcB, *srcC, *srcD, *srcE, *srcF;
    const void *vx, *vy, *vz, *m, *h, *rho, *c;
    void *ax, *ay, *az, *dudt, *divv, *vsig;
    int kernel, periodic;          // kernel: the kernel shape (kern_shape)
    int dim;                       // D = 1 or 3: grad W = sigma / h^(D+1) w'(q) r_ab / r
    int thermo;                    // 1: dudt receives de/dt of the thermokinetic formulation
    double L, alpha, beta, eps;
    df Ld, sig_d, alpha_d, beta_d, eps_d;   // the same constants as double-floats
    DevCounters *cnt;
};

// SPH_MIXED force pass in FP32: sources packed as A {xh, xl, yh, yl},
// B {zh, zl, m, -}, C {vx, vy, vz, h}, D {rho, P/rho^2, c, -}.
template <int KS>
__global__ void __launch_bounds__(FW * 32) k_forces_f32(ForceArgs a)
{
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * FW + (threadIdx.x >> 5);
    if (g >= a.n_groups) return;
    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const bool tgt = lane < ge - gb;
    const int i = gb + (tgt ? lane : 0);
    const float4 A = a.srcA[i], Bz = a.srcB[i], C = a.srcC[i], D = a.srcD[i];
    const float ha = C.w, rhoa = D.x, pra = D.y, ca = D.z;
    const float hainv = 1.f / ha;
    const float sig = kern_sigma<float>(a.kernel);
    const float sig_hg = sig * inv_pow_dim(hainv, a.dim) * hainv;     // sigma / h_a^(D+1)
    const float alpha = (float)a.alpha, beta = (float)a.beta, eps = (float)a.eps;
    const int64_t off = a.goff[g];
    const uint32_t *U = a.uni + a.uoff[g];
    const int img = a.periodic && a.group_img[g];   // else every source's direct image is the nearest
    int width = tgt ? a.gwidth[g] : 0;
    if (off + 32 * (int64_t)width > a.cap) width = 0;    // never read past the lists
    const float Lf = (float)a.L, half = 0.5f * Lf;
    const float thr_d = __fmul_rn(__fmul_rn(4.f, ha), ha);

    float accx = 0.f, accy = 0.f, accz = 0.f, du = 0.f, dv = 0.f, vs = ca;
    int nint = 0;
    // the list entry of slot k + 2 and the union index of slot k + 1 are in
    // flight while slot k is processed
    SlotStream st(a.nbl, off, width, lane);
    auto index = [&](uint32_t e) -> uint32_t { return e == SPH_LOCAL_NONE ? SPH_SENTINEL : __ldg(U + e); };
    const uint32_t e0 = st.next();
    uint32_t e2 = st.next();
    uint32_t b1 = index(e0);
    for (int k = 0; k < width; ++k) {
        const uint32_t b = b1;
        b1 = index(e2);
        e2 = st.next();
        if (b == SPH_SENTINEL) continue;
        const float4 P = a.srcA[b], Q = a.srcB[b], Cb = a.srcC[b];
        const float dx = sep_f(A.x, A.y, P.x, P.y, img, Lf, half);
        const float dy = sep_f(A.z, A.w, P.z, P.w, img, Lf, half);
        const float dz = sep_f(Bz.x, Bz.y, Q.x, Q.y, img, Lf, half);
        const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        const float hb = Cb.w;
        const float hs = __fadd_rn(ha, hb);
        const bool in_f = r2 < __fmul_rn(hs, hs);
        const bool in_d = r2 < thr_d;
        if (!in_f && !in_d) continue;
        const float4 Db = a.srcD[b];
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float vabx = C.x - Cb.x, vaby = C.y - Cb.y, vabz = C.z - Cb.z;
        const float vdotr = (vabx * dx + vaby * dy) + vabz * dz;
        const float mb = Q.z;
        if (in_d) {
            float w, dwq;
            kern_wdw<float>(KS, r * hainv, w, dwq);      // the kernel form fixed at compile time
            dv += mb * (sig_hg * dwq) * rinv * vdotr;
        }
        if (in_f) {
            // approximate reciprocals (within 2 ulp): the FP32 pass is held
            // to relative tolerances far above them
            const float hab = 0.5f * hs;
            const float habinv = __fdividef(1.f, hab);
            float w, dwq;
            kern_wdw<float>(KS, r * habinv, w, dwq);
            const float h2 = habinv * habinv;
            const float gr = sig * (a.dim == 1 ? h2 : h2 * h2) * dwq * rinv;   // grad_a W = gr * r_ab
            float Pi = 0.f;
            if (vdotr < 0.f) {
                const float mu = __fdividef(hab * vdotr, r2 + eps * hab * hab);
                Pi = __fdividef(-alpha * 0.5f * (ca + Db.z) * mu + beta * mu * mu, 0.5f * (rhoa + Db.x));
            }
            const float coef = mb * (pra + Db.y + Pi) * gr;
            accx -= coef * dx;
            accy -= coef * dy;
            accz -= coef * dz;
            if (a.thermo) {
                // Eq. thermo: -m_b (P_a/rho_a^2 v_b + P_b/rho_b^2 v_a + (v_a + v_b) Pi/2) . grad_a W
                const float vb_r = (Cb.x * dx + Cb.y * dy) + Cb.z * dz;
                const float va_r = (C.x * dx + C.y * dy) + C.z * dz;
                du -= mb * ((pra * vb_r + Db.y * va_r) + Pi * 0.5f * (va_r + vb_r)) * gr;
            } else {
                du += mb * (pra + 0.5f * Pi) * gr * vdotr;
            }
            const float vr = vdotr * rinv;
            const float sgn = ca + Db.z - 3.f * (vr < 0.f ? vr : 0.f);
            vs = sgn > vs ? sgn : vs;
            ++nint;
        }
    }
    if (tgt) {
        ((float *)a.ax)[i] = accx;
        ((float *)a.ay)[i] = accy;
        ((float *)a.az)[i] = accz;
        ((float *)a.dudt)[i] = du;
        ((float *)a.divv)[i] = -dv / rhoa;
        ((float *)a.vsig)[i] = vs;
    }
    for (int o = 16; o > 0; o >>= 1) nint += __shfl_xor_sync(0xffffffffu, nint, o);
    if (lane == 0) atomicAdd(&a.cnt->force_interactions, (unsigned long long)nint);
}

// Equation of state and packed FP32 force-pass sources: P = (gamma-1) rho u,
// c = sqrt(gamma (gamma-1) u) to the caller's P and c, and the records
// C {vx, vy, vz, h}, D {rho, P/rho^2, c, 0}.
__global__ void k_pack_force_f32(const float *__restrict__ vx, const float *__restrict__ vy,
                                 const float *__restrict__ vz, const float *__restrict__ h,
                                 const float *__restrict__ rho, const float *__restrict__ u, float g1, float gg1,
                                 int64_t n, float *__restrict__ P, float *__restrict__ c, float4 *__restrict__ C,
                                 float4 *__restrict__ D)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float r = rho[i], ui = u[i];
    const float pi = g1 * r * ui, ci = sqrtf(gg1 * ui);
    P[i] = pi;
    c[i] = ci;
    C[i] = make_float4(vx[i], vy[i], vz[i], h[i]);
    D[i] = make_float4(r, pi / (r * r), ci, 0.f);
}

// SPH_FP64 force pass in double-float (see the file comment).
__global__ void __launch_bounds__(FW * 32, 5) k_forces_df(ForceArgs a)
{
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * FW + (threadIdx.x >> 5);
    if (g >= a.n_groups) return;
    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const bool tgt = lane < ge - gb;
    const int i = gb + (tgt ? lane : 0);
    const double *h64 = (const double *)a.h;
    const int64_t off = a.goff[g];
    const uint32_t *U = a.uni + a.uoff[g];
    const int img = a.periodic && a.group_img[g];   // else every source's direct image is the nearest
    int width = tgt ? a.gwidth[g] : 0;
    if (off + 32 * (int64_t)width > a.cap) width = 0;

    const float4 A = a.srcA[i], Bz = a.srcB[i], C = a.srcC[i], D = a.srcD[i], E = a.srcE[i], F = a.srcF[i];
    // per-particle constants in double-float (FP64 runs at 1/64 of the FP32 rate)
    const df ha = df{D.z, D.w};
    const float thr_f = df_scale(df_sqr(ha), 4.f).hi;
    const float thr_hi = thr_f * (1.f + 1e-5f), thr_lo = thr_f * (1.f - 1e-5f);
    const float Lf = (float)a.L, half = 0.5f * Lf, guard = 0.45f * Lf;
    const df Ld = a.Ld, sig = a.sig_d;
    const df hainv = df_rcp(ha);
    const df hai2 = df_sqr(hainv);
    const df sig_hai4 = df_mul(sig, a.dim == 1 ? hai2 : df_sqr(hai2));   // sigma / h_a^(D+1)
    // the pair sums leave out the per-target factors sigma (a, du/dt) and
    // sigma / h_a^(D+1) (div v), applied once at the end
    const df vxa = df{C.x, C.y}, vya = df{C.z, C.w}, vza = df{D.x, D.y};
    const df rhoa = df{E.x, E.y}, pra = df{E.z, E.w}, ca = df{F.x, F.y};
    const df alpha = a.alpha_d, beta = a.beta_d, eps = a.eps_d;

    df accx = df{0.f, 0.f}, accy = accx, accz = accx, du = accx, dv = accx, vs = ca;
    int nint = 0;
    // the list entry of slot k + 2 and the union index of slot k + 1 are in
    // flight while slot k is processed
    SlotStream st(a.nbl, off, width, lane);
    auto index = [&](uint32_t e) -> uint32_t { return e == SPH_LOCAL_NONE ? SPH_SENTINEL : __ldg(U + e); };
    const uint32_t e0 = st.next();
    uint32_t e2 = st.next();
    uint32_t b1 = index(e0);
    for (int k = 0; k < width; ++k) {
        const uint32_t b = b1;
        b1 = index(e2);
        e2 = st.next();
        if (b == SPH_SENTINEL) continue;
        const float4 P = a.srcA[b], Q = a.srcB[b], Db = a.srcD[b];
        int wx, wy, wz;
        const float dxf = sep_fw(A.x, A.y, P.x, P.y, img, Lf, half, wx);
        const float dyf = sep_fw(A.z, A.w, P.z, P.w, img, Lf, half, wy);
        const float dzf = sep_fw(Bz.x, Bz.y, Q.x, Q.y, img, Lf, half, wz);
        const float r2f = (dxf * dxf + dyf * dyf) + dzf * dzf;
        const float hsf = D.z + Db.z;
        const float thf = hsf * hsf;
        const bool out_d = r2f > thr_hi, out_f = r2f > thf * (1.f + 1e-5f);
        if (out_d && out_f) continue;
        bool in_d = r2f < thr_lo, in_f = r2f < thf * (1.f - 1e-5f);
        const bool edge = (!in_d && !out_d) || (!in_f && !out_f) ||
                          (img && fmaxf(fmaxf(fabsf(dxf), fabsf(dyf)), fabsf(dzf)) > guard);
        if (edge) {
            // knife edge: the exact FP64 decisions of the plain definition
            const double L = a.L, hl = 0.5 * a.L;
            const double dx = sep_d(a.x[i], a.x[b], a.periodic, L, hl);
            const double dy = sep_d(a.y[i], a.y[b], a.periodic, L, hl);
            const double dz = sep_d(a.z[i], a.z[b], a.periodic, L, hl);
            const double rr = r2_d(dx, dy, dz);
            const double had = h64[i];
            const double hs = __dadd_rn(had, h64[b]);
            in_f = rr < __dmul_rn(hs, hs);
            in_d = rr < __dmul_rn(__dmul_rn(4.0, had), had);
            if (!in_f && !in_d) continue;
        }
        const float4 Cb = a.srcC[b], Eb = a.srcE[b], Fb = a.srcF[b];
        const df dx = df_sep_fast(A.x, A.y, P.x, P.y, wx, Ld);
        const df dy = df_sep_fast(A.z, A.w, P.z, P.w, wy, Ld);
        const df dz = df_sep_fast(Bz.x, Bz.y, Q.x, Q.y, wz, Ld);
        const df r2 = df_norm2(dx, dy, dz);
        const df r = df_sqrt_fast(r2);
        const df rinv = df_rcp_fast(r);
        const df vabx = df_sub(vxa, df{Cb.x, Cb.y}), vaby = df_sub(vya, df{Cb.z, Cb.w}), vabz = df_sub(vza, df{Db.x, Db.y});
        const df vdotr = df_add(df_add(df_mul_u(vabx, dx), df_mul_u(vaby, dy)), df_mul_u(vabz, dz));
        const df mb = df{Q.z, Q.w};
        const df rv = df_mul_u(rinv, vdotr);                  // v_ab . r_ab / r
        if (in_d) {
            const df dwq = df_kern_dw(a.kernel, df_mul_u(r, hainv));
            df_acc(dv, df_mul_u(df_mul_u(mb, dwq), rv));
        }
        if (in_f) {
            const df hb = df{Db.z, Db.w};
            const df hab = df_scale(df_add(ha, hb), 0.5f);
            const df habinv = df_rcp_fast(hab);
            const df dwq = df_kern_dw(a.kernel, df_mul_u(r, habinv));
            const df hi2 = df_sqr_u(habinv);
            const df mgq = df_mul_u(mb, df_mul_u(a.dim == 1 ? hi2 : df_sqr_u(hi2), dwq));   // m_b w'(q) / h_ab^(D+1)
            const df gr = df_mul_u(mgq, rinv);                 // m_b grad_a W / sigma = gr r_ab
            df Pi = df{0.f, 0.f};
            if (df_lt0(vdotr)) {
                // mu = hab v.r / den, Pi = (-alpha cbar mu + beta mu^2) / rbar with
                // den = r^2 + eps hab^2, through one reciprocal X = 1 / (den rbar):
                // mu / rbar = hab v.r X, mu = (mu / rbar) rbar
                const df hv = df_mul_u(hab, vdotr);
                const df den = df_add(r2, df_mul_u(eps, df_sqr_u(hab)));
                const df rbar = df_scale(df_add(rhoa, df{Eb.x, Eb.y}), 0.5f);
                const df mu_r = df_mul_u(hv, df_rcp_fast(df_mul_u(den, rbar)));
                const df mu = df_mul_u(mu_r, rbar);
                const df cbar = df_scale(df_add(ca, df{Fb.x, Fb.y}), 0.5f);
                Pi = df_mul_u(mu_r, df_sub(df_mul_u(beta, mu), df_mul_u(alpha, cbar)));
            }
            const df coef = df_mul_u(df_add(df_add(pra, df{Eb.z, Eb.w}), Pi), gr);
            df_acc(accx, df_neg(df_mul_u(coef, dx)));
            df_acc(accy, df_neg(df_mul_u(coef, dy)));
            df_acc(accz, df_neg(df_mul_u(coef, dz)));
            if (a.thermo) {
                // Eq. thermo: -m_b (P_a/rho_a^2 v_b + P_b/rho_b^2 v_a + (v_a + v_b) Pi/2) . grad_a W
                const df vxb = df{Cb.x, Cb.y}, vyb = df{Cb.z, Cb.w}, vzb = df{Db.x, Db.y};
                const df vb_r = df_add(df_add(df_mul_u(vxb, dx), df_mul_u(vyb, dy)), df_mul_u(vzb, dz));
                const df va_r = df_add(vdotr, vb_r);
                const df t = df_add(df_add(df_mul_u(pra, vb_r), df_mul_u(df{Eb.z, Eb.w}, va_r)),
                                    df_mul_u(df_scale(Pi, 0.5f), df_add(va_r, vb_r)));
                df_acc(du, df_neg(df_mul_u(t, gr)));
            } else {
                df_acc(du, df_mul_u(df_mul_u(df_add(pra, df_scale(Pi, 0.5f)), mgq), rv));
            }
            // v_sig: an FP32 estimate (relative error below 1e-6) screens
            // out the pairs that cannot raise the maximum
            const float sgf = (ca.hi + Fb.x) - 3.f * fminf(0.f, vdotr.hi * rinv.hi);
            if (sgf >= vs.hi * (1.f - 1e-5f)) {
                const df vr = df_norm(rv);
                df sg = df_add(ca, df{Fb.x, Fb.y});
                if (df_lt0(vr)) sg = df_sub(sg, df_mul_f_u(vr, 3.f));
                if (df_gt(sg, vs)) vs = sg;
            }
            ++nint;
        }
    }
    if (tgt) {
        ((double *)a.ax)[i] = df_to_double(df_mul(sig, df_norm(accx)));
        ((double *)a.ay)[i] = df_to_double(df_mul(sig, df_norm(accy)));
        ((double *)a.az)[i] = df_to_double(df_mul(sig, df_norm(accz)));
        ((double *)a.dudt)[i] = df_to_double(df_mul(sig, df_norm(du)));
        ((double *)a.divv)[i] = -df_to_double(df_mul(sig_hai4, df_norm(dv))) / ((const double *)a.rho)[i];
        ((double *)a.vsig)[i] = df_to_double(vs);
    }
    for (int o = 16; o > 0; o >>= 1) nint += __shfl_xor_sync(0xffffffffu, nint, o);
    if (lane == 0) atomicAdd(&a.cnt->force_interactions, (unsigned long long)nint);
}

__device__ __forceinline__ float2 split2(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// Equation of state and packed force-pass sources (FP64 mode): P = (gamma-1)
// rho u in FP64 and c = sqrt(gamma (gamma-1) u) in double-float, written to the
// caller's P and c, and the records C {vx, vy}, D {vz, h}, E {rho, P/rho^2},
// F {c, 0} as two-float pairs.
__global__ void k_pack_force(const double *__restrict__ vx, const double *__restrict__ vy,
                             const double *__restrict__ vz, const double *__restrict__ h,
                             const double *__restrict__ rho, const double *__restrict__ u, double g1d, df gg1,
                             int64_t n, double *__restrict__ P, double *__restrict__ c, float4 *__restrict__ C,
                             float4 *__restrict__ D, float4 *__restrict__ E, float4 *__restrict__ F)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double rd = rho[i], ud = u[i];
    const double pd = __dmul_rn(__dmul_rn(g1d, rd), ud);      // P exactly as the FP64 definition
    const df r = df_from_double(rd), ui = df_from_double(ud), pi = df_from_double(pd);
    const df ci = df_sqrt(df_mul(gg1, ui));
    const df q = df_mul(pi, df_sqr(df_rcp(r)));
    P[i] = pd;
    c[i] = df_to_double(ci);
    const float2 a = split2(vx[i]), b = split2(vy[i]), cz = split2(vz[i]), hh = split2(h[i]);
    C[i] = make_float4(a.x, a.y, b.x, b.y);
    D[i] = make_float4(cz.x, cz.y, hh.x, hh.y);
    E[i] = make_float4(r.hi, r.lo, q.hi, q.lo);
    F[i] = make_float4(ci.hi, ci.lo, 0.f, 0.f);
}

__global__ void k_reset_inter(DevCounters *c) { c->force_interactions = 0; }

template <typename T>
int run_impl(sph_ctx *ctx, sph_particles *p, const void *vx, const void *vy, const void *vz, const void *u,
             sph_force_stats *st, bool reuse_lists, cudaStream_t s)
{
    const int64_t launches0 = ctx->launches;
    k_reset_inter<<<1, 1, 0, s>>>(ctx->dcnt);
    const double g = ctx->prm.gamma;
    if (ctx->fp64)
        k_pack_force<<<grid_for(p->n, 256), 256, 0, s>>>(
            (const double *)vx, (const double *)vy, (const double *)vz, (const double *)p->h, (const double *)p->rho,
            (const double *)u, g - 1.0, df_host(g * (g - 1.0)), p->n, (double *)p->P, (double *)p->c,
            ctx->srcC, ctx->srcD, ctx->srcE, ctx->srcF);
    else
        k_pack_force_f32<<<grid_for(p->n, 256), 256, 0, s>>>(
            (const float *)vx, (const float *)vy, (const float *)vz, (const float *)p->h, (const float *)p->rho,
            (const float *)u, (float)(g - 1.0), (float)(g * (g - 1.0)), p->n, (float *)p->P, (float *)p->c, ctx->srcC,
            ctx->srcD);
    SPH_CHECK_LAUNCH();
    if (!reuse_lists || !ctx->lists_valid) SPH_TRY(lists_build(ctx, p, s));
    ForceArgs a{};
    a.group_begin = ctx->group_begin;
    a.goff = ctx->group_off;
    a.gwidth = ctx->group_width;
    a.nbl = ctx->nbl;
    a.cap = ctx->nbl_cap;
    a.uni = ctx->uni;
    a.uoff = ctx->union_off;
    a.n_groups = (int)ctx->n_groups;
    a.x = p->x; a.y = p->y; a.z = p->z;
    a.srcA = ctx->srcA; a.srcB = ctx->srcB; a.srcC = ctx->srcC; a.srcD = ctx->srcD; a.srcE = ctx->srcE;
    a.srcF = ctx->srcF;
    a.vx = vx; a.vy = vy; a.vz = vz; a.m = p->m; a.h = p->h; a.rho = p->rho; a.c = p->c;
    a.ax = p->ax; a.ay = p->ay; a.az = p->az; a.dudt = p->dudt; a.divv = p->divv; a.vsig = p->vsig;
    a.kernel = kern_shape(ctx->prm.kernel, ctx->prm.dim);
    a.dim = ctx->prm.dim;
    a.periodic = ctx->prm.periodic;
    a.group_img = ctx->group_img;
    a.thermo = ctx->prm.energy == SPH_ENERGY_TOTAL;
    a.L = ctx->dom[3];
    a.alpha = ctx->prm.alpha; a.beta = ctx->prm.beta; a.eps = ctx->prm.eps_visc;
    const double sig = kern_sigma<double>(a.kernel);
    a.Ld = df_host(a.L); a.sig_d = df_host(sig);
    a.alpha_d = df_host(a.alpha); a.beta_d = df_host(a.beta); a.eps_d = df_host(a.eps);
    a.cnt = ctx->dcnt;
    SPH_CUDA(cudaEventRecord(ctx->ev[5], s));
    if (ctx->fp64) k_forces_df<<<grid_for(ctx->n_groups, FW), FW * 32, 0, s>>>(a);
    else {
        // one instantiation per kernel form keeps the pair loop small
        const unsigned grid = grid_for(ctx->n_groups, FW);
        switch (a.kernel) {
        case 1: k_forces_f32<1><<<grid, FW * 32, 0, s>>>(a); break;
        case 2: k_forces_f32<2><<<grid, FW * 32, 0, s>>>(a); break;
        case 4: k_forces_f32<4><<<grid, FW * 32, 0, s>>>(a); break;
        case 5: k_forces_f32<5><<<grid, FW * 32, 0, s>>>(a); break;
        default: k_forces_f32<0><<<grid, FW * 32, 0, s>>>(a); break;   // M4, either D
        }
    }
    SPH_CHECK_LAUNCH();
    SPH_CUDA(cudaEventRecord(ctx->ev[6], s));
    ctx->force_launches = ctx->launches - launches0;
    if (st) {
        SPH_TRY(sync_counters(ctx, s));
        SPH_TRY(forces_collect(ctx, st));
    }
    return SPH_OK;
}

}  // namespace

int forces_collect(sph_ctx *ctx, sph_force_stats *st)
{
    float f = 0.f;
    SPH_CUDA(cudaEventElapsedTime(&f, ctx->ev[5], ctx->ev[6]));
    st->kernel_ms = f;
    st->launches = ctx->force_launches;
    st->interactions = (int64_t)ctx->hcnt->force_interactions;
    st->list_entries = (int64_t)ctx->hcnt->list_used;
    if (ctx->hcnt->err & (ERRB_LIST_CAPACITY | ERRB_STACK))
        return sph_fail(ctx, SPH_ERR_CAPACITY, "sph_forces: neighbour-list capacity exceeded");
    return SPH_OK;
}

// reuse_lists: the lists of the h iteration that just ended still cover 2h
// of every particle (sph_step); otherwise they are rebuilt for the current h.
int forces_run(sph_ctx *ctx, sph_particles *p, const void *vx, const void *vy, const void *vz, const void *u,
               sph_force_stats *st, bool reuse_lists, cudaStream_t s)
{
    auto run = [&]() {
        return ctx->fp64 ? run_impl<double>(ctx, p, vx, vy, vz, u, st, reuse_lists, s)
                         : run_impl<float>(ctx, p, vx, vy, vz, u, st, reuse_lists, s);
    };
    const bool bounded = !ctx->lists_exact;
    const int r = run();
    // lists sized by leaf bounds overflowed nb_capacity: size them exactly
    if (r != SPH_ERR_CAPACITY || !bounded || !st) return r;
    ctx->lists_exact = true;
    ctx->lists_valid = false;
    ctx->err.clear();
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
    return run();
}
