// Momentum and internal-energy equations (Eqs. 5-6, g = 0) with the Monaghan
// (1992) artificial viscosity the paper cites as its standard prescription:
//   dv_a/dt = -sum_b m_b (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) grad_a W(r_ab, h_ab)
//   du_a/dt =  sum_b m_b (P_a/rho_a^2 + Pi_ab/2) v_ab . grad_a W(r_ab, h_ab)
//   h_ab = (h_a + h_b)/2, pairs with r_ab < h_a + h_b (W_ab vanishes beyond),
//   mu_ab = h_ab v_ab.r_ab / (r_ab^2 + eps h_ab^2),
//   Pi_ab = (-alpha cbar mu + beta mu^2) / rhobar if v_ab.r_ab < 0 else 0.
// Also: div v_a = -(1/rho_a) sum_{r_ab < 2 h_a} m_b v_ab . grad_a W(r_ab, h_a)
// and the signal speed vsig_a = max_b (c_a + c_b - 3 min(0, v_ab . rhat_ab)).
// One lane per target, walking its own neighbour list and testing every entry
// exactly.  SPH_MIXED: FP32 throughout (reciprocal square root for 1/r), one
// block per target group with the group's sources staged in shared memory
// (see k_forces_f32).  SPH_FP64: one warp per group, pair terms in double-float on the
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
    const float4 *urec;            // their position records (mixed: written by the list fill)
    const int64_t *uoff;
    const int32_t *group_img;      // 1: the group's sources include periodic images
    const int32_t *group_union;    // union size per group
    const float4 *group_lo, *group_hi;
    int n_groups;
    const double *x, *y, *z;
    const float4 *srcA, *srcB, *srcC, *srcD, *srcE, *srcF;
    const void *vx, *vy, *vz, *m, *h, *rho, *c;
    void *ax, *ay, *az, *dudt, *divv, *vsig;
    int kernel, periodic;          // kernel: the kernel shape (kern_shape)
    int uc;                        // mixed force pass: union sources staged per group
    int dim;                       // D = 1 or 3: grad W = sigma / h^(D+1) w'(q) r_ab / r
    int thermo;                    // 1: dudt receives de/dt of the thermokinetic formulation
    double L, alpha, beta, eps;    // L in the packed positions' lengths
    double Lu, ls;                 // SPH_FP64: L in the caller's units; the length scale (outputs x ls)
    double rho_sc;                 // SPH_FP64: rho_scaled = rho rho_sc
    df Ld, sig_d, alpha_d, beta_d, eps_d;   // the same constants as double-floats
    DevCounters *cnt;
};

// ---------------------------------------------------------------- SPH_MIXED
// One block of FB warps per target group.  The group's source union (the
// sources any of its targets lists, in list-walk order) is staged once into
// shared memory (as many sources as the largest union of the lists when that
// is known, at most UC_MAX, else UC), as three interleaved records per source:
//   sP {x, y, z relative to the group centre (periodic image folded in), h}
//                               copied with cp.async from the record the list
//                               fill wrote for the union entry ({x, y, z, m};
//                               h from sT replaces m)
//   sV {vx, vy, vz, m}          copied with cp.async from the packed record C
//   sT {rho/2, P/rho^2, c, h}   copied with cp.async from the packed record D
// Every warp holds the group's 32 targets (one per lane) and walks every FB-th
// quad of its lanes' lists (quads q = w, w + FB, ...), reading its sources
// from shared memory; the FB partial sums of each target are added in warp
// order at the end.  A group of at most 16 targets gives each one a segment
// of k = 32 / nextpow2(count) lanes: lane r of a segment walks the quads
// w + FB r, w + FB (r + k), ... of its target, and the segment's partial sums
// meet by shuffles before the warps' sums are added (a lane per target would
// leave most lanes idle; groups of 1-8 targets hold about 12 % of the list
// rows of a turbulence box).  Union entries past UC (a rare, very large union) are
// read from global memory with the same arithmetic.
constexpr int FB = 4;          // warps per block (one target group per block)
constexpr int UC = 512;        // union sources staged per group when the largest union is not known
constexpr int UC_MAX = 1024;   // the most sources staged (48 KB of shared memory)


// source b relative to the group centre (gcx, gcy, gcz), its nearest periodic
// image when the group's sources include images: the same arithmetic as the
// density sweep's staged sources
__device__ __forceinline__ float4 rel_pos(const float4 qa, const float4 qb, float gcx, float gcy, float gcz,
                                          bool img, float L, float invL, float h)
{
    float rx = qa.x - gcx, ry = qa.z - gcy, rz = qb.x - gcz;
    if (img) {
        rx = wrap_diff(qa.x, gcx, L, invL);
        ry = wrap_diff(qa.z, gcy, L, invL);
        rz = wrap_diff(qb.x, gcz, L, invL);
    }
    return make_float4(rx + qa.y, ry + qa.w, rz + qb.y, h);
}

// KS: the kernel form (its dimension D with it); THERMO: dudt receives de/dt
// of Eq. thermo; FAR: some union may exceed the a.uc sources staged (entries
// past them are read from global memory).  Dynamic shared memory: 3 a.uc
// float4 (a.uc >= 224, a multiple of 32).
template <int KS, bool THERMO, bool FAR>
__global__ void __launch_bounds__(FB * 32, 8) k_forces_f32(ForceArgs a)
{
    constexpr bool D1 = KS >= 3;
    constexpr bool M4 = KS == 0 || KS == 3;
    extern __shared__ float4 s_dyn[];               // source t: sP, sV, sT at 3 t, 3 t + 1, 3 t + 2
    const int UCd = a.uc;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = blockIdx.x;
    if (g >= a.n_groups) return;
    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const int nt = ge - gb;
    const int lk = nt > 16 ? 0 : 5 - (nt > 1 ? 32 - __clz(nt - 1) : 0);   // log2 of the segment length
    const int tl = lane >> lk, r = lane & ((1 << lk) - 1);                // this lane's target, its rank
    const bool tgt = tl < nt;
    const int i = gb + (tgt ? tl : 0);
    const float4 qlo = a.group_lo[g], qhi = a.group_hi[g];
    const float gcx = 0.5f * (qlo.x + qhi.x), gcy = 0.5f * (qlo.y + qhi.y), gcz = 0.5f * (qlo.z + qhi.z);
    const float Lf = (float)a.L, invL = 1.f / Lf;
    const bool img = a.periodic && a.group_img[g];   // else every source's direct image is the nearest
    const uint32_t *Ug = a.uni + a.uoff[g];
    const float4 *Rg = a.urec + a.uoff[g];
    const int U = min(a.group_union[g], UCd);

    // ---- stage the union: the position record the list fill wrote (relative
    // to the group-box centre, nearest image; m in .w until h replaces it
    // below) and the two records of the force pass, all by asynchronous copies
    for (int t = threadIdx.x; t < U; t += FB * 32) {
        const uint32_t b = __ldg(Ug + t);
        cp_async16(&s_dyn[3 * t], Rg + t);
        cp_async16(&s_dyn[3 * t + 1], a.srcC + b);
        cp_async16(&s_dyn[3 * t + 2], a.srcD + b);
    }

    // ---- the target of this lane (every warp holds the same targets)
    const float4 A = __ldg(a.srcA + i), Bz = __ldg(a.srcB + i), C = __ldg(a.srcC + i), D = __ldg(a.srcD + i);
    const float tx = (A.x - gcx) + A.y, ty = (A.z - gcy) + A.w, tz = (Bz.x - gcz) + Bz.y;
    const float ha = D.w, rhoa_h = D.x, pra = D.y, ca = D.z;   // rhoa_h = rho_a / 2
    const float hainv = 1.f / ha;
    const float thr_d = 4.f * ha * ha;
    const float beta = (float)a.beta, eps = (float)a.eps;
    const float half_alpha = 0.5f * (float)a.alpha;
    const int64_t off = a.goff[g];
    int width = tgt ? a.gwidth[g] : 0;
    if (off + 32 * (int64_t)width > a.cap) width = 0;    // never read past the lists
    const int nq = width >> 2;
    const unsigned long long *lq = reinterpret_cast<const unsigned long long *>(a.nbl + off) + tl;
    cp_async_wait_all();
    for (int t = threadIdx.x; t < U; t += FB * 32) s_dyn[3 * t].w = s_dyn[3 * t + 2].w;   // h of the source
    __syncthreads();

    // pair sums without the per-target factors sigma (a, du/dt) and
    // sigma / h_a^(D+2) (div v), applied once at the end
    float accx = 0.f, accy = 0.f, accz = 0.f, du = 0.f, dv = 0.f, vs = ca;
    int nint = 0;
    const int q0 = w + FB * r, qs = FB << lk;          // this lane's quads: q0, q0 + qs, ...
    unsigned long long nxt = q0 < nq ? __ldg(lq + 32 * (int64_t)q0) : ~0ull;
    for (int q = q0; q < nq; q += qs) {
        const unsigned long long quad = nxt;
        nxt = q + qs < nq ? __ldg(lq + 32 * (int64_t)(q + qs)) : ~0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t e = (uint32_t)(quad >> (16 * u)) & 0xFFFFu;
            float4 P, V, T;
            uint32_t b = 0;
            const bool far = e >= (uint32_t)(FAR ? U : UCd);   // SPH_LOCAL_NONE is beyond every union
            if (!far) {
                P = s_dyn[3 * e];
            } else {
                if (!FAR || e == SPH_LOCAL_NONE) continue;
                b = __ldg(Ug + e);                     // beyond the staged part of the union
                T = __ldg(a.srcD + b);
                P = rel_pos(__ldg(a.srcA + b), __ldg(a.srcB + b), gcx, gcy, gcz, img, Lf, invL, T.w);
            }
            const float dx = tx - P.x, dy = ty - P.y, dz = tz - P.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float hs = ha + P.w;
            const bool in_f = r2 < hs * hs;
            const bool in_d = r2 < thr_d;
            if (!in_f && !in_d) continue;
            if (!far) {
                V = s_dyn[3 * e + 1];
                T = s_dyn[3 * e + 2];
            } else {
                V = __ldg(a.srcC + b);
            }
            const float rinv = rsqrtf(r2);
            const float r = r2 * rinv;
            const float vabx = C.x - V.x, vaby = C.y - V.y, vabz = C.z - V.z;
            const float vdotr = fmaf(vabz, dz, fmaf(vaby, dy, vabx * dx));
            const float mb = V.w;
            if (in_d) {                                // m_b v_ab . grad_a W(r, h_a) h_a^(D+2) / sigma
                const float wq = kern_dwq<float>(KS, r * hainv, M4 ? ha * rinv : 0.f);
                dv = fmaf(mb * wq, vdotr, dv);
            }
            if (in_f) {
                // approximate reciprocals (within 2 ulp): the FP32 pass is held
                // to relative tolerances far above them
                const float hab = 0.5f * hs;
                const float habinv = __fdividef(1.f, hab);
                const float wq = kern_dwq<float>(KS, r * habinv, M4 ? hab * rinv : 0.f);
                const float h2 = habinv * habinv;
                const float gr = mb * (D1 ? h2 * habinv : h2 * h2 * habinv) * wq;   // m_b grad_a W / sigma = gr r_ab
                const float csum = ca + T.z;
                float Pi = 0.f;
                if (vdotr < 0.f) {
                    // Pi = mu (beta mu - alpha cbar) / rhobar with mu = hv / den:
                    // hv (beta hv - alpha cbar den) / (den^2 rhobar), one reciprocal
                    const float hv = hab * vdotr;
                    const float den = fmaf(eps * hab, hab, r2);
                    const float num = hv * fmaf(beta, hv, -half_alpha * csum * den);
                    Pi = __fdividef(num, den * den * (rhoa_h + T.x));
                }
                const float coef = (pra + T.y + Pi) * gr;
                accx = fmaf(-coef, dx, accx);
                accy = fmaf(-coef, dy, accy);
                accz = fmaf(-coef, dz, accz);
                if (THERMO) {
                    // Eq. thermo: -m_b (P_a/rho_a^2 v_b + P_b/rho_b^2 v_a + (v_a + v_b) Pi/2) . grad_a W
                    const float vb_r = fmaf(V.z, dz, fmaf(V.y, dy, V.x * dx));
                    const float va_r = fmaf(C.z, dz, fmaf(C.y, dy, C.x * dx));
                    du -= ((pra * vb_r + T.y * va_r) + Pi * 0.5f * (va_r + vb_r)) * gr;
                } else {
                    du = fmaf(fmaf(0.5f, Pi, pra) * gr, vdotr, du);
                }
                vs = fmaxf(vs, fmaf(-3.f, fminf(vdotr * rinv, 0.f), csum));
                ++nint;
            }
        }
    }

    // ---- the partial sums of a segment meet in its first lane
    for (int o = (1 << lk) >> 1; o > 0; o >>= 1) {
        accx += __shfl_xor_sync(0xffffffffu, accx, o);
        accy += __shfl_xor_sync(0xffffffffu, accy, o);
        accz += __shfl_xor_sync(0xffffffffu, accz, o);
        du += __shfl_xor_sync(0xffffffffu, du, o);
        dv += __shfl_xor_sync(0xffffffffu, dv, o);
        vs = fmaxf(vs, __shfl_xor_sync(0xffffffffu, vs, o));
        nint += __shfl_xor_sync(0xffffffffu, nint, o);
    }
    // ---- the FB partial sums of each target, added in warp order
    __syncthreads();                                   // the union is no longer read
    float *red = reinterpret_cast<float *>(s_dyn);     // [FB][7][32], column = target
    if (r == 0) {
        red[(w * 7 + 0) * 32 + tl] = accx;
        red[(w * 7 + 1) * 32 + tl] = accy;
        red[(w * 7 + 2) * 32 + tl] = accz;
        red[(w * 7 + 3) * 32 + tl] = du;
        red[(w * 7 + 4) * 32 + tl] = dv;
        red[(w * 7 + 5) * 32 + tl] = vs;
        red[(w * 7 + 6) * 32 + tl] = __int_as_float(nint);
    }
    __syncthreads();
    if (w != 0) return;
    // lane t of the first warp finishes target t
    const bool to = lane < nt;
    accx = red[lane]; accy = red[32 + lane]; accz = red[64 + lane];
    du = red[96 + lane]; dv = red[128 + lane]; vs = red[160 + lane];
    nint = to ? __float_as_int(red[192 + lane]) : 0;
    for (int v = 1; v < FB; ++v) {
        accx += red[(v * 7 + 0) * 32 + lane];
        accy += red[(v * 7 + 1) * 32 + lane];
        accz += red[(v * 7 + 2) * 32 + lane];
        du += red[(v * 7 + 3) * 32 + lane];
        dv += red[(v * 7 + 4) * 32 + lane];
        vs = fmaxf(vs, red[(v * 7 + 5) * 32 + lane]);
        if (to) nint += __float_as_int(red[(v * 7 + 6) * 32 + lane]);
    }
    if (to) {
        const int io = gb + lane;
        const float4 Do = lk ? __ldg(a.srcD + io) : D;            // target io's {rho/2, P/rho^2, c, h}
        const float hoinv = lk ? 1.f / Do.w : hainv;
        const float sig = kern_sigma<float>(KS);
        const float h2 = hoinv * hoinv;
        const float sig_hg = sig * (D1 ? h2 * hoinv : h2 * h2 * hoinv);    // sigma / h_a^(D+2)
        ((float *)a.ax)[io] = sig * accx;
        ((float *)a.ay)[io] = sig * accy;
        ((float *)a.az)[io] = sig * accz;
        ((float *)a.dudt)[io] = sig * du;
        ((float *)a.divv)[io] = -sig_hg * dv / (2.f * Do.x);
        ((float *)a.vsig)[io] = vs;
    }
    for (int o = 16; o > 0; o >>= 1) nint += __shfl_xor_sync(0xffffffffu, nint, o);
    if (lane == 0) atomicAdd(&a.cnt->force_interactions, (unsigned long long)nint);
}

template <int KS>
void launch_f32(const ForceArgs &a, bool thermo, bool far, unsigned grid, cudaStream_t s)
{
    const size_t smem = 3 * sizeof(float4) * (size_t)a.uc;      // <= 48 KB: no opt-in needed
    if (thermo) {
        if (far) k_forces_f32<KS, true, true><<<grid, FB * 32, smem, s>>>(a);
        else k_forces_f32<KS, true, false><<<grid, FB * 32, smem, s>>>(a);
    } else {
        if (far) k_forces_f32<KS, false, true><<<grid, FB * 32, smem, s>>>(a);
        else k_forces_f32<KS, false, false><<<grid, FB * 32, smem, s>>>(a);
    }
}

// Equation of state and packed FP32 force-pass sources: P = (gamma-1) rho u,
// c = sqrt(gamma (gamma-1) u) to the caller's P and c, and the records
// C {vx, vy, vz, m}, D {rho/2, P/rho^2, c, h} (rho/2: the pair mean of the
// viscosity is then one addition).
__global__ void k_pack_force_f32(const float *__restrict__ vx, const float *__restrict__ vy,
                                 const float *__restrict__ vz, const float *__restrict__ m,
                                 const float *__restrict__ h, const float *__restrict__ rho,
                                 const float *__restrict__ u, float g1, float gg1, int64_t n, float *__restrict__ P,
                                 float *__restrict__ c, float4 *__restrict__ C, float4 *__restrict__ D)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float r = rho[i], ui = u[i];
    const float pi = g1 * r * ui, ci = sqrtf(gg1 * ui);
    P[i] = pi;
    c[i] = ci;
    C[i] = make_float4(vx[i], vy[i], vz[i], m[i]);
    D[i] = make_float4(0.5f * r, pi / (r * r), ci, h[i]);
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
            const double L = a.Lu, hl = 0.5 * a.Lu;
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
        // a, du/dt and div v scale as 1/length (velocities keep the caller's units)
        ((double *)a.ax)[i] = df_to_double(df_mul(sig, df_norm(accx))) * a.ls;
        ((double *)a.ay)[i] = df_to_double(df_mul(sig, df_norm(accy))) * a.ls;
        ((double *)a.az)[i] = df_to_double(df_mul(sig, df_norm(accz))) * a.ls;
        ((double *)a.dudt)[i] = df_to_double(df_mul(sig, df_norm(du))) * a.ls;
        // (the sum carries m_b in scaled mass and 1/h^(D+1) in scaled length:
        // ls / rho_sc brings sum / rho back to the caller's 1/time)
        ((double *)a.divv)[i] = (-df_to_double(df_mul(sig_hai4, df_norm(dv))) / ((const double *)a.rho)[i]) *
                                (a.ls / a.rho_sc);
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
                             int64_t n, double ls, double rho_sc, double *__restrict__ P, double *__restrict__ c,
                             float4 *__restrict__ C, float4 *__restrict__ D, float4 *__restrict__ E,
                             float4 *__restrict__ F)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double rd = rho[i], ud = u[i];
    const double pd = __dmul_rn(__dmul_rn(g1d, rd), ud);      // P exactly as the FP64 definition
    // the pair terms take h, rho and P in the scaled units (exact powers of two)
    const df r = df_from_double(rd * rho_sc), ui = df_from_double(ud), pi = df_from_double(pd * rho_sc);
    const df ci = df_sqrt(df_mul(gg1, ui));
    const df q = df_mul(pi, df_sqr(df_rcp(r)));
    P[i] = pd;
    c[i] = df_to_double(ci);
    const float2 a = split2(vx[i]), b = split2(vy[i]), cz = split2(vz[i]), hh = split2(h[i] * ls);
    C[i] = make_float4(a.x, a.y, b.x, b.y);
    D[i] = make_float4(cz.x, cz.y, hh.x, hh.y);
    E[i] = make_float4(r.hi, r.lo, q.hi, q.lo);
    F[i] = make_float4(ci.hi, ci.lo, 0.f, 0.f);
}

__global__ void k_reset_inter(DevCounters *c) { c->force_interactions = 0; }

// rho_scaled / rho = mass_scale / len_scale^D (a power of two)
double rho_scale(const sph_ctx *ctx)
{
    return std::ldexp(1.0, std::ilogb(ctx->mass_scale) - ctx->prm.dim * std::ilogb(ctx->len_scale));
}

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
            (const double *)u, g - 1.0, df_host(g * (g - 1.0)), p->n, ctx->len_scale, rho_scale(ctx),
            (double *)p->P, (double *)p->c, ctx->srcC, ctx->srcD, ctx->srcE, ctx->srcF);
    else
        k_pack_force_f32<<<grid_for(p->n, 256), 256, 0, s>>>(
            (const float *)vx, (const float *)vy, (const float *)vz, (const float *)p->m, (const float *)p->h,
            (const float *)p->rho, (const float *)u, (float)(g - 1.0), (float)(g * (g - 1.0)), p->n, (float *)p->P,
            (float *)p->c, ctx->srcC, ctx->srcD);
    SPH_CHECK_LAUNCH();
    if (!reuse_lists || !ctx->lists_valid) SPH_TRY(lists_build(ctx, p, s));
    ForceArgs a{};
    a.group_begin = ctx->group_begin;
    a.goff = ctx->group_off;
    a.gwidth = ctx->group_width;
    a.nbl = ctx->nbl;
    a.cap = ctx->nbl_cap;
    a.uni = ctx->uni;
    a.urec = ctx->urec;
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
    a.group_union = ctx->group_union;
    a.group_lo = ctx->group_lo;
    a.group_hi = ctx->group_hi;
    a.thermo = ctx->prm.energy == SPH_ENERGY_TOTAL;
    a.Lu = ctx->dom[3];
    a.ls = ctx->len_scale;
    a.rho_sc = rho_scale(ctx);
    a.L = ctx->dom[3] * ctx->len_scale;
    a.alpha = ctx->prm.alpha; a.beta = ctx->prm.beta; a.eps = ctx->prm.eps_visc;
    const double sig = kern_sigma<double>(a.kernel);
    a.Ld = df_host(a.L); a.sig_d = df_host(sig);
    a.alpha_d = df_host(a.alpha); a.beta_d = df_host(a.beta); a.eps_d = df_host(a.eps);
    a.cnt = ctx->dcnt;
    SPH_CUDA(cudaEventRecord(ctx->ev[5], s));
    if (ctx->fp64) k_forces_df<<<grid_for(ctx->n_groups, FW), FW * 32, 0, s>>>(a);
    else {
        // one instantiation per kernel form (and energy equation) keeps the
        // pair loop small; one block per target group.  Lists of this step's
        // density iteration tell their largest union; otherwise the kernel
        // reads entries beyond the staged part from global memory.
        const unsigned grid = grid_for(ctx->n_groups, 1);
        const bool th = a.thermo != 0;
        // stage the largest union when it is known and fits (the reduction
        // buffer of 7 x 32 x FB floats needs at least 224 sources' worth)
        const bool far = !(reuse_lists && ctx->lists_union_max <= UC_MAX);
        a.uc = far ? UC : std::max(224, (ctx->lists_union_max + 31) & ~31);
        switch (a.kernel) {
        case 1: launch_f32<1>(a, th, far, grid, s); break;
        case 2: launch_f32<2>(a, th, far, grid, s); break;
        case 3: launch_f32<3>(a, th, far, grid, s); break;
        case 4: launch_f32<4>(a, th, far, grid, s); break;
        case 5: launch_f32<5>(a, th, far, grid, s); break;
        default: launch_f32<0>(a, th, far, grid, s); break;
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
    int r = run();
    // lists that outgrew their predicted or bounded sizes: size them more safely
    while (r == SPH_ERR_CAPACITY && st && lists_escalate(ctx)) {
        SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
        r = run();
    }
    ctx->lists_pred_skip = false;
    return r;
}
