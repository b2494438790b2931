// Density and smoothing length (Eqs. 7 and 9): rho_a = sum_b m_b W(r_ab, h_a)
// with the self term, solved jointly with h_a = eta (m_a/rho_a)^(1/3) by a
// per-particle Newton iteration, one density evaluation per sweep:
//   f(h) = m eta^3 / h^3 - rho(h),  f'(h) = -3 m eta^3 / h^4 - drho/dh,
// bracketed by the evaluated smoothing lengths on either side of the root;
// a step leaving the closed interval [max(lo, h/2), min(hi, 2h)] (closed, so
// that a particle already at its root takes the zero step) or with f' >= 0
// is replaced by
// the midpoint towards the admissible end the sign of f points to; the
// result is clamped to [h_min, h_max].  When |h_new - h| < h_tol h the step
// is applied and one more evaluation at the final h gives rho, drho/dh and
// the neighbour count (taken as a first-order update inside the converging
// sweep when it is exact to FP64 rounding, see below).  The paper states the
// fixed point but not the solver.
//
// One warp per target group, one lane per target; each lane walks its own
// neighbour list (slot-major, coalesced).  SPH_MIXED: FP32 on two-float
// relative coordinates.  SPH_FP64: the pair terms are evaluated in
// double-float on the FP32 pipes (dfloat.cuh); the neighbour decision
// r^2 < 4 h^2 is taken in FP32 outside a relative band of 1e-5 around the
// threshold and inside it by the exact FP64 r^2 = (dx dx + dy dy) + dz dz
// without fused multiply-add, so the neighbour sets are those of plain FP64.
// Groups whose particles are all done drop out of the next sweep.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "dfloat.cuh"
#include "sph_internal.cuh"

namespace {

constexpr int DW = 4;          // warps per block
constexpr int SRC_CAP = 448;   // staged union sources per warp (mixed sweep; 7 KB)
// Mixed sweep: the largest Newton step |dh| / h accepted as converged and
// taken to first order, sqrt(h_tol / 10) (at most 1e-3): the error of the new
// h, about 2 dh^2 / h, stays below h_tol / 5 (3.2e-4 for h_tol = 1e-6)
inline double fo_step(double h_tol) { return std::min(std::sqrt(0.1 * h_tol), 1e-3); }

struct DensArgs {
    const int32_t *act;            // active groups of this sweep ...
    const int32_t *act_count;      // ... and their number (device)
    int32_t *group_mark;           // sweep stamp of the last append (sparse sweep)
    int32_t *act_next;             // groups still active after it ...
    int32_t *act_next_count;       // ... and their number (zeroed before the sweep)
    int32_t *work;                 // group claim counter (zeroed before the sweep)
    const int32_t *group_begin;
    const int64_t *goff;
    const int32_t *gwidth;
    const uint16_t *nbl;
    int64_t cap;
    const uint32_t *uni;           // group source unions
    const float4 *urec;            // their staged records (mixed: written by the list fill)
    const int64_t *uoff;
    const int32_t *group_union;    // union size per group
    const int32_t *group_img;      // 1: the group's sources include periodic images
    const float4 *group_lo, *group_hi;
    int src_cap;                   // union sources staged in shared memory per warp (mixed)
    const double *x, *y, *z;
    const float4 *srcA, *srcB;   // {xh, xl, yh, yl}, {zh, zl, m_hi, m_lo}
    void *h;
    const void *m;
    void *rho, *omega;
    int32_t *nnb;
    double *it_lo, *it_hi;
    int32_t *it_flags, *it_sweeps;
    const float *cov;
    int kernel, periodic, fixed_h, max_sweeps;   // kernel: the kernel shape (kern_shape)
    int dim;                                     // D = 1 or 3
    double L, etaD, h_tol, h_min, h_max;         // etaD = eta^D; L in the packed positions' lengths
    double fo_step;                              // fo_step(h_tol)
    df Ld, sig_d, etaD_d, hmin_d, hmax_d;        // the same constants as double-floats (h bounds scaled)
    // SPH_FP64 units (see sph_ctx::len_scale): h_scaled = h ls; the caller's
    // rho = rho_scaled rho_un, drho/dh = scaled om_un; Lu = L in the caller's units
    double ls, ls_inv, rho_un, om_un, Lu;
    DevCounters *cnt;
};

// r from r^2 by the hardware's approximate square root (one instruction,
// exact at 0); the FP32 sweep is held to relative tolerances far above its
// error
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// A warp's pair and evaluation counts over the groups it claims (lane 0),
// added to the sweep's counters once when the warp runs out of groups.
struct SweepTally {
    unsigned long long inter = 0;
    unsigned evals = 0;
};

// SPH_MIXED sweep of one group: FP32 pair terms, FP32 Newton update.  The
// group's source union is staged in shared memory (s_src, a.src_cap entries
// per chunk) as FP32 coordinates relative to the group-box centre, with the
// periodic shift folded in, and the mass; each lane then reads its
// neighbours there by their local index.
template <typename T, int KS>
__device__ __forceinline__ void density_group(const DensArgs &a, const int g, const int lane, float4 *s_src,
                                              SweepTally &tally)
{
    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const bool tgt = lane < ge - gb;
    const int i = gb + (tgt ? lane : 0);
    T *hp = (T *)a.h;
    const T *mp = (const T *)a.m;
    int32_t flags = tgt ? a.it_flags[i] : IT_DONE;
    bool active = !(flags & IT_DONE);
    const T h = active ? hp[i] : T(1);
    // a particle whose support 2h left its list waits (state unchanged) for
    // the list rebuild the host makes between sweep batches
    bool waiting = false;
    if (active && (double)(T(2) * h) > (double)a.cov[i]) {
        waiting = true;
        active = false;
        atomicAdd(&a.cnt->n_uncovered, 1);
    }
    const T hinv = T(1) / h;
    const T Dt = T(a.dim);
    const int64_t off = a.goff[g];
    int width = a.gwidth[g];
    if (off + 32 * (int64_t)width > a.cap) width = 0;    // never read past the lists

    T sum_w = T(0), sum_dh = T(0);
    int cnt = 0;
    float gap = FLT_MAX;  // smallest |r^2 - 4 h^2| over the list entries
    if (__any_sync(0xffffffffu, active)) {
        const float4 qlo = a.group_lo[g], qhi = a.group_hi[g];
        const float gcx = 0.5f * (qlo.x + qhi.x), gcy = 0.5f * (qlo.y + qhi.y), gcz = 0.5f * (qlo.z + qhi.z);
        const float4 A = a.srcA[i], Bz = a.srcB[i];
        const float tx = (A.x - gcx) + A.y, ty = (A.z - gcy) + A.w, tz = (Bz.x - gcz) + Bz.y;
        const float hf = (float)h;
        const float thr = __fmul_rn(__fmul_rn(4.f, hf), hf);
        const int U = a.group_union[g];
        const float4 *Rg = a.urec + a.uoff[g];
        const unsigned long long *lq = reinterpret_cast<const unsigned long long *>(a.nbl + off) + lane;
        // a group with at most 16 targets left to evaluate gives each one a
        // segment of k = 32 / nextpow2(count) lanes that splits its list (a
        // lane-per-target walk would leave most lanes idle)
        const unsigned amask = __ballot_sync(0xffffffffu, active);
        const int nact = __popc(amask);
        const int lk = nact > 16 ? 0 : 5 - (nact > 1 ? 32 - __clz(nact - 1) : 0);   // log2 k
        for (int c0 = 0; c0 < U; c0 += a.src_cap) {
            const int cn = min(a.src_cap, U - c0);
            __syncwarp();
            // the list fill wrote each union member's record {x, y, z
            // relative to the group-box centre, nearest image, m}: one
            // asynchronous 16-byte copy per source, all of them in flight
            for (int t = lane; t < cn; t += 32) cp_async16(&s_src[t], Rg + c0 + t);
            cp_async_wait_all();
            __syncwarp();
            if (lk > 0) {
                // segment s (lanes [s k, s k + k)) takes the s-th active
                // target; lane r of the segment walks its quads r, r + k, ...
                // and the segment's partial sums meet by shuffles, then move
                // to the target's own lane
                const int k = 1 << lk, seg = lane >> lk, r = lane & (k - 1);
                const bool has = seg < nact;
                const int t = has ? (int)__fns(amask, 0u, seg + 1) : 0;
                const float ttx = __shfl_sync(0xffffffffu, tx, t), tty = __shfl_sync(0xffffffffu, ty, t),
                            ttz = __shfl_sync(0xffffffffu, tz, t);
                const float tthr = __shfl_sync(0xffffffffu, thr, t);
                const T thinv = __shfl_sync(0xffffffffu, hinv, t);
                const unsigned long long *lq0 = reinterpret_cast<const unsigned long long *>(a.nbl + off) + t;
                const int nq = has ? width >> 2 : 0;
                T sw = T(0), sd = T(0);
                int c = 0;
                float gp = FLT_MAX;
                // quads r, r + k in one batch, the next two in flight
                auto quad = [&](int qi) -> unsigned long long {
                    return qi < nq ? __ldg(lq0 + 32 * (int64_t)qi) : ~0ull;
                };
                unsigned long long n0 = quad(r), n1 = quad(r + k);
                for (int qi = r; qi < nq; qi += 2 * k) {
                    const unsigned long long q0 = n0, q1 = n1;
                    n0 = quad(qi + 2 * k);
                    n1 = quad(qi + 3 * k);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const uint32_t e = (uint32_t)((u < 4 ? q0 : q1) >> (16 * (u & 3))) & 0xFFFFu;
                        const int le = (int)e - c0;
                        if ((unsigned)le >= (unsigned)cn) continue;
                        const float4 q = s_src[le];
                        const float dx = ttx - q.x, dy = tty - q.y, dz = ttz - q.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        gp = fminf(gp, fabsf(r2 - tthr));
                        if (!(r2 < tthr)) continue;
                        const T qq = (T)sqrt_approx(r2) * thinv;
                        T w, gg;
                        kern_wg<T>(KS, qq, w, gg);
                        const T mb = (T)q.w;
                        sw = fmaf(mb, w, sw);
                        sd = fmaf(mb, gg, sd);
                        ++c;
                    }
                }
                for (int o = k >> 1; o > 0; o >>= 1) {
                    sw += __shfl_xor_sync(0xffffffffu, sw, o);
                    sd += __shfl_xor_sync(0xffffffffu, sd, o);
                    c += __shfl_xor_sync(0xffffffffu, c, o);
                    gp = fminf(gp, __shfl_xor_sync(0xffffffffu, gp, o));
                }
                // an active lane's segment is its rank among the active lanes
                const int from = active ? __popc(amask & ((1u << lane) - 1u)) << lk : 0;
                sw = __shfl_sync(0xffffffffu, sw, from);
                sd = __shfl_sync(0xffffffffu, sd, from);
                c = __shfl_sync(0xffffffffu, c, from);
                gp = __shfl_sync(0xffffffffu, gp, from);
                if (active) {
                    sum_w += sw;
                    sum_dh += sd;
                    cnt += c;
                    gap = fminf(gap, gp);
                }
            } else if (active) {
                // list entries in batches of LB = 8 (two quads), the next
                // batch in flight while this one is processed (empty slots
                // fall outside [0, cn))
                constexpr int LB = 8;
                auto quad = [&](int qi) -> unsigned long long {
                    return 4 * qi < width ? __ldg(lq + 32 * (int64_t)qi) : ~0ull;
                };
                unsigned long long n0 = quad(0), n1 = quad(1);
                for (int k0 = 0; k0 < width; k0 += LB) {
                    const unsigned long long q0 = n0, q1 = n1;
                    n0 = quad((k0 >> 2) + 2);
                    n1 = quad((k0 >> 2) + 3);
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                    const uint32_t e = (uint32_t)((u < 4 ? q0 : q1) >> (16 * (u & 3))) & 0xFFFFu;
                    const int le = (int)e - c0;
                    if ((unsigned)le >= (unsigned)cn) continue;
                    const float4 q = s_src[le];
                    const float dx = tx - q.x, dy = ty - q.y, dz = tz - q.z;
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    gap = fminf(gap, fabsf(r2 - thr));
                    if (!(r2 < thr)) continue;
                    const T qq = (T)sqrt_approx(r2) * hinv;
                    T w, g;
                    kern_wg<T>(KS, qq, w, g);          // the kernel form fixed at compile time
                    const T mb = (T)q.w;
                    sum_w = fmaf(mb, w, sum_w);
                    sum_dh = fmaf(mb, g, sum_dh);     // m (D w + q w')
                    ++cnt;
                    }
                }
            }
        }
    }

    bool still = false;
    if (active) {
        const T ma = mp[i];
        sum_w += ma;                    // self term, w(0) = 1 for every kernel
        sum_dh += Dt * ma;              // D w(0) + 0 w'(0)
        const T sig = kern_sigma<T>(a.kernel);
        const T hDi = inv_pow_dim(hinv, a.dim);
        const T rho = sig * hDi * sum_w;
        const T drho = -sig * hDi * hinv * sum_dh;
        const T metaD = ma * (T)a.etaD;
        const int sweeps = a.it_sweeps[i] + 1;
        a.it_sweeps[i] = sweeps;
        bool done = false;
        T hn = h, hfin = h, rho_out = rho;
        if (flags & IT_FINAL) {
            done = true;
        } else {
            const T f = metaD * hDi - rho;
            if (f == T(0)) {
                done = true;
            } else if (sweeps >= a.max_sweeps) {
                done = true;
                flags |= IT_NOT_CONV;
            } else {
                const T fp = -Dt * metaD * hDi * hinv - drho;
                double lo = a.it_lo[i], hi = a.it_hi[i];
                if (f > T(0)) { if ((double)h > lo) lo = (double)h; }
                else { if ((double)h < hi) hi = (double)h; }
                const T alo = T(0.5) * h > (T)lo ? T(0.5) * h : (T)lo;
                const T ahi = T(2) * h < (T)hi ? T(2) * h : (T)hi;
                bool ok = false;
                if (fp < T(0)) {
                    hn = h - f / fp;
                    ok = (hn >= alo) && (hn <= ahi);
                }
                if (!ok) hn = f > T(0) ? T(0.5) * (h + ahi) : T(0.5) * (h + alo);
                if (hn < (T)a.h_min) { hn = (T)a.h_min; ok = false; }
                if (hn > (T)a.h_max) { hn = (T)a.h_max; ok = false; }
                // Newton converges quadratically: after a Newton step of
                // |dh| < fo_step h the error of the new h is about 2 dh^2 / h
                // (f''/2f' ~ -2/h for f = m eta^D / h^D - rho near the root,
                // rho nearly constant in h), below h_tol / 5; the FP32 sweep
                // accepts such a step
                const double adh = fabs((double)(hn - h));
                const bool conv = adh < a.h_tol * (double)h || (ok && adh < a.fo_step * (double)h);
                a.it_lo[i] = lo;
                a.it_hi[i] = hi;
                hp[i] = hn;
                if (conv) {
                    // The reading evaluates rho once more at the final h.  When
                    // no list entry's r^2 lies between 4 h^2 and 4 (h + dh)^2
                    // (|4 (h + dh)^2 - 4 h^2| <= 8.004 h |dh| for |dh| <=
                    // fo_step h <= 1e-3 h; tested with 10 h |dh| plus 4e-6 h^2
                    // for the FP32 rounding of r^2), the neighbour set at
                    // h + dh is this one and rho(h + dh) = rho + rho' dh up to
                    // rho'' dh^2 / 2, a relative O(10 (dh/h)^2) <= h_tol (1e-6
                    // by default: inside the mixed mode's stated density
                    // error).  That evaluation is taken here without another
                    // sweep.
                    // (and the list must still cover 2 (h + dh))
                    const double need = (double)h * (10.0 * adh + 4e-6 * (double)h);
                    if (adh < a.fo_step * (double)h && (double)gap > need && 2.0 * (double)hn <= (double)a.cov[i]) {
                        rho_out = rho + drho * (hn - h);
                        hfin = hn;
                        done = true;
                    } else {
                        flags |= IT_FINAL;
                    }
                }
            }
        }
        if (done) {
            flags |= IT_DONE;
            if (flags & IT_NOT_CONV) atomicAdd(&a.cnt->n_not_conv, 1);
            else if (!a.fixed_h && ((double)hfin <= a.h_min || (double)hfin >= a.h_max)) {
                flags |= IT_H_BOUNDS;
                atomicAdd(&a.cnt->n_hbounds, 1);
            }
        }
        ((T *)a.rho)[i] = rho_out;
        ((T *)a.omega)[i] = drho;
        a.nnb[i] = cnt;
        a.it_flags[i] = flags;
        still = !done;
    }
    if (waiting) still = true;
    int c = cnt;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    const unsigned smask = __ballot_sync(0xffffffffu, still);
    if (lane == 0) {
        tally.inter += (unsigned long long)c;
        tally.evals += (unsigned)__popc(amask);
        if (smask) a.act_next[atomicAdd(a.act_next_count, 1)] = g;
    }
}

// SPH_FP64 sweep of one group.  GB300 executes FP64 at 1/64 of the FP32
// rate, so besides the pair terms the per-particle Newton update also runs in
// double-float (about 48 significant bits); FP64 instructions remain only for
// reading and writing the caller's double arrays and for the exact neighbour
// decisions near the support radius.  The iteration bracket of FP64 mode is
// kept as double-floats in the 8-byte slots of it_lo / it_hi.
__device__ __forceinline__ bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ df df_ld(const double *p) { const float2 v = *reinterpret_cast<const float2 *>(p); return df{v.x, v.y}; }
__device__ __forceinline__ void df_st(double *p, df v) { *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo); }

// One list entry b of target i in FP64 mode: the exact neighbour decision and
// the double-float terms m_b W and m_b (3 W + q W') of rho and drho/dh.
struct DfTarget {
    float4 A, Bz;                  // two-float position and mass of the target
    double hd;                     // its h
    df hinv;
    float thr_hi, thr_lo;          // FP32 band around 4 h^2
    int64_t i;
    int img;                       // periodic images among the group's sources
};

__device__ __forceinline__ DfTarget df_target(const DensArgs &a, int64_t i, double hd, df h, int g)
{
    DfTarget t;
    t.img = a.periodic && a.group_img[g];
    t.A = a.srcA[i];
    t.Bz = a.srcB[i];
    t.hd = hd;
    t.hinv = df_rcp(h);
    const float thr_f = df_scale(df_sqr(h), 4.f).hi;
    t.thr_hi = thr_f * (1.f + 1e-5f);
    t.thr_lo = thr_f * (1.f - 1e-5f);
    t.i = i;
    return t;
}

__device__ __forceinline__ void df_pair(const DensArgs &a, const DfTarget &t, uint32_t b, const float4 &P,
                                        const float4 &Q, df &sw, df &sd, int &cnt, int &band)
{
    const float Lf = (float)a.L, half = 0.5f * Lf, guard = 0.45f * Lf;
    int wx, wy, wz;
    const float dxf = sep_fw(t.A.x, t.A.y, P.x, P.y, t.img, Lf, half, wx);
    const float dyf = sep_fw(t.A.z, t.A.w, P.z, P.w, t.img, Lf, half, wy);
    const float dzf = sep_fw(t.Bz.x, t.Bz.y, Q.x, Q.y, t.img, Lf, half, wz);
    const float r2f = (dxf * dxf + dyf * dyf) + dzf * dzf;
    if (r2f > t.thr_hi) return;
    if (r2f >= t.thr_lo) ++band;
    if (r2f >= t.thr_lo || (t.img && fmaxf(fmaxf(fabsf(dxf), fabsf(dyf)), fabsf(dzf)) > guard)) {
        // knife edge: the exact FP64 decision of the plain definition
        const double L = a.Lu, hl = 0.5 * a.Lu;
        const double dx = sep_d(a.x[t.i], a.x[b], a.periodic, L, hl);
        const double dy = sep_d(a.y[t.i], a.y[b], a.periodic, L, hl);
        const double dz = sep_d(a.z[t.i], a.z[b], a.periodic, L, hl);
        if (!(r2_d(dx, dy, dz) < __dmul_rn(__dmul_rn(4.0, t.hd), t.hd))) return;
    }
    const df dx = df_sep_fast(t.A.x, t.A.y, P.x, P.y, wx, a.Ld);
    const df dy = df_sep_fast(t.A.z, t.A.w, P.z, P.w, wy, a.Ld);
    const df dz = df_sep_fast(t.Bz.x, t.Bz.y, Q.x, Q.y, wz, a.Ld);
    const df q = df_mul_u(df_sqrt_fast(df_norm2(dx, dy, dz)), t.hinv);
    df w, g3;
    df_kern_w_g3(a.kernel, q, w, g3);
    const df mb = df{Q.z, Q.w};
    df_acc(sw, df_mul_u(mb, w));
    df_acc(sd, df_mul_u(mb, g3));
    ++cnt;
}

// The Newton update of target t from its sums (self term added here); writes
// h, rho, omega, nnb and the iteration state; returns whether it iterates on.
__device__ __forceinline__ bool df_finalize(const DensArgs &a, const DfTarget &t, df h, int32_t flags, df sw,
                                            df sd, int cnt, int band)
{
    const int64_t i = t.i;
    double *hp = (double *)a.h;
    const df hinv = t.hinv;
    const df ma = df{t.Bz.z, t.Bz.w};
    sw = df_add(df_norm(sw), ma);                   // self term, w(0) = 1 for every kernel
    sd = df_add(df_norm(sd), df_mul_f(ma, (float)a.dim));    // D w(0) + 0 w'(0)
    const df hDi = a.dim == 1 ? hinv : df_mul(df_sqr(hinv), hinv);
    const df shD = df_mul(a.sig_d, hDi);
    const df rho = df_mul(shD, sw);
    const df drho = df_neg(df_mul(df_mul(shD, hinv), sd));
    const df metaD = df_mul(ma, a.etaD_d);
    const int sweeps = a.it_sweeps[i] + 1;
    a.it_sweeps[i] = sweeps;
    bool done = false;
    df hn = h, hfin = h, rho_out = rho;
    if (flags & IT_FINAL) {
        done = true;
    } else {
        const df mhD = df_mul(metaD, hDi);
        const df f = df_sub(mhD, rho);
        if (f.hi == 0.f) {
            done = true;
        } else if (sweeps >= a.max_sweeps) {
            done = true;
            flags |= IT_NOT_CONV;
        } else {
            const df fp = df_sub(df_mul_f(df_mul(mhD, hinv), -(float)a.dim), drho);
            df lo = df_ld(a.it_lo + i), hi = df_ld(a.it_hi + i);
            if (f.hi > 0.f) { if (df_lt(lo, h)) lo = h; }
            else { if (df_lt(h, hi)) hi = h; }
            const df h2 = df_scale(h, 0.5f), h_2 = df_scale(h, 2.f);
            const df alo = df_lt(lo, h2) ? h2 : lo;
            const df ahi = df_lt(h_2, hi) ? h_2 : hi;
            bool ok = false;
            if (df_lt0(fp)) {
                hn = df_sub(h, df_mul(f, df_rcp(fp)));
                ok = !df_lt(hn, alo) && !df_lt(ahi, hn);
            }
            if (!ok) hn = df_scale(df_add(h, f.hi > 0.f ? ahi : alo), 0.5f);
            int clamp = 0;                           // the bounds are written exactly
            if (df_lt(hn, a.hmin_d)) { hn = a.hmin_d; clamp = -1; }
            if (df_lt(a.hmax_d, hn)) { hn = a.hmax_d; clamp = 1; }
            const df dh = df_sub(hn, h);
            const float adh = fabsf(dh.hi);
            const bool conv = adh < (float)a.h_tol * h.hi;
            df_st(a.it_lo + i, lo);
            df_st(a.it_hi + i, hi);
            hp[i] = clamp < 0 ? a.h_min : clamp > 0 ? a.h_max : df_to_double(hn) * a.ls_inv;
            if (conv) {
                // first-order finalization as in the mixed path (see there),
                // for |dh| <= 1e-7 h: the neglected term, a relative
                // O(10 (dh/h)^2) <= 1e-13, sits at the double-float rounding
                if (band == 0 && adh <= 1e-7f * h.hi) {
                    rho_out = df_add(rho, df_mul(drho, dh));
                    hfin = hn;
                    done = true;
                } else {
                    flags |= IT_FINAL;
                }
            }
        }
    }
    if (done) {
        flags |= IT_DONE;
        if (flags & IT_NOT_CONV) atomicAdd(&a.cnt->n_not_conv, 1);
        else if (!a.fixed_h && (!df_lt(a.hmin_d, hfin) || !df_lt(hfin, a.hmax_d))) {
            flags |= IT_H_BOUNDS;
            atomicAdd(&a.cnt->n_hbounds, 1);
        }
    }
    ((double *)a.rho)[i] = df_to_double(rho_out) * a.rho_un;
    ((double *)a.omega)[i] = df_to_double(drho) * a.om_un;
    a.nnb[i] = cnt;
    a.it_flags[i] = flags;
    return !done;
}

// a particle whose support 2h left its list waits (state unchanged) for the
// list rebuild the host makes between sweep batches
__device__ __forceinline__ bool df_waiting(const DensArgs &a, int64_t i, df h)
{
    return df_lt(df{a.cov[i], 0.f}, df_scale(h, 2.f));
}

// Dense FP64 sweep of one group: one lane per target, each walking its list.
__device__ __forceinline__ void density_group_df(const DensArgs &a, const int g, const int lane, SweepTally &tally)
{
    const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
    const bool tgt = lane < ge - gb;
    const int i = gb + (tgt ? lane : 0);
    int32_t flags = tgt ? a.it_flags[i] : IT_DONE;
    bool active = !(flags & IT_DONE);
    const double hd = active ? ((const double *)a.h)[i] : 1.0;
    const df h = df_from_double(hd * a.ls);
    bool waiting = false;
    if (active && df_waiting(a, i, h)) {
        waiting = true;
        active = false;
        atomicAdd(&a.cnt->n_uncovered, 1);
    }
    const DfTarget t = df_target(a, i, hd, h, g);
    const int64_t off = a.goff[g];
    int width = a.gwidth[g];
    if (off + 32 * (int64_t)width > a.cap) width = 0;    // never read past the lists

    df sw = df{0.f, 0.f}, sd = df{0.f, 0.f};
    int cnt = 0;
    int band = 0;        // list entries within a relative 1e-5 of the support radius
    if (active)
        walk_list<true>(a.nbl, off, width, lane, (uint32_t)i, a.uni, a.uoff[g], a.srcA, a.srcB,
                        [&](uint32_t b, const float4 &P, const float4 &Q) { df_pair(a, t, b, P, Q, sw, sd, cnt, band); });
    bool still = false;
    if (active) still = df_finalize(a, t, h, flags, sw, sd, cnt, band);
    if (waiting) still = true;
    int c = cnt;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    const unsigned smask = __ballot_sync(0xffffffffu, still);
    if (lane == 0) {
        tally.inter += (unsigned long long)c;
        tally.evals += (unsigned)__popc(amask);
        if (smask) a.act_next[atomicAdd(a.act_next_count, 1)] = g;
    }
}

// Sparse FP64 sweep, for sweeps with few active groups: a warp per target
// still iterating, its list split over the 32 lanes (slots k = lane mod 32)
// and the double-float sums combined by a shuffle tree.  The dense sweep puts
// one whole list on one lane, whose serial double-float chain then bounds a
// sweep that touches few particles.
constexpr int SPARSE_MAX_GROUPS = 1024;   // active groups below which the sparse sweep runs

__global__ void __launch_bounds__(DW * 32) k_density_sparse(DensArgs a)
{
    const int lane = threadIdx.x & 31;
    const int n_act = *a.act_count;
    if (n_act >= SPARSE_MAX_GROUPS) return;
    const int stamp = a.cnt->sweep_stamp;
    const int items = 32 * n_act;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(a.work, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= items) break;
        const int g = a.act[it >> 5], p = it & 31;
        const int gb = a.group_begin[g], ge = a.group_begin[g + 1];
        if (p >= ge - gb) continue;
        const int i = gb + p;
        const int32_t flags = a.it_flags[i];
        if (flags & IT_DONE) continue;
        const double hd = ((const double *)a.h)[i];
        const df h = df_from_double(hd * a.ls);
        bool still;
        if (df_waiting(a, i, h)) {
            if (lane == 0) atomicAdd(&a.cnt->n_uncovered, 1);
            still = true;
        } else {
            const DfTarget t = df_target(a, i, hd, h, g);
            const int64_t off = a.goff[g];
            int width = a.gwidth[g];
            if (off + 32 * (int64_t)width > a.cap) width = 0;
            const uint32_t *U = a.uni + a.uoff[g];
            df sw = df{0.f, 0.f}, sd = df{0.f, 0.f};
            int cnt = 0, band = 0;
            for (int k = lane; k < width; k += 32) {
                const uint32_t e = a.nbl[slot_index(off, k, p)];
                if (e == SPH_LOCAL_NONE) continue;
                const uint32_t b = __ldg(U + e);
                df_pair(a, t, b, __ldg(a.srcA + b), __ldg(a.srcB + b), sw, sd, cnt, band);
            }
            sw = df_norm(sw);
            sd = df_norm(sd);
            for (int o = 16; o > 0; o >>= 1) {
                sw = df_add(sw, df{__shfl_xor_sync(0xffffffffu, sw.hi, o), __shfl_xor_sync(0xffffffffu, sw.lo, o)});
                sd = df_add(sd, df{__shfl_xor_sync(0xffffffffu, sd.hi, o), __shfl_xor_sync(0xffffffffu, sd.lo, o)});
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
                band += __shfl_xor_sync(0xffffffffu, band, o);
            }
            still = false;
            if (lane == 0) {
                still = df_finalize(a, t, h, flags, sw, sd, cnt, band);
                atomicAdd(&a.cnt->interactions, (unsigned long long)cnt);
                atomicAdd(&a.cnt->evaluations, 1ull);
            }
        }
        // the group iterates on if any of its targets does (appended once per sweep)
        if (lane == 0 && still && atomicExch(a.group_mark + g, stamp) != stamp)
            a.act_next[atomicAdd(a.act_next_count, 1)] = g;
    }
}

// One sweep over the active groups, whose number is read on the device, so
// sweeps can be queued without a host round trip.  The grid is sized to the
// resident blocks; each warp claims its next group from a counter, so groups
// of unequal list widths balance across the SMs.
template <typename T, bool FP64POS, int KS>
__global__ void __launch_bounds__(DW * 32) k_density(DensArgs a)
{
    extern __shared__ float4 s_dyn[];
    const int lane = threadIdx.x & 31;
    float4 *s_src = s_dyn + (threadIdx.x >> 5) * a.src_cap;
    const int n_act = *a.act_count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && n_act > 0) atomicAdd(&a.cnt->sweeps_done, 1);
    if (FP64POS && n_act < SPARSE_MAX_GROUPS) return;   // k_density_sparse takes this sweep
    SweepTally tally;
    auto claim = [&]() {
        int gi = 0;
        if (lane == 0) gi = atomicAdd(a.work, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        return gi < n_act ? a.act[gi] : -1;
    };
    if constexpr (FP64POS) {
        for (int g = claim(); g >= 0; g = claim()) density_group_df(a, g, lane, tally);
    } else {
        // the next group is claimed (and its index read) before this one is
        // evaluated, so the claim's round trip overlaps the evaluation
        int g = claim();
        while (g >= 0) {
            const int next = claim();
            density_group<T, KS>(a, g, lane, s_src, tally);
            g = next;
        }
    }
    if (lane == 0 && tally.evals) {
        atomicAdd(&a.cnt->interactions, tally.inter);
        atomicAdd(&a.cnt->evaluations, (unsigned long long)tally.evals);
    }
}

template <typename T>
__global__ void k_dens_init(T *__restrict__ h, const T *__restrict__ seed, int64_t n, int fixed_h,
                            int32_t *__restrict__ flags, int32_t *__restrict__ sweeps, double *__restrict__ lo,
                            double *__restrict__ hi, int df_bracket)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (seed) h[i] = seed[i];
    flags[i] = fixed_h ? IT_FINAL : 0;
    sweeps[i] = 0;
    if (df_bracket) {                               // double-float {0, 0} and {+inf, 0}
        df_st(lo + i, df{0.f, 0.f});
        df_st(hi + i, df{__int_as_float(0x7f800000), 0.f});
    } else {
        lo[i] = 0.0;
        hi[i] = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    }
}

__global__ void k_iota_i32(int32_t *v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

// before a sweep: nothing active yet for the next one
__global__ void k_begin_sweep(DevCounters *c, int next)
{
    c->act_count[next] = 0;
    c->work[next ^ 1] = 0;
    c->sweep_stamp += 1;
}

__global__ void k_clear_uncovered(DevCounters *c) { c->n_uncovered = 0; }

__global__ void k_reset_status(DevCounters *c, int n_groups)
{
    c->n_not_conv = 0;
    c->n_hbounds = 0;
    c->err = 0;
    c->interactions = 0;
    c->evaluations = 0;
    c->sweeps_done = 0;
    c->n_uncovered = 0;
    c->act_count[0] = n_groups;
}

// Ideal-gas EOS: P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u).
template <typename T>
__global__ void k_eos(const T *__restrict__ rho, const T *__restrict__ u, int64_t n, double gamma,
                      T *__restrict__ P, T *__restrict__ c)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T g = (T)gamma, g1 = (T)(gamma - 1.0);
    const T ui = u[i];
    P[i] = g1 * rho[i] * ui;
    c[i] = sqrt(g * g1 * ui);
}

// resident blocks per SM of the sweep kernel (from the occupancy calculator)
template <typename T>
unsigned resident_blocks(bool fp64pos)
{
    static int cached[2] = {0, 0};
    int &c = cached[fp64pos ? 1 : 0];
    if (c == 0) {
        int nb = 0;
        const cudaError_t e = fp64pos
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_density<double, true, 0>, DW * 32, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_density<float, false, 1>, DW * 32,
                                                            sizeof(float4) * DW * SRC_CAP);
        c = (e == cudaSuccess && nb > 0) ? nb : 8;
    }
    return (unsigned)c;
}

template <typename T>
int run_once(sph_ctx *ctx, sph_particles *p, const void *seed, sph_density_stats *st, bool eos, cudaStream_t s)
{
    const int64_t n = p->n;
    const sph_params &q = ctx->prm;
    const int64_t launches0 = ctx->launches;
    const int ng = (int)ctx->n_groups;
    k_reset_status<<<1, 1, 0, s>>>(ctx->dcnt, ng);
    SPH_CHECK_LAUNCH();
    k_dens_init<T><<<grid_for(n, 256), 256, 0, s>>>((T *)p->h, (const T *)seed, n, q.fixed_h, ctx->it_flags,
                                                     ctx->it_sweeps, ctx->it_lo, ctx->it_hi, ctx->fp64 ? 1 : 0);
    SPH_CHECK_LAUNCH();
    SPH_CUDA(cudaEventRecord(ctx->lev[0], s));
    SPH_TRY(lists_build(ctx, p, s));
    SPH_CUDA(cudaEventRecord(ctx->lev[1], s));
    k_iota_i32<<<grid_for(ng, 256), 256, 0, s>>>(ctx->act_groups[0], ng);
    SPH_CHECK_LAUNCH();
    DensArgs a{};
    a.group_begin = ctx->group_begin;
    a.goff = ctx->group_off;
    a.gwidth = ctx->group_width;
    a.nbl = ctx->nbl;
    a.cap = ctx->nbl_cap;
    a.uni = ctx->uni;
    a.urec = ctx->urec;
    a.uoff = ctx->union_off;
    a.group_union = ctx->group_union;
    a.group_img = ctx->group_img;
    a.group_mark = ctx->group_mark;
    a.group_lo = ctx->group_lo;
    a.group_hi = ctx->group_hi;
    a.src_cap = ctx->fp64 ? 0 : SRC_CAP;
    const size_t smem = ctx->fp64 ? 0 : sizeof(float4) * DW * SRC_CAP;
    a.x = p->x; a.y = p->y; a.z = p->z;
    a.srcA = ctx->srcA; a.srcB = ctx->srcB;
    a.h = p->h; a.m = p->m; a.rho = p->rho; a.omega = p->omega; a.nnb = p->nnb;
    a.it_lo = ctx->it_lo; a.it_hi = ctx->it_hi; a.it_flags = ctx->it_flags; a.it_sweeps = ctx->it_sweeps;
    a.cov = ctx->cov;
    a.kernel = kern_shape(q.kernel, q.dim); a.dim = q.dim;
    a.periodic = q.periodic; a.fixed_h = q.fixed_h; a.max_sweeps = q.max_sweeps;
    const double ls = ctx->len_scale;
    a.ls = ls;
    a.ls_inv = 1.0 / ls;                           // powers of two: exact
    a.rho_un = std::ldexp(1.0, q.dim * std::ilogb(ls) - std::ilogb(ctx->mass_scale));   // rho scales as m / L^D
    a.om_un = a.rho_un * ls;
    a.Lu = ctx->dom[3];
    a.L = ctx->dom[3] * ls;
    a.etaD = q.dim == 1 ? q.eta : q.eta * q.eta * q.eta;
    a.h_tol = q.h_tol; a.h_min = q.h_min; a.h_max = q.h_max;
    a.fo_step = fo_step(q.h_tol);
    const double sig = kern_sigma<double>(a.kernel);
    a.Ld = df_host(a.L); a.sig_d = df_host(sig); a.etaD_d = df_host(a.etaD);
    a.hmin_d = df_host(q.h_min * ls); a.hmax_d = df_host(q.h_max * ls);
    a.cnt = ctx->dcnt;
    // sweeps are queued in batches without a host round trip: each reads the
    // number of active groups left by the previous one on the device.  A
    // particle whose 2h outgrew its list sits out (unchanged) until the host
    // rebuilds the lists at the end of the batch.
    const unsigned grid = std::min<unsigned>(grid_for(ng, DW), (unsigned)ctx->num_sms * resident_blocks<T>(ctx->fp64));
    const int max_launch = 4 * (q.max_sweeps + 2);
    // a seeded iteration (the h-predictor's guess) typically ends after three
    // sweeps, the plain one after four
    const int batch = q.fixed_h ? 1 : (seed ? 3 : 4);
    int cur = 0, launched = 0, rebuilds = 0;
    bool rebuilt = false;                  // a rebuild is timed by lev[2..3] until the next synchronisation
    double lists_ms = 0.0;
    for (;;) {
        for (int j = 0; j < batch && launched < max_launch; ++j) {
            k_begin_sweep<<<1, 1, 0, s>>>(ctx->dcnt, cur ^ 1);
            SPH_CHECK_LAUNCH();
            a.act = ctx->act_groups[cur];
            a.act_count = &ctx->dcnt->act_count[cur];
            a.act_next = ctx->act_groups[cur ^ 1];
            a.act_next_count = &ctx->dcnt->act_count[cur ^ 1];
            a.work = &ctx->dcnt->work[cur];
            if (launched < 64) SPH_CUDA(cudaEventRecord(ctx->kev[2 * launched], s));
            if constexpr (std::is_same<T, double>::value) {
                k_density<double, true, 0><<<grid, DW * 32, 0, s>>>(a);
                SPH_CHECK_LAUNCH();
                k_density_sparse<<<(unsigned)ctx->num_sms * 8u, DW * 32, 0, s>>>(a);
            } else {
                // one instantiation per kernel form keeps the hot loop small
                switch (a.kernel) {
                case 1: k_density<float, false, 1><<<grid, DW * 32, smem, s>>>(a); break;
                case 2: k_density<float, false, 2><<<grid, DW * 32, smem, s>>>(a); break;
                case 3: k_density<float, false, 3><<<grid, DW * 32, smem, s>>>(a); break;   // M4, D = 1
                case 4: k_density<float, false, 4><<<grid, DW * 32, smem, s>>>(a); break;
                case 5: k_density<float, false, 5><<<grid, DW * 32, smem, s>>>(a); break;
                default: k_density<float, false, 0><<<grid, DW * 32, smem, s>>>(a); break;   // M4, D = 3
                }
            }
            SPH_CHECK_LAUNCH();
            if (launched < 64) SPH_CUDA(cudaEventRecord(ctx->kev[2 * launched + 1], s));
            cur ^= 1;
            ++launched;
        }
        SPH_TRY(sync_counters(ctx, s));
        if (rebuilt) {
            float f = 0.f;
            SPH_CUDA(cudaEventElapsedTime(&f, ctx->lev[2], ctx->lev[3]));
            lists_ms += f;
            rebuilt = false;
        }
        if (ctx->hcnt->err & (ERRB_LIST_CAPACITY | ERRB_STACK))
            return sph_fail(ctx, SPH_ERR_CAPACITY, "sph_density: neighbour-list capacity exceeded");
        if (ctx->hcnt->act_count[cur] == 0 || launched >= max_launch) break;
        if (ctx->hcnt->n_uncovered > 0) {
            SPH_CUDA(cudaEventRecord(ctx->lev[2], s));
            SPH_TRY(lists_build(ctx, p, s));
            SPH_CUDA(cudaEventRecord(ctx->lev[3], s));
            k_clear_uncovered<<<1, 1, 0, s>>>(ctx->dcnt);
            SPH_CHECK_LAUNCH();
            ++rebuilds;
            rebuilt = true;
        }
    }
    {
        float f = 0.f;
        SPH_CUDA(cudaEventElapsedTime(&f, ctx->lev[0], ctx->lev[1]));
        lists_ms += f;
    }
    // the lists of this iteration were built before its last synchronisation
    if (!(ctx->hcnt->err & (ERRB_LIST_CAPACITY | ERRB_STACK))) ctx->lists_union_max = ctx->hcnt->union_max;
    double kernel_ms = 0.0;
    for (int k = 0; k < launched && k < 64; ++k) {
        float f = 0.f;
        SPH_CUDA(cudaEventElapsedTime(&f, ctx->kev[2 * k], ctx->kev[2 * k + 1]));
        kernel_ms += f;
    }
    if (eos) SPH_TRY(eos_run(ctx, p, p->u, s));
    if (st) {
        st->sweeps = ctx->hcnt->sweeps_done;
        st->list_builds = 1 + rebuilds;
        st->n_unconverged = ctx->hcnt->n_not_conv;
        st->n_hbounds = ctx->hcnt->n_hbounds;
        st->interactions = (int64_t)ctx->hcnt->interactions;
        st->list_entries = (int64_t)ctx->hcnt->list_used;
        st->evaluations = (int64_t)ctx->hcnt->evaluations;
        st->kernel_ms = kernel_ms;
        st->lists_ms = lists_ms;
        st->launches = ctx->launches - launches0;
    }
    if (ctx->hcnt->act_count[cur] > 0)
        return sph_fail(ctx, SPH_ERR_NOT_CONVERGED, "sph_density: sweep budget exhausted with " +
                                                        std::to_string(ctx->hcnt->act_count[cur]) + " groups active");
    if (ctx->hcnt->n_not_conv > 0)
        return sph_fail(ctx, SPH_ERR_NOT_CONVERGED, "sph_density: h iteration reached max_sweeps for " +
                                                        std::to_string(ctx->hcnt->n_not_conv) + " particles");
    if (ctx->hcnt->n_hbounds > 0)
        return sph_fail(ctx, SPH_ERR_H_BOUNDS, "sph_density: converged h on h_min/h_max for " +
                                                   std::to_string(ctx->hcnt->n_hbounds) + " particles");
    return SPH_OK;
}

// Lists sized by prediction or by leaf bounds can outgrow their sizes where
// exact counts fit in nb_capacity: the iteration then restarts from its first
// guess with the safer sizing (leaf bounds for this call after a prediction,
// exact counts from now on after leaf bounds).
template <typename T>
int run_impl(sph_ctx *ctx, sph_particles *p, const void *seed, sph_density_stats *st, bool eos, cudaStream_t s)
{
    const void *first = seed;
    if (!ctx->lists_exact && !seed) {
        SPH_TRY(copy_field(ctx, ctx->hstart, p->h, p->n, s));
        first = ctx->hstart;
    }
    int r = run_once<T>(ctx, p, seed, st, eos, s);
    while (r == SPH_ERR_CAPACITY && lists_escalate(ctx)) r = run_once<T>(ctx, p, first, st, eos, s);
    ctx->lists_pred_skip = false;
    return r;
}

}  // namespace

int density_run(sph_ctx *ctx, sph_particles *p, const void *h_seed, sph_density_stats *st, cudaStream_t s,
                bool eos)
{
    return ctx->fp64 ? run_impl<double>(ctx, p, h_seed, st, eos, s) : run_impl<float>(ctx, p, h_seed, st, eos, s);
}

int eos_run(sph_ctx *ctx, sph_particles *p, const void *u, cudaStream_t s)
{
    const double g = ctx->prm.gamma;
    if (ctx->fp64)
        k_eos<double><<<grid_for(p->n, 256), 256, 0, s>>>((const double *)p->rho, (const double *)u, p->n, g,
                                                          (double *)p->P, (double *)p->c);
    else
        k_eos<float><<<grid_for(p->n, 256), 256, 0, s>>>((const float *)p->rho, (const float *)u, p->n, g,
                                                         (float *)p->P, (float *)p->c);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}
