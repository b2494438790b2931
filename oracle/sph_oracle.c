/*
 * Plain FP64 CPU oracle for the SPH hydro right-hand side of the FleCSPH
 * paper (arXiv 2007.03097).  TEST INFRASTRUCTURE ONLY: it is called by the
 * tests, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py,
 * never by the product path.  It shares no code, header or table with the
 * CUDA library.
 *
 * Everything is brute force: every target particle is tested against every
 * source particle, in FP64, with loops written in the order the equations
 * are printed.  Compiled with -ffp-contract=off so no multiply-add is fused.
 *
 * Paper passages followed (section / equation numbers of the paper):
 *   Eq. 1  (Sec. 1)      SPH interpolant, volume element m_b / rho_b
 *   Eq. 5  (Sec. 2.2.1)  du_a/dt = sum_b m_b (P_a/rho_a^2 + Pi_ab/2) v_ab . grad_a W_ab
 *   Eq. 6  (Sec. 2.2.1)  dv_a/dt = -sum_b m_b (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) grad_a W_ab
 *                        with W_ab = W(|r_a - r_b|, h_ab), h_ab = (h_a + h_b)/2
 *   Eq. 7  (Sec. 2.2.1)  rho_a = sum_b m_b W_ab (density reconstructed, not evolved)
 *   Eq. 9  (Sec. 2.2.1)  h_a = C eta (m_a/rho_a)^(1/D), D = 1 or 3
 *   Sec. 2.1 (Tree topology): Morton (Z-order) and Hilbert keys with a
 *                        leading 1 digit, unique particle ids to resolve
 *                        equal keys.
 * Readings where the paper is silent (kernels, viscosity, iteration) are
 * stated at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* kernel ids */
enum { ORC_M4 = 0, ORC_WC2 = 1, ORC_WC4 = 2 };

/* per-particle density flags */
enum { ORC_DONE = 1, ORC_NOT_CONVERGED = 2, ORC_H_BOUNDS = 4 };

typedef struct {
    int kernel;        /* ORC_M4 / ORC_WC2 / ORC_WC4                     */
    int periodic;      /* 1: periodic box, minimum image                  */
    double box_lo[3];  /* periodic box [lo, hi)                           */
    double box_hi[3];
    double gamma;      /* ideal-gas adiabatic index                       */
    double eta;        /* h = eta (m/rho)^(1/3)                            */
    double alpha, beta, eps_visc; /* Monaghan viscosity                   */
    int fixed_h;       /* 1: h is an input, one density evaluation         */
    double h_tol;      /* |dh|/h convergence threshold                     */
    int max_sweeps;    /* cap on density evaluations per particle          */
    double h_min, h_max;
    int dim;           /* spatial dimension D: 1 (particles on the x axis) or 3 */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Smoothing kernels.  The paper lists several kernels (Sec. 2.1, Physics
 * Functionalities) without printing any; the three used here are the
 * standard published forms with support radius 2h, q = r/h, s = 1 - q/2:
 *   M4 cubic spline (Monaghan 1992), the same w in every dimension:
 *       w = 1 - 3/2 q^2 + 3/4 q^3 (q<1),  1/4 (2-q)^3 (1<=q<2);
 *       sigma = 1/pi (D = 3), 2/3 (D = 1)
 *   Wendland C2 (Dehnen & Aly 2012):  D = 3: sigma = 21/(16 pi), w = s^4 (1+2q)
 *                                     D = 1: sigma = 5/8,        w = s^3 (1+3q/2)
 *   Wendland C4:                      D = 3: sigma = 495/(256 pi),
 *                                            w = s^6 (1 + 3q + 35/12 q^2)
 *                                     D = 1: sigma = 3/4, w = s^5 (1 + 5q/2 + 2q^2)
 * (the 1D Wendland functions are (1-x)^3 (1+3x) and (1-x)^5 (1+5x+8x^2) of
 * x = r/(2h)).  W(r,h) = sigma/h^D w(q).  Derivatives by differentiating
 * these by hand:
 *   dW/dr = sigma/h^(D+1) w'(q),  dW/dh = -sigma/h^(D+1) (D w(q) + q w'(q)). */

static double kern_sigma(int k, int dim)
{
    if (dim == 1) {
        if (k == ORC_M4) return 2.0 / 3.0;
        if (k == ORC_WC2) return 5.0 / 8.0;
        return 3.0 / 4.0;
    }
    if (k == ORC_M4) return 1.0 / ORC_PI;
    if (k == ORC_WC2) return 21.0 / (16.0 * ORC_PI);
    return 495.0 / (256.0 * ORC_PI);
}

static double kern_w(int k, int dim, double q)
{
    if (q >= 2.0) return 0.0;
    if (k == ORC_M4) {
        if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
        double t = 2.0 - q;
        return 0.25 * t * t * t;
    }
    double s = 1.0 - 0.5 * q;
    if (dim == 1) {
        if (k == ORC_WC2) return s * s * s * (1.0 + 1.5 * q);
        return s * s * s * s * s * (1.0 + 2.5 * q + 2.0 * q * q);
    }
    if (k == ORC_WC2) {
        double s2 = s * s;
        return s2 * s2 * (1.0 + 2.0 * q);
    }
    double s2 = s * s;
    return s2 * s2 * s2 * (1.0 + 3.0 * q + (35.0 / 12.0) * q * q);
}

/* derivative of w with respect to q */
static double kern_dw(int k, int dim, double q)
{
    if (q >= 2.0) return 0.0;
    if (k == ORC_M4) {
        if (q < 1.0) return -3.0 * q + 2.25 * q * q;
        double t = 2.0 - q;
        return -0.75 * t * t;
    }
    double s = 1.0 - 0.5 * q;
    if (dim == 1) {
        if (k == ORC_WC2) {
            /* d/dq [s^3 (1 + 3q/2)] = -3/2 s^2 (1 + 3q/2) + 3/2 s^3 = -3 q s^2 */
            return -3.0 * q * s * s;
        }
        /* d/dq [s^5 P] = s^4 (-5/2 P + s P'),  P = 1 + 5q/2 + 2 q^2 */
        double P = 1.0 + 2.5 * q + 2.0 * q * q;
        double dP = 2.5 + 4.0 * q;
        return s * s * s * s * (-2.5 * P + s * dP);
    }
    if (k == ORC_WC2) {
        /* d/dq [s^4 (1+2q)] = -2 s^3 (1+2q) + 2 s^4 = -5 q s^3 */
        return -5.0 * q * s * s * s;
    }
    /* d/dq [s^6 P] = s^5 (-3 P + s P'),  P = 1 + 3q + 35/12 q^2 */
    double P = 1.0 + 3.0 * q + (35.0 / 12.0) * q * q;
    double dP = 3.0 + (35.0 / 6.0) * q;
    double s5 = s * s * s * s * s;
    return s5 * (-3.0 * P + s * dP);
}

/* h^D for D = 1 or 3 */
static double pow_dim(double h, int dim) { return dim == 1 ? h : h * h * h; }

double orc_W(int k, int dim, double r, double h)
{
    double q = r / h;
    return kern_sigma(k, dim) / pow_dim(h, dim) * kern_w(k, dim, q);
}

double orc_dWdr(int k, int dim, double r, double h)
{
    double q = r / h;
    return kern_sigma(k, dim) / (pow_dim(h, dim) * h) * kern_dw(k, dim, q);
}

double orc_dWdh(int k, int dim, double r, double h)
{
    double q = r / h;
    return -kern_sigma(k, dim) / (pow_dim(h, dim) * h) * (dim * kern_w(k, dim, q) + q * kern_dw(k, dim, q));
}

/* vectorised wrappers for the tests */
void orc_kernel_eval(int k, int dim, int64_t n, const double *r, const double *h,
                     double *W, double *dWdr, double *dWdh)
{
    for (int64_t i = 0; i < n; ++i) {
        if (W) W[i] = orc_W(k, dim, r[i], h[i]);
        if (dWdr) dWdr[i] = orc_dWdr(k, dim, r[i], h[i]);
        if (dWdh) dWdh[i] = orc_dWdh(k, dim, r[i], h[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Separation r_a - r_b.  Periodic box: one minimum-image shift per axis
 * (reading: supports never exceed half the box, so one image suffices).
 * r2 is summed as (dx*dx + dy*dy) + dz*dz.                                  */
static inline double sep(const orc_params *p, int d, double xa, double xb)
{
    double dx = xa - xb;
    if (p->periodic) {
        double L = p->box_hi[d] - p->box_lo[d];
        double half = 0.5 * L;
        if (dx > half) dx -= L;
        else if (dx < -half) dx += L;
    }
    return dx;
}

/* ------------------------------------------------------------------------ */
/* Morton keys (Sec. 2.1, Tree topology; Fig. 1 keys carry a leading 1).
 * Cell index per axis: i = floor((x - lo) * (2^21 / L)), clamped to
 * [0, 2^21 - 1].  Key = 1 << 63 | bits of (ix, iy, iz) interleaved one bit at
 * a time, x in the lowest bit of each triple.  Written as a bit loop.       */
void orc_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                     const double lo[3], double L, uint64_t *keys)
{
    const double scale = 2097152.0 / L;
    for (int64_t i = 0; i < n; ++i) {
        const double c[3] = {x[i], y[i], z[i]};
        uint64_t cell[3];
        for (int d = 0; d < 3; ++d) {
            double t = (c[d] - lo[d]) * scale;
            double f = floor(t);
            if (!(f >= 0.0)) f = 0.0;
            if (f > 2097151.0) f = 2097151.0;
            cell[d] = (uint64_t)f;
        }
        uint64_t key = 0;
        for (int b = 0; b < 21; ++b)
            for (int d = 0; d < 3; ++d)
                key |= ((cell[d] >> b) & 1ull) << (3 * b + d);
        keys[i] = key | (1ull << 63);
    }
}

/* Hilbert keys (Sec. 2.1, Tree topology names the Hilbert curve beside
 * Morton's).  Index of a cell (X[0], X[1], X[2]) of `bits` bits per axis
 * after J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707
 * (2004), in the steps of that method:
 *   1. for Q = 2^(bits-1) down to 2, with P = Q - 1, and for each axis i in
 *      turn: if bit Q of X[i] is set, invert the bits P of X[0]; otherwise
 *      exchange the bits P of X[0] and X[i];
 *   2. Gray-encode the axes: X[i] ^= X[i-1] for i = 1, 2;
 *   3. t = XOR of (Q - 1) over the bits Q >= 2 set in X[2]; X[i] ^= t;
 *   4. the index takes, from the top bit down, the bits of X[0], X[1], X[2]
 *      in that order.
 * Keys use the Morton cells and the leading 1.                            */
uint64_t orc_hilbert_index(uint32_t ix, uint32_t iy, uint32_t iz, int bits)
{
    uint32_t X[3] = {ix, iy, iz};
    for (uint32_t Q = 1u << (bits - 1); Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = 1u << (bits - 1); Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t h = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
    return h;
}

void orc_hilbert_index_many(int64_t n, const uint32_t *ix, const uint32_t *iy, const uint32_t *iz, int bits,
                            uint64_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_hilbert_index(ix[i], iy[i], iz[i], bits);
}

void orc_hilbert_keys(int64_t n, const double *x, const double *y, const double *z,
                      const double lo[3], double L, uint64_t *keys)
{
    const double scale = 2097152.0 / L;
    for (int64_t i = 0; i < n; ++i) {
        const double c[3] = {x[i], y[i], z[i]};
        uint32_t cell[3];
        for (int d = 0; d < 3; ++d) {
            double f = floor((c[d] - lo[d]) * scale);
            if (!(f >= 0.0)) f = 0.0;
            if (f > 2097151.0) f = 2097151.0;
            cell[d] = (uint32_t)f;
        }
        keys[i] = orc_hilbert_index(cell[0], cell[1], cell[2], 21) | (1ull << 63);
    }
}

/* Permutation sorting (key, id) ascending; ids are unique so the order is
 * unique (Sec. 2.1 gives every particle a unique id for this purpose).    */
typedef struct { uint64_t key; uint32_t id; uint32_t pos; } kip;

static int kip_cmp(const void *a, const void *b)
{
    const kip *u = (const kip *)a, *v = (const kip *)b;
    if (u->key != v->key) return u->key < v->key ? -1 : 1;
    if (u->id != v->id) return u->id < v->id ? -1 : 1;
    return 0;
}

void orc_sort_perm(int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm)
{
    kip *a = (kip *)malloc(sizeof(kip) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].key = keys[i]; a[i].id = ids[i]; a[i].pos = (uint32_t)i; }
    qsort(a, (size_t)n, sizeof(kip), kip_cmp);
    for (int64_t i = 0; i < n; ++i) perm[i] = a[i].pos;
    free(a);
}

/* ------------------------------------------------------------------------ */
/* Density sum Eq. 7 at a trial h for target a, gather form W(r_ab, h_a)
 * (reading: the fixed point of Eq. 9 is then one scalar equation per
 * particle).  Self term included in rho; neighbour count excludes it.
 * b is a neighbour iff r2 < 4 h^2, evaluated as (4*h)*h.                   */
static void density_sum(const orc_params *p, int64_t n, const double *x, const double *y,
                        const double *z, const double *m, int64_t a, double h,
                        double *rho, double *drho_dh, int32_t *nnb)
{
    const double thr = 4.0 * h * h;
    double r_sum = 0.0, d_sum = 0.0;
    int32_t cnt = 0;
    for (int64_t b = 0; b < n; ++b) {
        double dx = sep(p, 0, x[a], x[b]);
        double dy = sep(p, 1, y[a], y[b]);
        double dz = sep(p, 2, z[a], z[b]);
        double r2 = (dx * dx + dy * dy) + dz * dz;
        if (!(r2 < thr)) continue;
        double r = sqrt(r2);
        r_sum += m[b] * orc_W(p->kernel, p->dim, r, h);
        d_sum += m[b] * orc_dWdh(p->kernel, p->dim, r, h);
        if (b != a) ++cnt;
    }
    *rho = r_sum;
    *drho_dh = d_sum;
    *nnb = cnt;
}

/* h-rho fixed point of Eq. 9 with C = 1: h = eta (m/rho)^(1/D), D = 1 or 3.
 * The paper does not say how the fixed point is solved; reading: Newton on
 *   f(h)  = m eta^D / h^D - rho(h),   f'(h) = -D m eta^D / h^(D+1) - drho/dh,
 * one density evaluation per sweep, with a bracket [lo, hi] of evaluated
 * smoothing lengths kept from the sign of f (f > 0 means the root lies above
 * h; the bracket starts as [0, inf)).  A Newton step outside the closed
 * interval [max(lo, h/2), min(hi, 2h)] or with f' >= 0 is replaced by the
 * midpoint
 * between h and the nearer admissible end in the direction the sign of f
 * points.  The result is clamped to [h_min, h_max].  When |h_new - h| <
 * h_tol * h the step is applied and one more evaluation at the final h gives
 * the returned rho, drho/dh and count.  If max_sweeps evaluations pass first,
 * the particle keeps its last evaluated h and is flagged NOT_CONVERGED.  A
 * converged h sitting on h_min or h_max is flagged H_BOUNDS.               */
int orc_density(const orc_params *p, int64_t n, const double *x, const double *y,
                const double *z, const double *m, const double *h_seed,
                int64_t nt, const int64_t *targets,
                double *h_out, double *rho_out, double *drho_out, int32_t *nnb_out,
                int32_t *sweeps_out, int32_t *flags_out, int64_t *pairs_out)
{
    const double etaD = p->dim == 1 ? p->eta : p->eta * p->eta * p->eta;   /* eta^D */
    int worst = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : worst)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t a = targets ? targets[t] : t;
        double h = h_seed[a];
        double lo = 0.0, hi = INFINITY;  /* evaluated bracket ends */
        double rho = 0.0, drho = 0.0;
        int32_t cnt = 0, sweeps = 0, flags = 0, final_eval = p->fixed_h ? 1 : 0;
        int64_t pairs = 0;   /* neighbour pairs over all evaluations */
        for (;;) {
            density_sum(p, n, x, y, z, m, a, h, &rho, &drho, &cnt);
            ++sweeps;
            pairs += cnt;
            if (final_eval) { flags |= ORC_DONE; break; }
            double ma = m[a];
            double f = ma * etaD / pow_dim(h, p->dim) - rho;
            if (f == 0.0) { flags |= ORC_DONE; break; }
            if (sweeps >= p->max_sweeps) { flags |= ORC_NOT_CONVERGED; break; }
            double fp = -p->dim * ma * etaD / (pow_dim(h, p->dim) * h) - drho;
            if (f > 0.0) { if (h > lo) lo = h; }
            else { if (h < hi) hi = h; }
            double a_lo = 0.5 * h > lo ? 0.5 * h : lo;
            double a_hi = 2.0 * h < hi ? 2.0 * h : hi;
            double hn = 0.0;
            int newton_ok = 0;
            if (fp < 0.0) {
                hn = h - f / fp;
                newton_ok = (hn >= a_lo) && (hn <= a_hi);
            }
            if (!newton_ok) hn = f > 0.0 ? 0.5 * (h + a_hi) : 0.5 * (h + a_lo);
            if (hn < p->h_min) hn = p->h_min;
            if (hn > p->h_max) hn = p->h_max;
            int conv = fabs(hn - h) < p->h_tol * h;
            h = hn;
            if (conv) final_eval = 1;
        }
        if ((flags & ORC_DONE) && !p->fixed_h && (h <= p->h_min || h >= p->h_max))
            flags |= ORC_H_BOUNDS;
        h_out[a] = h;
        rho_out[a] = rho;
        if (drho_out) drho_out[a] = drho;
        if (nnb_out) nnb_out[a] = cnt;
        if (sweeps_out) sweeps_out[a] = sweeps;
        if (flags_out) flags_out[a] = flags;
        if (pairs_out) pairs_out[a] = pairs;
        worst |= flags & (ORC_NOT_CONVERGED | ORC_H_BOUNDS);
    }
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Neighbour sets by definition, for parity of the GPU neighbour search.
 * kind 0 (density): b != a with r2 < (4*h_a)*h_a.
 * kind 1 (force):   b != a with r2 < (h_a+h_b)^2 or r2 < (4*h_a)*h_a
 *                   (the force pass also needs the h_a support for div v).
 * Output: counts[t] for each target; if idx != NULL, the sorted source
 * indices are written at offsets[t] (caller-computed exclusive scan).      */
void orc_neighbors(const orc_params *p, int kind, int64_t n, const double *x, const double *y,
                   const double *z, const double *h, int64_t nt, const int64_t *targets,
                   int64_t *counts, const int64_t *offsets, int64_t *idx)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t a = targets ? targets[t] : t;
        const double thr_a = 4.0 * h[a] * h[a];
        int64_t c = 0;
        for (int64_t b = 0; b < n; ++b) {
            if (b == a) continue;
            double dx = sep(p, 0, x[a], x[b]);
            double dy = sep(p, 1, y[a], y[b]);
            double dz = sep(p, 2, z[a], z[b]);
            double r2 = (dx * dx + dy * dy) + dz * dz;
            int in = r2 < thr_a;
            if (kind == 1) {
                double hs = h[a] + h[b];
                in = in || (r2 < hs * hs);
            }
            if (!in) continue;
            if (idx) idx[offsets[t] + c] = b;
            ++c;
        }
        counts[t] = c;
    }
}

/* ------------------------------------------------------------------------ */
/* Ideal-gas EOS (Sec. 2.1 lists several equations of state; the workloads
 * use the ideal gas): P = (gamma - 1) rho u,  c = sqrt(gamma (gamma - 1) u). */
void orc_eos(int64_t n, double gamma, const double *rho, const double *u, double *P, double *c)
{
    for (int64_t i = 0; i < n; ++i) {
        P[i] = (gamma - 1.0) * rho[i] * u[i];
        c[i] = sqrt(gamma * (gamma - 1.0) * u[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Momentum and internal-energy equations, Eqs. 5-6, g = 0.
 * Pair set: b != a with r_ab < h_a + h_b (W_ab uses h_ab = (h_a+h_b)/2 and
 * vanishes beyond 2 h_ab).  grad_a W_ab = dW/dr(r_ab, h_ab) r_ab / r_ab.
 * Artificial viscosity: the paper cites the standard prescription
 * (Monaghan 1992) without printing it; reading:
 *   mu_ab = h_ab (v_ab . r_ab) / (r_ab^2 + eps h_ab^2),
 *   Pi_ab = (-alpha cbar_ab mu_ab + beta mu_ab^2) / rhobar_ab  if v_ab . r_ab < 0,
 *   Pi_ab = 0 otherwise;  cbar, rhobar are pair means.
 * Also returned:
 *   divv_a = -(1/rho_a) sum_{r_ab < 2 h_a} m_b v_ab . grad_a W(r_ab, h_a)
 *            (the SPH estimate of div v that Eq. 2 relates to drho/dt),
 *   vsig_a = max_b (c_a + c_b - 3 min(0, v_ab . r_ab / r_ab)), c_a if no pair,
 *   S_a    = sum_b m_b |P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab| |grad_a W_ab|,
 *   S_u    = sum_b m_b |P_a/rho_a^2 + Pi_ab/2| |v_ab . grad_a W_ab|,
 * the last two being the cancellation scales used to normalise errors.
 * npairs_out receives the number of (a, b) pairs with r_ab < h_a + h_b.   */
void orc_forces(const orc_params *p, int64_t n, const double *x, const double *y,
                const double *z, const double *vx, const double *vy, const double *vz,
                const double *m, const double *h, const double *rho, const double *P,
                const double *c, int64_t nt, const int64_t *targets,
                double *ax, double *ay, double *az, double *dudt, double *divv,
                double *vsig, double *S_a, double *S_u, int64_t *npairs_out)
{
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t a = targets ? targets[t] : t;
        const double Pa_r2 = P[a] / (rho[a] * rho[a]);
        const double thr_a = 4.0 * h[a] * h[a];
        double acc[3] = {0.0, 0.0, 0.0};
        double du = 0.0, dv = 0.0, vs = c[a], sa = 0.0, su = 0.0;
        for (int64_t b = 0; b < n; ++b) {
            if (b == a) continue;
            double dx = sep(p, 0, x[a], x[b]);
            double dy = sep(p, 1, y[a], y[b]);
            double dz = sep(p, 2, z[a], z[b]);
            double r2 = (dx * dx + dy * dy) + dz * dz;
            double hs = h[a] + h[b];
            int in_f = r2 < hs * hs;
            int in_d = r2 < thr_a;
            if (!in_f && !in_d) continue;
            double r = sqrt(r2);
            double vabx = vx[a] - vx[b], vaby = vy[a] - vy[b], vabz = vz[a] - vz[b];
            double vdotr = (vabx * dx + vaby * dy) + vabz * dz;
            if (in_d) {
                /* v_ab . grad_a W(r, h_a) */
                dv += m[b] * orc_dWdr(p->kernel, p->dim, r, h[a]) / r * vdotr;
            }
            if (!in_f) continue;
            ++pairs;
            double hab = 0.5 * hs;
            double g = orc_dWdr(p->kernel, p->dim, r, hab) / r;
            double gx = g * dx, gy = g * dy, gz = g * dz;
            double Pi = 0.0;
            if (vdotr < 0.0) {
                double mu = hab * vdotr / (r2 + p->eps_visc * hab * hab);
                double cbar = 0.5 * (c[a] + c[b]);
                double rbar = 0.5 * (rho[a] + rho[b]);
                Pi = (-p->alpha * cbar * mu + p->beta * mu * mu) / rbar;
            }
            double coef = Pa_r2 + P[b] / (rho[b] * rho[b]) + Pi;
            acc[0] -= m[b] * coef * gx;
            acc[1] -= m[b] * coef * gy;
            acc[2] -= m[b] * coef * gz;
            double vdotg = (vabx * gx + vaby * gy) + vabz * gz;
            double ecoef = Pa_r2 + 0.5 * Pi;
            du += m[b] * ecoef * vdotg;
            double vr = vdotr / r;
            double sig = c[a] + c[b] - 3.0 * (vr < 0.0 ? vr : 0.0);
            if (sig > vs) vs = sig;
            sa += m[b] * fabs(coef) * sqrt((gx * gx + gy * gy) + gz * gz);
            su += m[b] * fabs(ecoef) * fabs(vdotg);
        }
        ax[a] = acc[0];
        ay[a] = acc[1];
        az[a] = acc[2];
        dudt[a] = du;
        if (divv) divv[a] = -dv / rho[a];
        if (vsig) vsig[a] = vs;
        if (S_a) S_a[a] = sa;
        if (S_u) S_u[a] = su;
    }
    if (npairs_out) *npairs_out = pairs;
}

/* ------------------------------------------------------------------------ */
/* Thermokinetic energy equation (Sec. 2.1, Eq. thermo, after Rosswog 2015):
 * the specific total energy e_a = u_a + v_a^2 / 2 evolves with
 *   de_a/dt = - sum_b m_b ( P_a v_b / rho_a^2 + P_b v_a / rho_b^2
 *                          + (v_a + v_b) Pi_ab / 2 ) . grad_a W_ab,
 * over the same pairs, with the same W_ab = W(r_ab, h_ab) and Pi_ab as
 * orc_forces.  S_e receives the cancellation scale
 *   sum_b m_b ( |P_a/rho_a^2| |v_b . g| + |P_b/rho_b^2| |v_a . g|
 *               + |Pi_ab| |(v_a + v_b)/2 . g| ),  g = grad_a W_ab.        */
void orc_energy_rate(const orc_params *p, int64_t n, const double *x, const double *y,
                     const double *z, const double *vx, const double *vy, const double *vz,
                     const double *m, const double *h, const double *rho, const double *P,
                     const double *c, int64_t nt, const int64_t *targets, double *dedt, double *S_e)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int64_t a = targets ? targets[t] : t;
        const double Pa_r2 = P[a] / (rho[a] * rho[a]);
        double de = 0.0, se = 0.0;
        for (int64_t b = 0; b < n; ++b) {
            if (b == a) continue;
            double dx = sep(p, 0, x[a], x[b]);
            double dy = sep(p, 1, y[a], y[b]);
            double dz = sep(p, 2, z[a], z[b]);
            double r2 = (dx * dx + dy * dy) + dz * dz;
            double hs = h[a] + h[b];
            if (!(r2 < hs * hs)) continue;
            double r = sqrt(r2);
            double hab = 0.5 * hs;
            double g = orc_dWdr(p->kernel, p->dim, r, hab) / r;
            double gx = g * dx, gy = g * dy, gz = g * dz;
            double vabx = vx[a] - vx[b], vaby = vy[a] - vy[b], vabz = vz[a] - vz[b];
            double vdotr = (vabx * dx + vaby * dy) + vabz * dz;
            double Pi = 0.0;
            if (vdotr < 0.0) {
                double mu = hab * vdotr / (r2 + p->eps_visc * hab * hab);
                double cbar = 0.5 * (c[a] + c[b]);
                double rbar = 0.5 * (rho[a] + rho[b]);
                Pi = (-p->alpha * cbar * mu + p->beta * mu * mu) / rbar;
            }
            double Pb_r2 = P[b] / (rho[b] * rho[b]);
            double vb_g = (vx[b] * gx + vy[b] * gy) + vz[b] * gz;
            double va_g = (vx[a] * gx + vy[a] * gy) + vz[a] * gz;
            double vm_g = 0.5 * (va_g + vb_g);
            de -= m[b] * ((Pa_r2 * vb_g + Pb_r2 * va_g) + Pi * vm_g);
            se += m[b] * ((fabs(Pa_r2) * fabs(vb_g) + fabs(Pb_r2) * fabs(va_g)) + fabs(Pi) * fabs(vm_g));
        }
        dedt[a] = de;
        if (S_e) S_e[a] = se;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
