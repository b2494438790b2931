/*
 * sph.h - C ABI of the GB300 (sm_103a) SPH hydro right-hand side.
 *
 * The library computes, on one GPU, the smoothed-particle-hydrodynamics
 * right-hand side described in Sec. 2.1-2.2.1 of the FleCSPH paper
 * (arXiv 2007.03097):
 *   - Morton (Z-order) keys with a leading 1 bit and a (key, id) sort
 *     (Sec. 2.1, Tree topology; Fig. 1),
 *   - an octree of leaf cells over the sorted particles for neighbour search
 *     within the kernel support 2h (Sec. 2.1, group tree traversal),
 *   - the density sum rho_a = sum_b m_b W(r_ab, h_a) (Eq. 7) solved jointly
 *     with h_a = eta (m_a / rho_a)^(1/3) (Eq. 9, C = 1, D = 3),
 *   - the momentum and internal-energy equations with artificial viscosity
 *     (Eqs. 5-6, g = 0),
 *   - a kick-drift-kick leapfrog step around them.
 * All pointers named "device" must be device memory of the current CUDA
 * device; "host" pointers are ordinary host memory.  Every call is ordered on
 * the CUDA stream passed as `stream` (a cudaStream_t; NULL = legacy default
 * stream).  Calls that fill a host stats struct synchronise that stream.
 *
 * Errors: every int-returning call returns an sph_status; no call aborts or
 * throws.  sph_last_error() gives a message for the last failing call on a
 * context.  On error the contents of output arrays are unspecified, but no
 * call writes outside the arrays it was given.
 *
 * Ownership: the caller owns every particle array.  The context owns all
 * scratch memory, allocated once by sph_create for at most n_max particles;
 * no later call allocates device memory.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = -1,            /* invalid argument or parameter              */
    SPH_ERR_CUDA = -2,           /* a CUDA runtime call failed                 */
    SPH_ERR_CAPACITY = -3,       /* a context capacity would be exceeded       */
    SPH_ERR_NOT_CONVERGED = -4,  /* h-rho iteration hit max_sweeps             */
    SPH_ERR_H_BOUNDS = -5,       /* a converged h sits on h_min or h_max       */
    SPH_ERR_NONFINITE = -6,      /* NaN or Inf in an input array               */
    SPH_ERR_STATE = -7           /* call order violated (e.g. no tree yet)     */
} sph_status;

/* Smoothing kernels, 3D, support radius 2h, q = r/h (the paper offers several
 * kernels without printing them, Sec. 2.1; these are the standard forms). */
typedef enum {
    SPH_KERNEL_M4 = 0,   /* cubic spline, Monaghan 1992                         */
    SPH_KERNEL_WC2 = 1,  /* Wendland C2, Dehnen & Aly 2012                      */
    SPH_KERNEL_WC4 = 2   /* Wendland C4                                          */
} sph_kernel;

/* Arithmetic of the pair sums.
 * SPH_FP64:  every particle field and every pair term in FP64.
 * SPH_MIXED: positions x, y, z stay FP64 (and so do the leapfrog position
 *            update and the conserved totals); every other field is FP32 and
 *            the pair terms are evaluated in FP32 on relative coordinates
 *            formed from a two-float split of the FP64 positions.           */
typedef enum { SPH_FP64 = 0, SPH_MIXED = 1 } sph_precision;

/* Energy equation (Sec. 2.1).
 * SPH_ENERGY_INTERNAL: the specific internal energy u evolves with Eq. 5.
 * SPH_ENERGY_TOTAL:    the thermokinetic formulation (Eq. thermo): the
 *                      specific total energy e = u + v^2/2 evolves with
 *                      de_a/dt = -sum_b m_b (P_a v_b/rho_a^2 + P_b v_a/rho_b^2
 *                      + (v_a + v_b) Pi_ab/2) . grad_a W_ab; the force pass
 *                      writes de_a/dt to dudt, and sph_step advances e and
 *                      recovers u = e - v^2/2 after each kick.             */
typedef enum { SPH_ENERGY_INTERNAL = 0, SPH_ENERGY_TOTAL = 1 } sph_energy;

/* Space-filling curve of the particle keys (Sec. 2.1, Tree topology: both
 * the Morton and the Hilbert curve order the particles).  Either key is
 * 1 << 63 | a 63-bit index of the particle's cell on the 2^21-per-axis grid
 * of the key domain, three bits per octree level, so that the top 3l bits
 * below the leading 1 name the level-l octree cell in both.
 * SPH_CURVE_MORTON:  bits of (ix, iy, iz) interleaved, x lowest in each triple.
 * SPH_CURVE_HILBERT: the Hilbert index of (ix, iy, iz) after J. Skilling,
 *                    "Programming the Hilbert curve", AIP Conf. Proc. 707
 *                    (2004): cell (0, 0, 0) first, consecutive cells face
 *                    neighbours.                                           */
typedef enum { SPH_CURVE_MORTON = 0, SPH_CURVE_HILBERT = 1 } sph_curve;

typedef struct {
    int32_t kernel;      /* sph_kernel                                          */
    int32_t precision;   /* sph_precision                                       */
    int32_t periodic;    /* 1: periodic box [box_lo, box_hi), minimum image     */
    int32_t fixed_h;     /* 1: h is an input; one density evaluation            */
    double box_lo[3];    /* periodic box; must be a cube when periodic          */
    double box_hi[3];
    double gamma;        /* ideal gas: P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u) */
    double eta;          /* h = eta (m/rho)^(1/3)  (Eq. 9 with C = 1, D = 3)    */
    double alpha, beta;  /* Monaghan viscosity coefficients                     */
    double eps_visc;     /* mu_ab = h_ab v_ab.r_ab / (r_ab^2 + eps_visc h_ab^2) */
    double cfl;          /* dt = cfl * min_a h_a / vsig_a                       */
    double h_tol;        /* converged when |h_new - h| < h_tol * h              */
    int32_t max_sweeps;  /* cap on density evaluations per particle (>= 1)      */
    int32_t leaf_size;   /* max particles per octree leaf, 1..32                */
    double h_min, h_max; /* clamp of the h iteration                            */
    double skin;         /* density lists cover 2h (1 + skin); >= 0             */
    double rho_ref;      /* density scale of the h-predictor feature log(h/hbar) */
    int64_t nb_capacity; /* neighbour-list slots to reserve; 0 = 640 n_max.  A
                            build sizes each list by the particles of the leaves
                            within reach and, when those bounds exceed the
                            capacity, by exact counts from then on            */
    double hnet_lr;      /* Adam learning rate of online h-predictor training   */
    int32_t hnet_batch;  /* samples per online training step (strided subset)   */
    int32_t hnet_iters;  /* Adam steps per sph_step when training online        */
    int32_t energy;      /* sph_energy                                          */
    int32_t curve;       /* sph_curve                                           */
    int32_t dim;         /* spatial dimension D, 1 or 3.  D = 1 puts every
                            particle on the x axis (y = z = 0, else
                            SPH_ERR_ARG from the tree build); the kernels take
                            their 1D normalisations and shapes, and Eq. 9
                            reads h = eta (m/rho)^(1/D)                        */
    int32_t pad;         /* 0                                                   */
} sph_params;

/* Particle arrays, structure of arrays, length n, caller-owned DEVICE memory.
 * x, y, z are always double.  Every pointer typed void* points to double in
 * SPH_FP64 and to float in SPH_MIXED.  Arrays must be 16-byte aligned.
 * State (in/out):   x y z vx vy vz m h u hprev id
 * Derived (out):    rho omega(=drho/dh) P c ax ay az dudt divv vsig nnb
 * A NULL derived array is allowed where stated; NULL state arrays are not.
 * id is any set of unique 32-bit labels; sph_build_tree permutes it with the
 * particles so the caller can map results back to its own order.          */
typedef struct {
    int64_t n;                       /* 1 <= n <= n_max (0: SPH_ERR_ARG)         */
    double *x, *y, *z;
    void *vx, *vy, *vz;
    void *m, *h, *u;
    void *hprev;                     /* h of the previous step (h-predictor)     */
    void *rho, *omega, *P, *c;
    void *ax, *ay, *az, *dudt, *divv, *vsig;
    int32_t *nnb;                    /* neighbours b != a with r_ab < 2 h_a      */
    uint32_t *id;
} sph_particles;

typedef struct {
    int32_t sweeps;          /* density evaluations (kernel launches)               */
    int32_t list_builds;     /* neighbour-list constructions                        */
    int64_t n_unconverged;   /* particles that hit max_sweeps                       */
    int64_t n_hbounds;       /* converged particles sitting on h_min / h_max        */
    int64_t interactions;    /* pairs b != a with r_ab < 2 h_a, summed over sweeps  */
    int64_t list_entries;    /* list slots (incl. padding) of the last build        */
    int64_t evaluations;     /* particle density evaluations, summed over sweeps    */
    int64_t launches;        /* kernels launched by the call                        */
    double ms;               /* device time of the call (CUDA events)               */
    double kernel_ms;        /* device time of the density-sum kernels alone        */
    double lists_ms;         /* device time of the call's neighbour-list builds     */
} sph_density_stats;

typedef struct {
    int64_t interactions;    /* pairs b != a with r_ab < h_a + h_b                  */
    int64_t list_entries;
    int64_t launches;        /* kernels launched by the call                        */
    double ms;
    double kernel_ms;        /* device time of the pair-force kernel alone          */
} sph_force_stats;

typedef struct {
    double dt;               /* step used                                           */
    double dt_next;          /* cfl * min h / vsig after the step                   */
    double momentum[3];      /* sum m v (end of step)                               */
    double force[3];         /* sum m a                                             */
    double energy;           /* sum m (v^2/2 + u) (end of step)                     */
    double power;            /* sum m (v_pred . a + du/dt), 0 up to roundoff        */
    int32_t hnet_used;       /* 1 if the h-predictor seeded the iteration           */
    int32_t hnet_fallback;   /* particles reseeded from h after a bad prediction    */
    float hnet_loss;         /* loss of the most recent completed online training
                                round (the round of a step overlaps its force pass) */
    int32_t tree_moved;      /* particles the key-order rebuild moved: 0 when the
                                previous order held, -1 after a full sort          */
    int64_t launches;        /* kernels launched by the step                        */
    sph_density_stats density;
    sph_force_stats forces;
    double ms_tree, ms_hnet, ms_total;
} sph_step_stats;

/* ---- context --------------------------------------------------------------- */

/* Validate *params and allocate every scratch buffer for up to n_max
 * particles on the current device.  On success *out owns them. */
int sph_create(const sph_params *params, int64_t n_max, sph_ctx **out);
void sph_destroy(sph_ctx *ctx);
/* Replace the parameters (same validation; precision and capacity fixed). */
int sph_set_params(sph_ctx *ctx, const sph_params *params);
/* Message of the last failing call on ctx; with ctx == NULL, the message of
 * the calling thread's last failing context-free call (sph_sort_keys_noalloc). */
const char *sph_last_error(const sph_ctx *ctx);
/* Library build string, e.g. "sph sm_103a". */
const char *sph_version(void);

/* ---- hot path ---------------------------------------------------------------- */

/* Sec. 2.1 (Tree topology): Morton keys of the FP64 positions in the cubic
 * key domain (the periodic box, or the bounding cube of an open set), sort of
 * (key, id), in-place permutation of every particle array into key order,
 * octree leaves of at most leaf_size particles and the search hierarchy.
 * Returns SPH_ERR_NONFINITE for NaN/Inf positions or h. */
int sph_build_tree(sph_ctx *ctx, sph_particles *p, void *stream);

/* Eqs. 7 and 9: Newton iteration on h_a until |dh| < h_tol h, then rho and
 * nnb at the final h (rho to first order in dh when that is exact to the
 * arithmetic's rounding, else by one more evaluation) and omega = drho/dh at
 * the last evaluated h (within h_tol h of the final h); P and c from u.  Seeds: h_seed
 * (device, FP64 or FP32 per precision) if not NULL, else the current h.
 * With fixed_h, one evaluation at the given h.  Needs sph_build_tree first. */
int sph_density(sph_ctx *ctx, sph_particles *p, const void *h_seed,
                sph_density_stats *stats, void *stream);

/* Eqs. 5-6 with Monaghan viscosity: a, du/dt, div v (Eq. 2's div v estimate
 * with W(r, h_a)), vsig.  Uses rho, P, c from sph_density. */
int sph_forces(sph_ctx *ctx, sph_particles *p, sph_force_stats *stats, void *stream);

/* One kick-drift-kick step of length dt (dt <= 0: the stored CFL dt):
 * half kick with the stored a, du/dt; FP64 drift and periodic wrap;
 * sph_build_tree; sph_density; forces at v + a dt/2, u + du dt/2; closing
 * half kick; FP64 totals and next CFL dt.  use_hnet is a bit set:
 *   SPH_HNET_SEED  seed the h iteration from the h-predictor (particles whose
 *                  prediction is non-finite or changes h by more than a
 *                  factor 2 keep the current h; if the seeded iteration fails
 *                  to converge it is rerun from the current h),
 *   SPH_HNET_TRAIN after convergence, take hnet_iters Adam steps on the
 *                  step's features and targets log(h_new/h_old) (a strided
 *                  subset of hnet_batch particles).
 * The network's work runs on a second stream owned by the context: the seed
 * beside the tree build (joined before the density iteration), the training
 * round beside the force pass, joined by the next call on the context; until
 * then it reads the particles' h, so a caller that rewrites h between calls
 * trains on the rewritten values (nothing is written outside the context).
 * The particle set must already carry a, du/dt from an earlier force pass.
 * The step's tree build leaves omega, P, c and vsig in the previous order
 * (its density iteration and force pass rewrite them for every particle), so
 * after an error return these four arrays hold no particle's values. */
#define SPH_HNET_SEED 1
#define SPH_HNET_TRAIN 2
int sph_step(sph_ctx *ctx, sph_particles *p, double dt, int use_hnet,
             sph_step_stats *stats, void *stream);

/* FP64 totals of the current arrays: out[0..2] = sum m v, out[3..5] = sum m a,
 * out[6] = sum m (v^2/2 + u), out[7] = sum m (v . a + du/dt).  Host output. */
int sph_totals(sph_ctx *ctx, const sph_particles *p, double out[8], void *stream);

/* ---- stages exposed for verification ------------------------------------------ */

/* Keys of p's current positions on the context's curve (sph_params.curve:
 * Morton or Hilbert) into keys (device, n), and the key domain
 * (lo_x, lo_y, lo_z, L) into dom (host, 4 doubles). */
int sph_morton_keys(sph_ctx *ctx, const sph_particles *p, uint64_t *keys,
                    double dom[4], void *stream);

/* Permutation perm (device, n) with (keys[perm[i]], ids[perm[i]]) ascending. */
int sph_sort_keys(sph_ctx *ctx, int64_t n, const uint64_t *keys, const uint32_t *ids,
                  uint32_t *perm, void *stream);

/* After sph_build_tree: number of leaves and of target groups (host out). */
int sph_tree_info(sph_ctx *ctx, int64_t *n_leaves, int64_t *n_groups);

/* Neighbour-list storage of the last list build, as of the last call that
 * returned (host out, each may be NULL): slots reserved (32 x the per-group
 * widths the build sized), slots holding the exact lists, entries of the
 * per-group source unions the lists index, whether exact sizing is on, the
 * largest union of one group, whether the last build predicted its widths,
 * and how many predicted builds overflowed.
 * A target's list is predicted to hold at most 1.25 n + 16 entries, n its
 * length in the previous build (the lengths follow the particles through
 * every tree build); the first build of a context, and every build after 4
 * predicted builds overflowed, sizes by the particles of the leaves within
 * reach (leaf bounds).  A build that
 * outgrows predicted widths is taken again with leaf bounds; one that
 * outgrows leaf bounds within nb_capacity switches the context to exact
 * counts for the rest of its life.  Results do not depend on the sizing.
 * Implementation detail of the list builder; the paper has no counterpart. */
int sph_list_info(sph_ctx *ctx, int64_t *slots_reserved, int64_t *slots_used, int64_t *union_used,
                  int32_t *exact_sizing, int32_t *union_max, int32_t *predicted,
                  int32_t *pred_failures);

/* After sph_build_tree: leaf_begin (device, n_leaves + 1 entries, the last is
 * n) and level (device, n_leaves; octree level of each leaf cell). */
int sph_export_leaves(sph_ctx *ctx, int32_t *leaf_begin, int32_t *level, void *stream);

/* Exact neighbour sets of the current state, kind 0: b != a with
 * r_ab^2 < 4 h_a^2; kind 1: b != a with r_ab^2 < (h_a + h_b)^2 or
 * r_ab^2 < 4 h_a^2, with r_ab^2 = (dx dx + dy dy) + dz dz in the arithmetic of
 * the precision mode (no fused multiply-add in FP64).  counts (device, n)
 * always; if offsets (device, n + 1) is not NULL the indices (current order)
 * are written to idx (device) at offsets[a] (unsorted within a target). */
int sph_neighbors(sph_ctx *ctx, const sph_particles *p, int kind, int64_t *counts,
                  const int64_t *offsets, uint32_t *idx, void *stream);

/* ---- h-predictor network (not in the paper) --------------------------------------
 * y = W3 silu(W2 silu(W1 f + b1) + b2) + b3, 5 -> 64 -> 64 -> 1.  The
 * context keeps FP32 master weights and the BF16 copy the kernels read.
 * Flat layout (SPH_HNET_NPARAM floats): W1[64][5], b1[64], W2[64][64], b2[64],
 * W3[1][64], b3[1], row-major with the output index first.
 * Features f (FP32, nb x 5, row-major): log(h/hbar) with
 * hbar = eta (m/rho_ref)^(1/3), log(nnb/nbar) with nbar = 32 pi eta^3 / 3,
 * log(rho h^3 / (m eta^3)), div v * dt, log(h/hprev); target
 * log(h_next / h). */
#define SPH_HNET_NPARAM 4609

int sph_hnet_set_weights(sph_ctx *ctx, const float *params_host, int64_t count);
int sph_hnet_get_weights(sph_ctx *ctx, float *params_host, int64_t count);
/* features of the current particles (device, n x 5) for step length dt */
int sph_hnet_features(sph_ctx *ctx, const sph_particles *p, double dt, float *feats,
                      void *stream);
/* predicted log(h_next/h) s = f3 * y (device, nb) from features (device,
 * nb x 5) with the BF16 weights; f3 = div v * dt, so s = 0 at rest.  The
 * 64 x 64 layer runs on the tensor cores (tcgen05, FP32 accumulation of the
 * exact products of the BF16 weights with a three-term BF16 split of the
 * FP32 activations).  Synchronises the stream; SPH_ERR_CUDA if an MMA did
 * not complete within 1 s (the kernel then frees its tensor memory and
 * returns). */
int sph_hnet_infer(sph_ctx *ctx, const float *feats, int64_t nb, float *y, void *stream);
/* the seed of the h iteration that sph_step takes with SPH_HNET_SEED, from
 * the particle fields in one kernel (features, network, exponential):
 * h_seed[a] = h_a exp(s_a) with s_a = f3 y(f_a) where s_a is finite and
 * |s_a| <= ln 2, else h_a (a fallback).  h_seed: device, n entries of the
 * context's float type (double in SPH_FP64, float in SPH_MIXED), caller-owned.
 * *fallbacks (host, may be NULL) = the particles that kept h.  Synchronises
 * the stream; SPH_ERR_CUDA as for sph_hnet_infer. */
int sph_hnet_seed(sph_ctx *ctx, const sph_particles *p, double dt, void *h_seed, int64_t *fallbacks,
                  void *stream);
/* loss = mean (f3 y - t)^2 and its gradient (host, SPH_HNET_NPARAM) at the
 * BF16 weights, FP32 accumulation; no update. */
int sph_hnet_grad(sph_ctx *ctx, const float *feats, const float *target, int64_t nb,
                  float *grad_host, float *loss_host, void *stream);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master weights,
 * then refresh the BF16 copy; loss before the step to *loss_host (may be NULL) */
int sph_hnet_train_step(sph_ctx *ctx, const float *feats, const float *target, int64_t nb,
                        float lr, float *loss_host, void *stream);

/* ---- test hook --------------------------------------------------------------------
 * The paper has no counterpart to this call.  The tensor-core kernels of the
 * h-predictor wait for their MMAs with a bounded wait (1 s), after which they
 * record an error, free their tensor memory and return, and the call returns
 * SPH_ERR_CUDA with the context still usable.  sph_test_hooks lets a test
 * take that path without any GPU fault: with SPH_TEST_SKIP_MMA set, those
 * kernels issue no MMA, so the wait runs out (about 2 s per call: the wait and
 * one more bounded wait for work in flight).  flags = 0 restores normal
 * operation.  SPH_ERR_ARG for a NULL context or an unknown flag. */
#define SPH_TEST_SKIP_MMA 1
int sph_test_hooks(sph_ctx *ctx, int flags);

/* ---- calibration ------------------------------------------------------------------
 * The paper has no counterpart to this call: it measures the hardware the
 * library runs on.  sph_peak_fp32 times independent FP32 fused multiply-add
 * chains (8 per thread, 2048 threads per SM) on the current device, one
 * warm-up launch and the best of five, and writes the rate in TFLOP/s
 * (2 flops per FMA) to *tflops (host) and that launch's duration to *ms
 * (host, may be NULL).  This is the measured ceiling of the pair kernels,
 * which are bound by the FP32 pipe.  Unlike the context calls it allocates
 * (and frees) a small device buffer; it synchronises `stream`.
 * SPH_ERR_ARG if tflops is NULL, SPH_ERR_CUDA if a CUDA call fails. */
int sph_peak_fp32(double *tflops, double *ms, void *stream);

/* ---- allocation-free sort ------------------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory: code running under a framework whose caching
 * allocator owns the device memory budget, plugins that their host forbids to
 * allocate, and latency-critical paths that cannot afford cudaMalloc (which can
 * synchronise the whole device).  Such callers cannot create an sph_ctx.
 *
 * sph_sort_keys_noalloc computes the same permutation as sph_sort_keys
 * ((keys[perm[i]], ids[perm[i]]) ascending; ids may be NULL, then ties keep
 * index order) with no context.  keys (n), ids (n) and perm (n) are caller
 * arrays in device memory of the CURRENT device.  Its scratch is one static
 * device array of about 6.1 MB in the library, present on every device that
 * loads the library until the process exits; the call itself never calls
 * cudaMalloc or cudaFree.
 *   - n must be in [1, SPH_SORT_NOALLOC_MAX]; larger n returns
 *     SPH_ERR_CAPACITY without touching the GPU.  A run of more than 64 equal
 *     keys also returns SPH_ERR_CAPACITY.
 *   - keys, perm (and ids when not NULL) must be device memory of the current
 *     device; otherwise SPH_ERR_ARG, checked before anything is launched.
 *   - Every call looks up the device address of the static array on the
 *     current device (a device reset moves it); the first call on a device
 *     also loads the library's device code there, which can synchronise
 *     that device.
 *   - Every call uses the same scratch and leaves the last call's contents in
 *     it.  Calls that overlap on the GPU (other streams, other threads, same
 *     device) race: serialise them.
 *   - The call synchronises `stream` before returning (it reads a status word).
 *   - On failure sph_last_error(NULL) gives the reason (per calling thread).
 */
#define SPH_SORT_NOALLOC_MAX 262144
int sph_sort_keys_noalloc(int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
