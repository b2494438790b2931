// Internal declarations of the GB300 SPH library: the context, device
// counters, and the small device helpers shared by the kernels (smoothing
// kernels, minimum image, two-float positions).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <climits>
#include <string>

#include "sph.h"

#define SPH_WARP 32
#define SPH_SENTINEL 0xFFFFFFFFu

#define SPH_LOCAL_NONE 0xFFFFu

// Lists are stored in quads: slots 4q .. 4q + 3 of lane l form one 8-byte
// word, quad q of lane l at 64-bit index off / 4 + 32 q + l (off, the group's
// offset in 16-bit slots, is a multiple of 128 and list widths are multiples
// of 4), so that a lane writes four entries with one store and a warp reading
// one quad of every lane reads 256 contiguous bytes.
__device__ __forceinline__ int64_t slot_index(int64_t off, int k, int lane)
{
    return off + 128 * (int64_t)(k >> 2) + 4 * lane + (k & 3);
}

// Sequential reader of one lane's slots: next() returns slots 0, 1, 2, ...
// (SPH_LOCAL_NONE past the width), one 8-byte load per four slots.
struct SlotStream {
    const unsigned long long *q;
    int width, k;
    unsigned long long cur;
    __device__ __forceinline__ SlotStream(const uint16_t *nbl, int64_t off, int width_, int lane)
        : q(reinterpret_cast<const unsigned long long *>(nbl + off) + lane), width(width_), k(0), cur(~0ull)
    {
    }
    __device__ __forceinline__ uint32_t next()
    {
        if ((k & 3) == 0) cur = k < width ? __ldg(q + 32 * (int64_t)(k >> 2)) : ~0ull;
        const uint32_t e = (uint32_t)(cur >> (16 * (k & 3))) & 0xFFFFu;
        ++k;
        return e;
    }
};

// Walks one lane's neighbour list (slots k < width in quads, see above),
// whose 16-bit entries index the group's source union uni[uoff ..]; calls
// proc(b, A[b], B[b]) for every entry's global index b.  PIPELINED: entry
// k + 3, the index of entry k + 2 and the records of entry k + 1 are in
// flight while entry k is processed (an empty slot's records are fetched from
// `self`, a valid index, and never processed).  This pays for the long
// double-float pair arithmetic; the short FP32 one runs faster without it.
template <bool PIPELINED, class Proc>
__device__ __forceinline__ void walk_list(const uint16_t *__restrict__ nbl, int64_t off, int width, int lane,
                                          uint32_t self, const uint32_t *__restrict__ uni, int64_t uoff,
                                          const float4 *__restrict__ A, const float4 *__restrict__ B, Proc &&proc)
{
    const uint32_t *U = uni + uoff;
    SlotStream st(nbl, off, width, lane);
    if (!PIPELINED) {
        for (int k = 0; k < width; ++k) {
            const uint32_t e = st.next();
            if (e == SPH_LOCAL_NONE) continue;
            const uint32_t b = __ldg(U + e);
            proc(b, A[b], B[b]);
        }
        return;
    }
    if (width <= 0) return;
    auto index = [&](uint32_t e) -> uint32_t { return e == SPH_LOCAL_NONE ? SPH_SENTINEL : __ldg(U + e); };
    const uint32_t e0 = st.next(), e1 = st.next();
    uint32_t e2 = st.next();
    uint32_t b0 = index(e0);
    uint32_t b1 = index(e1);
    uint32_t j = b0 == SPH_SENTINEL ? self : b0;
    float4 P = __ldg(A + j), Q = __ldg(B + j);
    for (int k = 0; k < width; ++k) {
        const uint32_t b = b0;
        const float4 Pc = P, Qc = Q;
        b0 = b1;
        b1 = index(e2);
        e2 = st.next();
        j = b0 == SPH_SENTINEL ? self : b0;
        P = __ldg(A + j);
        Q = __ldg(B + j);
        if (b != SPH_SENTINEL) proc(b, Pc, Qc);
    }
}

// bits of DevCounters::err
enum : uint32_t {
    ERRB_NONFINITE = 1u,
    ERRB_LEAF_DEGENERATE = 2u,   // more than leaf_size particles share one key
    ERRB_LIST_CAPACITY = 4u,     // neighbour lists exceed nb_capacity
    ERRB_STACK = 8u,             // traversal stack overflow
    ERRB_TIE_RUN = 16u,          // equal-key run too long to order by id
    ERRB_OFF_AXIS = 32u,         // D = 1 with a particle off the x axis
    ERRB_PREFIX_RUN = 64u,       // a run of equal top key halves too long to order in place
};

// per-particle density iteration flags
enum : int32_t {
    IT_DONE = 1,          // rho, omega, nnb final
    IT_FINAL = 2,         // h converged; next evaluation is the final one
    IT_NOT_CONV = 4,
    IT_H_BOUNDS = 8,
};

// Device-side counters, mirrored into pinned host memory at sync points.
struct DevCounters {
    unsigned long long interactions;   // accepted pairs of the last pass/sweep
    unsigned long long evaluations;    // particle evaluations of the last sweep
    unsigned long long list_total;     // list slots of the last build
    uint32_t err;
    int32_t n_uncovered;               // evaluations skipped: 2h outgrew the list
    int32_t n_not_conv;
    int32_t n_hbounds;
    int32_t n_leaves;
    int32_t n_groups;
    int32_t hnet_fallback;
    double dom[4];                     // key domain lo_x, lo_y, lo_z, L
    double totals[8];                  // conserved totals
    double min_dt;                     // min h / vsig
    float loss;
    int32_t sweeps_done;               // sweeps that evaluated at least one particle
    int32_t act_count[2];              // active groups read / written by the sweeps
    int32_t work[2];                   // next active-group slot a sweep's warps claim
    unsigned long long force_interactions;
    unsigned long long list_used;      // list slots holding the exact lists of the last build
    uint32_t hnet_err;                 // h-predictor tensor-core kernel: an MMA timed out
    uint32_t pad3;
    long long ns_total;                // misplaced keys found by the near-sorted pass
    unsigned long long union_used;     // union slots holding the group unions of the last build
    int32_t sweep_stamp;               // counts density sweeps (group append marks)
    int32_t union_max;                 // largest group source union of the last build
    double unit_ref[2];                // h and m of the first particle in key order (unit choice)
};

// Start-cell table of the neighbour search: levels 1..CELL_LEVELS of the
// key grid, 8^l int32 entries for level l, stored one level after another.
constexpr int CELL_LEVELS = 7;
__host__ __device__ constexpr int64_t cell_table_offset(int l) { return ((int64_t(1) << (3 * l)) - 8) / 7; }
__host__ __device__ constexpr int64_t cell_table_size() { return cell_table_offset(CELL_LEVELS + 1); }

// near-sorted key pass: (key, id) pairs and per-tile extremes, prefix
// maximum, suffix minimum and misplaced counts
struct NsKey {
    uint64_t k;
    uint32_t i;
    uint32_t pad;
};
struct NsTile {
    NsKey mx, mn, pre, suf;
    int32_t cnt, off, pad[2];
};

struct sph_ctx {
    sph_params prm{};
    int64_t n_max = 0;
    int device = 0;
    int num_sms = 0;
    bool fp64 = true;
    std::string err;

    // tree of the current particle order
    int64_t n = 0;
    int64_t n_leaves = 0, n_groups = 0;
    bool tree_valid = false;
    bool lists_valid = false;           // lists cover 2h of every particle
    bool lists_exact = false;           // size lists by exact counts (set once leaf bounds overflowed)
    // Predicted sizing: each target's list is sized from its length in the
    // previous build (lcount: the length in the low 16 bits, the low 16 bits
    // of the particle's id in the high ones; written by every fill, permuted
    // with the particles by every tree build), with no per-target culling in
    // the sizing pass; a group whose id bits do not match is sized by leaf
    // bounds.  A build whose lists outgrow the prediction is taken again
    // with leaf bounds; after PRED_FAIL_MAX such builds the context stops
    // predicting.
    uint32_t *lcount = nullptr;
    bool lcount_valid = false;          // a fill has written lcount for the current particles
    bool lists_pred = false;            // the last build used predicted widths
    bool lists_pred_skip = false;       // the call being retried sizes by leaf bounds
    int lists_pred_fail = 0;
    double dom[4] = {0, 0, 0, 1};
    double dt_cfl = 0.0;
    // Units of the double-float arithmetic (SPH_FP64): lengths are multiplied
    // by len_scale = 2^kL and masses by mass_scale = 2^kM, powers of two chosen
    // at each tree build so that the first particle's h and m lie in [1, 2).
    // The scaling is exact, so results are those of the caller's units; it
    // keeps every intermediate of the pair sums (h^-(D+2), m_b P_b/rho_b^2 ...)
    // inside the FP32 exponent range that double-float numbers share.  SPH_MIXED
    // keeps 1 (its pair sums are FP32 by definition).
    double len_scale = 1.0, mass_scale = 1.0;

    // ---- sort / keys
    uint64_t *key_a = nullptr, *key_b = nullptr;
    uint32_t *val_a = nullptr, *val_b = nullptr;
    uint32_t *hist = nullptr;           // radix histograms, 256 x tiles
    int64_t hist_cap = 0;
    NsTile *ns_tiles = nullptr;         // near-sorted pass, one per 1024 keys
    int64_t ns_moved = -1;              // particles the last build moved (-1: full sort)
    int ns_full_streak = 0;             // consecutive builds that needed the full sort
    int ns_skip = 0;                    // builds left that go straight to the full sort
    // ---- tree
    uint8_t *dlev = nullptr;            // first differing level with predecessor
    uint8_t *plev = nullptr;            // leaf level of each particle
    int32_t *itmp0 = nullptr, *itmp1 = nullptr;   // per-particle int scratch
    int32_t *itmp2 = nullptr, *itmp3 = nullptr;
    int32_t *leaf_begin = nullptr;      // n_leaves + 1
    int32_t *leaf_level = nullptr;
    int32_t *group_begin = nullptr;     // n_groups + 1
    float4 *leaf_lo = nullptr, *leaf_hi = nullptr;   // box; .w of lo = max coverage
    int32_t *node_child = nullptr;      // 2 per internal node; leaf = idx | 1<<31
    int32_t *node_parent = nullptr;     // internal nodes
    int32_t *leaf_parent = nullptr;
    uint32_t *node_visit = nullptr;
    int32_t *node_delta = nullptr;      // leading key bits shared by an internal node's leaves
    int32_t *cell_table = nullptr;      // start cells of the neighbour search (cell_table_offset)
    int pow2_shift = -1;                // the key grid by shifts (>= 0) or by FP64 scaling
    int infer_per_sm = 1;               // resident blocks per SM of the seed inference
    float4 *node_lo = nullptr, *node_hi = nullptr;   // .w of lo = max coverage
    float4 *group_lo = nullptr, *group_hi = nullptr; // .w of lo = max coverage
    // ---- two-float split of the positions (padded)
    // packed per-particle sources of the pair kernels (two-float pairs):
    // A {x, y}, B {z, m}, C {vx, vy}, D {vz, h}, E {rho, P/rho^2}, F {c, -}
    float4 *srcA = nullptr, *srcB = nullptr, *srcC = nullptr, *srcD = nullptr, *srcE = nullptr, *srcF = nullptr;
    // ---- neighbour lists (group slabs, slot-major within a group)
    // lists: per group a union of its source particles (global indices) and
    // per-lane lists of 16-bit local indices into it
    uint16_t *nbl = nullptr;
    int64_t nbl_cap = 0;
    int32_t *group_width = nullptr;
    int64_t *group_off = nullptr;       // n_groups + 1
    uint32_t *uni = nullptr;            // union slots
    float4 *urec = nullptr;             // SPH_MIXED: per union slot {x, y, z relative to the group-box
                                        // centre (nearest image), m}, as the sweeps stage them
    int64_t uni_cap = 0;
    int32_t *group_ubound = nullptr;    // union slots sized per group
    int64_t *union_off = nullptr;       // n_groups + 1
    int32_t *group_union = nullptr;     // union size per group
    int32_t *group_img = nullptr;       // 1: a list candidate of the group lies across a periodic face
    int32_t *group_mark = nullptr;      // sweep stamp of a group's last append to the active list
    int2 *kept = nullptr;               // leaves kept by the list sizing pass, per group: {first particle, count}
    int32_t *kept_count = nullptr;
    int64_t kept_cap = 0;
    // ---- density iteration state
    double *it_lo = nullptr, *it_hi = nullptr;
    int32_t *it_flags = nullptr;
    int32_t *it_sweeps = nullptr;
    float *cov = nullptr;               // coverage radius of each particle's list
    int32_t *act_groups[2] = {nullptr, nullptr};
    // ---- force pass / step scratch (precision-typed, 8 bytes per entry)
    void *vpx = nullptr, *vpy = nullptr, *vpz = nullptr, *upred = nullptr;
    void *hold = nullptr;               // h before the density iteration
    void *hstart = nullptr;             // first guess of the running iteration (for a restart)
    void *hseed = nullptr;              // h-predictor seeds
    // ---- gather scratch
    unsigned char *gbuf = nullptr;
    size_t gbuf_bytes = 0;
    // ---- scans and reductions
    void *scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    double *red = nullptr;              // block partials of reductions
    int red_blocks = 0;
    // ---- counters
    DevCounters *dcnt = nullptr;        // device
    DevCounters *hcnt = nullptr;        // pinned host mirror
    // ---- h-predictor network
    float *hn_master = nullptr;         // FP32 master weights
    __nv_bfloat16 *hn_bf16 = nullptr;   // copy read by the kernels
    float *hn_m = nullptr, *hn_v = nullptr;  // Adam moments
    float *hn_grad = nullptr;           // reduced gradient
    float *hn_part = nullptr;           // per-block partial gradients
    int hn_part_blocks = 0;
    int64_t hn_step = 0;
    float *hn_sample = nullptr;         // hnet_batch x 6 (features, target)
    // ---- timing and launch accounting
    cudaEvent_t ev[8] = {};
    // the online training of a step runs on a side stream, overlapping the
    // force pass; the next call on the context waits for it
    cudaStream_t side = nullptr;
    cudaEvent_t ev_dens = nullptr, ev_train = nullptr;
    cudaEvent_t ev_order = nullptr, ev_seed = nullptr;   // particles in key order; h seed written (side stream)
    bool side_pending = false;
    cudaEvent_t kev[2 * 64] = {};       // per-sweep density kernel events
    cudaEvent_t lev[4] = {};            // list builds of the density iteration (first, rebuild)
    int64_t launches = 0;               // kernels launched so far
    int32_t lists_union_max = INT32_MAX; // largest union of the current lists, when a synchronisation has told
    int test_flags = 0;                 // sph_test_hooks
    int64_t force_launches = 0;         // kernels of the last force pass
};

// ------------------------------------------------------------------ helpers
#define SPH_CUDA(call)                                                             \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return SPH_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)

#define SPH_CHECK_LAUNCH()                                                         \
    do {                                                                           \
        ++ctx->launches;                                                           \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess) {                                                   \
            ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e_);    \
            return SPH_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)

#define SPH_TRY(expr)                                                              \
    do {                                                                           \
        int s_ = (expr);                                                           \
        if (s_ != SPH_OK) return s_;                                               \
    } while (0)

static inline int sph_fail(sph_ctx *ctx, int code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

static inline unsigned grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

// ---------------------------------------------------- smoothing kernel math
// W(r, h) = sigma / h^D w(q), q = r / h, support q < 2 (the same published
// forms as the oracle, evaluated here in Horner form).  A kernel shape is the
// kernel id in three dimensions and the id + 3 in one (kern_shape):
//   0 M4    (D = 3, sigma 1/pi;  D = 1 as shape 3, sigma 2/3):
//           w = 1 - 3/2 q^2 + 3/4 q^3 (q < 1),  (2 - q)^3 / 4 (1 <= q < 2)
//   1 WC2   D = 3, sigma 21/(16 pi):  w = s^4 (1 + 2q),             s = 1 - q/2
//   2 WC4   D = 3, sigma 495/(256 pi): w = s^6 (1 + 3q + 35/12 q^2)
//   4 WC2   D = 1, sigma 5/8:          w = s^3 (1 + 3q/2)
//   5 WC4   D = 1, sigma 3/4:          w = s^5 (1 + 5q/2 + 2 q^2)
// (the Wendland functions of Dehnen & Aly 2012 for each dimension, support
// 2h).  kern_wdw returns w(q) and dw/dq.
#define SPH_PI 3.14159265358979323846
__host__ __device__ __forceinline__ int kern_shape(int kernel, int dim) { return kernel + (dim == 1 ? 3 : 0); }

template <typename T>
__host__ __device__ __forceinline__ T kern_sigma(int shape)
{
    switch (shape) {
    case 0: return T(1.0 / SPH_PI);
    case 1: return T(21.0 / (16.0 * SPH_PI));
    case 2: return T(495.0 / (256.0 * SPH_PI));
    case 3: return T(2.0 / 3.0);
    case 4: return T(5.0 / 8.0);
    default: return T(3.0 / 4.0);
    }
}

template <typename T>
__device__ __forceinline__ void kern_wdw(int k, T q, T &w, T &dw)
{
    if (k == 1) {
        T s = T(1) - T(0.5) * q;
        T s2 = s * s;
        T s3 = s2 * s;
        w = s3 * s * (T(1) + T(2) * q);
        dw = T(-5) * q * s3;
    } else if (k == 2) {
        T s = T(1) - T(0.5) * q;
        T s2 = s * s;
        T s5 = s2 * s2 * s;
        w = s5 * s * (T(1) + q * (T(3) + q * T(35.0 / 12.0)));
        dw = T(-14.0 / 3.0) * q * (T(1) + T(2.5) * q) * s5;
    } else if (k == 0 || k == 3) {
        if (q < T(1)) {
            w = T(1) + q * q * (T(-1.5) + T(0.75) * q);
            dw = q * (T(-3) + T(2.25) * q);
        } else {
            T t = T(2) - q;
            w = T(0.25) * t * t * t;
            dw = T(-0.75) * t * t;
        }
    } else if (k == 4) {
        T s = T(1) - T(0.5) * q;
        T s2 = s * s;
        w = s2 * s * (T(1) + T(1.5) * q);
        dw = T(-3) * q * s2;
    } else {
        T s = T(1) - T(0.5) * q;
        T s2 = s * s;
        T s4 = s2 * s2;
        w = s4 * s * (T(1) + q * (T(2.5) + T(2) * q));
        dw = T(-3.5) * q * (T(1) + T(2) * q) * s4;
    }
}

// w(q) and g(q) = D w(q) + q w'(q) of kernel shape k (D its dimension), the
// two terms of the density sum and of its h derivative, each as a power of
// s = 1 - q/2 times a short polynomial (the same functions as kern_wdw,
// expanded):
//   WC2 3D  w = s^3 s (1 + 2q)                 g = s^3 (3 + 9/2 q - 8 q^2)
//   WC4 3D  w = s^5 (1 + 5/2 q + 17/12 q^2 - 35/24 q^3)
//           g = s^5 (3 + 15/2 q - 5/12 q^2 - 385/24 q^3)
//   WC2 1D  w = s^2 (1 + q - 3/4 q^2)          g = s^2 (1 + q - 15/4 q^2)
//   WC4 1D  w = s^4 (1 + 2q + 3/4 q^2 - q^3)   g = s^4 (1 + 2q - 11/4 q^2 - 8 q^3)
//   M4      q < 1: g = D - 3 (D + 2)/2 q^2 + 3 (D + 3)/4 q^3;
//           q >= 1 (t = 2 - q): 3D g = 3/2 t^2 (1 - q), 1D g = t^2 (1 - 2q)/2
template <typename T>
__device__ __forceinline__ void kern_wg(int k, T q, T &w, T &g)
{
    const T s = T(1) - T(0.5) * q;
    if (k == 1) {
        const T s3 = s * s * s;
        w = s3 * (s * (T(1) + T(2) * q));
        g = s3 * (T(3) + q * (T(4.5) - T(8) * q));
    } else if (k == 2) {
        const T s2 = s * s;
        const T s5 = s2 * s2 * s;
        w = s5 * (T(1) + q * (T(2.5) + q * (T(17.0 / 12.0) - T(35.0 / 24.0) * q)));
        g = s5 * (T(3) + q * (T(7.5) - q * (T(5.0 / 12.0) + T(385.0 / 24.0) * q)));
    } else if (k == 0 || k == 3) {
        if (q < T(1)) {
            w = T(1) + q * q * (T(-1.5) + T(0.75) * q);
            g = k == 0 ? T(3) + q * q * (T(-7.5) + T(4.5) * q) : T(1) + q * q * (T(-4.5) + T(3) * q);
        } else {
            const T t = T(2) - q;
            w = T(0.25) * t * t * t;
            g = k == 0 ? T(1.5) * t * t * (T(1) - q) : T(0.5) * t * t * (T(1) - T(2) * q);
        }
    } else if (k == 4) {
        const T s2 = s * s;
        w = s2 * (T(1) + q * (T(1) - T(0.75) * q));
        g = s2 * (T(1) + q * (T(1) - T(3.75) * q));
    } else {
        const T s2 = s * s;
        const T s4 = s2 * s2;
        w = s4 * (T(1) + q * (T(2) + q * (T(0.75) - q)));
        g = s4 * (T(1) + q * (T(2) - q * (T(2.75) + T(8) * q)));
    }
}

// w'(q) / q of kernel shape k: the Wendland forms and the inner piece of M4
// are polynomials in q; the outer piece of M4 takes 1/q from the caller
// (qinv), which only that shape reads.  The gradient is then
// grad_a W(r, h) = sigma / h^(D+2) (w'(q)/q) r_ab, with no 1/r.
template <typename T>
__device__ __forceinline__ T kern_dwq(int k, T q, T qinv)
{
    const T s = T(1) - T(0.5) * q;
    if (k == 1) return T(-5) * (s * s * s);
    if (k == 2) {
        const T s2 = s * s;
        return T(-14.0 / 3.0) * (T(1) + T(2.5) * q) * (s2 * s2 * s);
    }
    if (k == 0 || k == 3) {
        if (q < T(1)) return T(-3) + T(2.25) * q;
        const T t = T(2) - q;
        return T(-0.75) * t * t * qinv;
    }
    if (k == 4) return T(-3) * (s * s);
    const T s2 = s * s;
    return T(-3.5) * (T(1) + T(2) * q) * (s2 * s2);
}

// 1 / h^D from 1 / h (D = 1 or 3)
template <typename T>
__device__ __forceinline__ T inv_pow_dim(T hinv, int dim) { return dim == 1 ? hinv : hinv * hinv * hinv; }

// Minimum-image separation, FP64 without contraction (bit-identical to the
// plain expression xa - xb; if > L/2 subtract L; if < -L/2 add L).
__device__ __forceinline__ double sep_d(double xa, double xb, int periodic, double L, double half)
{
    double d = __dsub_rn(xa, xb);
    if (periodic) {
        if (d > half) d = __dsub_rn(d, L);
        else if (d < -half) d = __dadd_rn(d, L);
    }
    return d;
}

// r^2 = (dx dx + dy dy) + dz dz in FP64 without fused multiply-add
__device__ __forceinline__ double r2_d(double dx, double dy, double dz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// FP32 separation (ha + la) - (hb + lb) of two-float positions to the
// nearest periodic image.  The difference of the high parts is exact for
// nearby points (to half an ulp of the separation); for an image pair it is
// near +-L and rounded to half an ulp of L, which would swamp a separation of
// a few smoothing lengths, so its rounding error is recovered by two-sum and
// the shift by L, exact by Sterbenz's lemma, comes first.  wrap: the image
// taken (-1: L subtracted, +1: L added, 0: none).
__device__ __forceinline__ float sep_fw(float ha, float la, float hb, float lb, int periodic, float L,
                                        float half, int &wrap)
{
    float d = ha - hb;
    wrap = 0;
    if (periodic && fabsf(d) > half) {
        const float bb = d - ha;
        const float err = (ha - (d - bb)) + (-hb - bb);
        wrap = d > 0.f ? -1 : 1;
        d = (d + (float)wrap * L) + err;
    }
    return d + (la - lb);
}

__device__ __forceinline__ float sep_f(float ha, float la, float hb, float lb, int periodic,
                                       float L, float half)
{
    int w;
    return sep_fw(ha, la, hb, lb, periodic, L, half, w);
}

// a - c (FP32, |a - c| < L + half) to the nearest periodic image, with the
// rounding error of an image pair's raw difference recovered as in sep_fw.
__device__ __forceinline__ float wrap_diff(float a, float c, float L, float invL)
{
    float d = a - c;
    const float k = rintf(d * invL);
    if (k != 0.f) {
        const float bb = d - a;
        const float err = (a - (d - bb)) + (-c - bb);
        d = (d - k * L) + err;
    }
    return d;
}

// 16-byte global -> shared copy without a register round trip (cp.async;
// both addresses 16-byte aligned), and the wait for all of a thread's copies
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ------------------------------------------------------------ launchers
// tree.cu
// after_order (may be null) is called with the build's stream as soon as
// the particle fields exist in their final key order, before the leaves are
// built (a second time in the rare build that sorts again on all key bits).
// view holds them: the caller's arrays, or the tree build's scratch copy
// that the full sort gathers into and copies back from (unchanged until the
// next tree build; fields the build does not permute keep the caller's
// pointers).
// derived = false leaves omega, P, c and vsig unpermuted: for a caller that
// rewrites all four for every particle before reading them (sph_step).
// join(s) makes s wait for the work the hook queued elsewhere (before the
// build overwrites its scratch copy again).
struct OrderHook {
    virtual int operator()(cudaStream_t s, const sph_particles *view) = 0;
    virtual int join(cudaStream_t) { return SPH_OK; }
};
int tree_build(sph_ctx *ctx, sph_particles *p, cudaStream_t s, OrderHook *after_order = nullptr,
               bool derived = true);
int tree_keys(sph_ctx *ctx, const sph_particles *p, uint64_t *keys_out, cudaStream_t s);
int tree_sort(sph_ctx *ctx, int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm,
              cudaStream_t s);
int tree_boxes(sph_ctx *ctx, cudaStream_t s);
// scan.cu
int scan_exclusive_i32(sph_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
int scan_exclusive_i64(sph_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
int scan_inclusive_max_i32(sph_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s);
size_t scan_tmp_bytes(int64_t n);
// neighbors.cu
int lists_build(sph_ctx *ctx, const sph_particles *p, cudaStream_t s);

constexpr int PRED_FAIL_MAX = 4;

// After a list-capacity error: choose the safer sizing for the call's retry
// (leaf bounds after a prediction, exact counts after leaf bounds).  False
// when the lists were already sized exactly, so the error stands.
inline bool lists_escalate(sph_ctx *ctx)
{
    if (ctx->lists_pred) {
        ++ctx->lists_pred_fail;
        ctx->lists_pred_skip = true;
    } else if (!ctx->lists_exact) {
        ctx->lists_exact = true;
    } else {
        return false;
    }
    ctx->lists_pred = false;
    ctx->lists_valid = false;
    ctx->err.clear();
    return true;
}
// device copy of n elements of the context's precision
int copy_field(sph_ctx *ctx, void *dst, const void *src, int64_t n, cudaStream_t s);
// order stream s (or the host, for s == nullptr with host = true) after the
// pending side-stream training of the previous step
int join_side(sph_ctx *ctx, cudaStream_t s, bool host = false);
int neighbors_export(sph_ctx *ctx, const sph_particles *p, int kind, int64_t *counts,
                     const int64_t *offsets, uint32_t *idx, cudaStream_t s);
// density.cu
int density_run(sph_ctx *ctx, sph_particles *p, const void *h_seed, sph_density_stats *st, cudaStream_t s,
                bool eos = true);
int eos_run(sph_ctx *ctx, sph_particles *p, const void *u, cudaStream_t s);
// forces.cu
int forces_run(sph_ctx *ctx, sph_particles *p, const void *vx, const void *vy, const void *vz, const void *u,
               sph_force_stats *st, bool reuse_lists, cudaStream_t s);
// after a sync_counters that follows a forces_run with st == nullptr
int forces_collect(sph_ctx *ctx, sph_force_stats *st);
// integrate.cu
int kick_drift(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s);
int predict(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s);
int kick(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s);
int totals_run(sph_ctx *ctx, const sph_particles *p, const void *vx, const void *vy,
               const void *vz, const void *u, cudaStream_t s);
int sync_counters(sph_ctx *ctx, cudaStream_t s);
// hnet.cu
int hnet_init(sph_ctx *ctx);
int hnet_features(sph_ctx *ctx, const sph_particles *p, double dt, float *feats, cudaStream_t s);
int hnet_infer(sph_ctx *ctx, const float *feats, int64_t nb, float *y, cudaStream_t s);
int hnet_grad(sph_ctx *ctx, const float *feats, const float *target, int64_t nb, cudaStream_t s);
int hnet_adam(sph_ctx *ctx, float lr, cudaStream_t s);
int hnet_seed_from_fields(sph_ctx *ctx, const sph_particles *p, double dt, bool train, void *h_seed,
                          cudaStream_t s);
int hnet_sample_features(sph_ctx *ctx, const sph_particles *p, double dt, cudaStream_t s);
int hnet_online(sph_ctx *ctx, const sph_particles *p, cudaStream_t s);
