// Tree build (Sec. 2.1, Tree topology): Morton or Hilbert keys with a
// leading 1 bit, LSD radix sort of (key, index) with equal keys ordered by
// particle id, in-place permutation of every particle array into key order,
// octree leaf cells of at most leaf_size particles, target groups of at most
// 32 particles, and a binary radix tree over the leaves (Karras 2012) with
// bounding boxes and maximal coverage radius for pruning the neighbour search.
//
// The paper builds a hashed octree by inserting particles one by one and
// refining nodes.  Here the octree is implicit in the sorted keys: a leaf is
// the shallowest key-prefix cell holding at most leaf_size particles, found
// per particle from the levels at which neighbouring keys first differ.
#include <cfloat>
#include <cmath>

#include <algorithm>

#include "sph_internal.cuh"

namespace {

// ------------------------------------------------------------------ domain
__global__ void k_bbox_partial(const double *__restrict__ x, const double *__restrict__ y,
                               const double *__restrict__ z, int64_t n, double *part)
{
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double c[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) { mn[d] = fmin(mn[d], c[d]); mx[d] = fmax(mx[d], c[d]); }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    }
    __shared__ double s[32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) { s[warp][d] = mn[d]; s[warp][3 + d] = mx[d]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[0][threadIdx.x];
        for (int w = 1; w < nw; ++w)
            v = threadIdx.x < 3 ? fmin(v, s[w][threadIdx.x]) : fmax(v, s[w][threadIdx.x]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

// Key domain: periodic box, or lo = bounding-box minimum and
// L = (largest extent) * (1 + 2^-20) for an open set.
__global__ void k_domain(const double *part, int nparts, int periodic, double blx, double bly,
                         double blz, double boxL, DevCounters *cnt)
{
    if (threadIdx.x != 0) return;
    if (periodic) {
        cnt->dom[0] = blx; cnt->dom[1] = bly; cnt->dom[2] = blz; cnt->dom[3] = boxL;
        return;
    }
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int b = 0; b < nparts; ++b)
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], part[b * 6 + d]);
            mx[d] = fmax(mx[d], part[b * 6 + 3 + d]);
        }
    double ext = fmax(fmax(__dsub_rn(mx[0], mn[0]), __dsub_rn(mx[1], mn[1])), __dsub_rn(mx[2], mn[2]));
    double L = __dmul_rn(ext, 1.0 + 0x1p-20);
    if (!(L > 0.0)) L = 1.0;
    cnt->dom[0] = mn[0]; cnt->dom[1] = mn[1]; cnt->dom[2] = mn[2]; cnt->dom[3] = L;
}

// ------------------------------------------------------------------ keys
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Hilbert index of cell (x, y, z), 21 bits per axis, after J. Skilling,
// "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004).  From the top
// level down, each axis that has the level's bit set reflects the lower bits
// of x, and each that has it clear swaps its lower bits with those of x; the
// axes are then Gray-coded (y ^= x, z ^= y) and every axis is XOR-ed with
// the mask whose bit j is the parity of the bits of z above j.  The index
// interleaves the three words, x highest in each triple.  Written with
// select masks so that the warp does not diverge.
__device__ __forceinline__ uint64_t hilbert3(uint32_t x, uint32_t y, uint32_t z)
{
#pragma unroll
    for (int lev = 20; lev >= 1; --lev) {
        const uint32_t P = (1u << lev) - 1u;
        const uint32_t sx = 0u - ((x >> lev) & 1u), sy = 0u - ((y >> lev) & 1u), sz = 0u - ((z >> lev) & 1u);
        x ^= P & sx;                                   // x against itself: reflect or nothing
        uint32_t t = (x ^ y) & P & ~sy;                // y: swap with x where clear
        x ^= (P & sy) ^ t;
        y ^= t;
        t = (x ^ z) & P & ~sz;                         // z: the same
        x ^= (P & sz) ^ t;
        z ^= t;
    }
    y ^= x;
    z ^= y;
    uint32_t s = z;                                    // s_j = parity of z's bits at j and above
    s ^= s >> 1;
    s ^= s >> 2;
    s ^= s >> 4;
    s ^= s >> 8;
    s ^= s >> 16;
    const uint32_t t = s >> 1;                         // parity of the bits above j
    x ^= t;
    y ^= t;
    z ^= t;
    return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}

__device__ __forceinline__ uint64_t cell_of(double c, double lo, double scale)
{
    double f = floor(__dmul_rn(__dsub_rn(c, lo), scale));
    if (!(f >= 0.0)) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    return (uint64_t)f;
}

// floor(c 2^sh) clamped to [0, 2^21 - 1] from the bits of c (a box with its
// low corner at 0 and a power-of-two side, sh = 21 - log2 L): c 2^sh is then
// exact and cell_of's FP64 arithmetic reduces to a shift of the significand.
// Same cells as cell_of(c, 0, 2^sh) for every finite c.
__device__ __forceinline__ uint64_t cell_pow2(double c, int sh)
{
    const uint64_t b = (uint64_t)__double_as_longlong(c);
    if (b >> 63) return 0;                              // negative: the lowest cell
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0) return 0;                               // zero or subnormal
    const int p = e - 1023 + sh;                        // c 2^sh = 1.f x 2^p
    if (p < 0) return 0;
    if (p >= 21) return 2097151;                        // beyond the grid (or not finite)
    return (((b & ((1ull << 52) - 1)) | (1ull << 52)) >> (52 - p));
}

__device__ __forceinline__ bool finite_bits(double v)
{
    return (((uint64_t)__double_as_longlong(v) >> 52) & 0x7FF) != 0x7FF;
}

// the 21-bit cell coordinates of a point on the key grid (the same cells
// for the keys and for the start-cell table of the neighbour search)
__device__ __forceinline__ void grid_cell(double xi, double yi, double zi, int pow2_shift, const DevCounters *cnt,
                                          uint64_t &cx, uint64_t &cy, uint64_t &cz)
{
    if (pow2_shift >= 0) {
        cx = cell_pow2(xi, pow2_shift);
        cy = cell_pow2(yi, pow2_shift);
        cz = cell_pow2(zi, pow2_shift);
    } else {
        const double lx = cnt->dom[0], ly = cnt->dom[1], lz = cnt->dom[2];
        const double scale = 2097152.0 / cnt->dom[3];
        cx = cell_of(xi, lx, scale);
        cy = cell_of(yi, ly, scale);
        cz = cell_of(zi, lz, scale);
    }
}

template <typename T>
__global__ void k_keys(const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, const T *__restrict__ h,
                       const T *__restrict__ m, int64_t n, int curve, int dim, int pow2_shift, DevCounters *cnt,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xi = x[i], yi = y[i], zi = z[i];
    bool ok = finite_bits(xi) && finite_bits(yi) && finite_bits(zi);
    if (h) ok = ok && isfinite(h[i]) && h[i] > T(0);
    if (m) ok = ok && isfinite(m[i]);
    if (!ok) atomicOr(&cnt->err, ERRB_NONFINITE);
    if (dim == 1 && (yi != 0.0 || zi != 0.0)) atomicOr(&cnt->err, ERRB_OFF_AXIS);
    uint64_t cx, cy, cz;
    grid_cell(xi, yi, zi, pow2_shift, cnt, cx, cy, cz);
    const uint64_t key = (curve == SPH_CURVE_HILBERT ? hilbert3((uint32_t)cx, (uint32_t)cy, (uint32_t)cz)
                                                     : spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2)) |
                         (1ull << 63);
    keys[i] = key;
    if (vals) vals[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096 keys per tile
constexpr int RS_BINS = 256;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ keys, int64_t n,
                                                        int shift, uint32_t *__restrict__ hist,
                                                        int ntiles)
{
    __shared__ uint32_t hs[RS_BINS];
    hs[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&hs[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hs[threadIdx.x];
}

// Stable scatter: elements keep their input order within a digit.  Each
// warp ranks its own 512 consecutive keys of the tile (16 rounds of 32:
// __match_any_sync within a round, a warp-private digit counter across
// rounds), one block-wide pass turns the per-warp counts into offsets, the
// tile is reordered by digit in shared memory and then written out with
// consecutive threads on consecutive destinations (runs of ~16 keys per
// digit).  The per-tile digit counts are differences of the scanned offsets
// (digit-major layout: the entry after (d, t) is (d, t + 1), or (d + 1, 0)
// for the last tile).
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_PER_WARP = RS_TILE / RS_WARPS;      // 512 keys, 16 per lane
constexpr size_t RS_SCATTER_SMEM = (size_t)RS_TILE * (8 + 4) + sizeof(uint32_t) * RS_BINS * (RS_WARPS + 2);

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin,
                                                           uint64_t *__restrict__ kout,
                                                           uint32_t *__restrict__ vout, int64_t n,
                                                           int shift, const uint32_t *__restrict__ hist,
                                                           int ntiles)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    uint64_t *skey = (uint64_t *)rs_smem;                                   // RS_TILE keys
    uint32_t *sval = (uint32_t *)(skey + RS_TILE);                          // RS_TILE values
    uint32_t (*wc)[RS_BINS] = (uint32_t (*)[RS_BINS])(sval + RS_TILE);     // per-warp digit counts
    uint32_t *loff = &wc[RS_WARPS][0];                                      // tile-local digit offsets
    uint32_t *gofs = loff + RS_BINS;                                        // global digit offsets
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    const int64_t base = (int64_t)b * RS_TILE;
    const int tile_n = n - base < RS_TILE ? (int)(n - base) : RS_TILE;
    gofs[tid] = hist[(int64_t)tid * ntiles + b];
#pragma unroll
    for (int q = 0; q < RS_BINS / 32; ++q) wc[warp][q * 32 + lane] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[RS_ROUNDS];
    uint32_t val[RS_ROUNDS], rk[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int t = warp * RS_PER_WARP + r * 32 + lane;
        const bool valid = t < tile_n;
        key[r] = valid ? kin[base + t] : 0ull;
        val[r] = valid ? vin[base + t] : 0u;
        const uint32_t digit = valid ? (uint32_t)((key[r] >> shift) & 0xff) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int leader = __ffs(peers) - 1;
        uint32_t prev = 0;
        if (valid && lane == leader) {
            prev = wc[warp][digit];
            wc[warp][digit] = prev + __popc(peers);
        }
        rk[r] = __shfl_sync(0xffffffffu, prev, leader) + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // digit tid: offsets of the warps within the tile's run of that digit,
    // then the tile-local start of each digit (exclusive scan of the totals)
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = wc[w][tid];
        wc[w][tid] = tot;
        tot += c;
    }
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) loff[warp] = inc;                  // scratch for the warp totals
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += loff[w];
    __syncthreads();
    loff[tid] = before + inc - tot;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int t = warp * RS_PER_WARP + r * 32 + lane;
        if (t < tile_n) {
            const uint32_t digit = (uint32_t)((key[r] >> shift) & 0xff);
            const uint32_t lp = loff[digit] + wc[warp][digit] + rk[r];
            skey[lp] = key[r];
            sval[lp] = val[r];
        }
    }
    __syncthreads();
    // the tile in digit order: position j of digit d goes to gofs[d] + j - loff[d]
    for (int t = tid; t < tile_n; t += RS_THREADS) {
        const uint64_t k = skey[t];
        const uint32_t d = (uint32_t)((k >> shift) & 0xff);
        const uint32_t pos = gofs[d] + (uint32_t)t - loff[d];
        kout[pos] = k;
        vout[pos] = sval[t];
    }
}

// Runs of equal keys are ordered by particle id (Sec. 2.1: ids resolve
// equal keys).  Runs are tiny in practice; longer than 64 is flagged.
__global__ void k_fix_ties(const uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                           const uint32_t *__restrict__ ids, int64_t n, DevCounters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    if (i > 0 && keys[i - 1] == k) return;
    if (i + 1 >= n || keys[i + 1] != k) return;
    int64_t e = i + 1;
    while (e < n && keys[e] == k && e - i <= 64) ++e;
    if (e - i > 64) { atomicOr(&cnt->err, ERRB_TIE_RUN); return; }
    for (int64_t a = i + 1; a < e; ++a) {
        uint32_t v = vals[a];
        uint32_t idv = ids ? ids[v] : v;
        int64_t b = a - 1;
        while (b >= i && (ids ? ids[vals[b]] : vals[b]) > idv) { vals[b + 1] = vals[b]; --b; }
        vals[b + 1] = v;
    }
}

// After a sort on the top 32 key bits only (the tree build), runs of equal
// top halves are put in (key, id) order, which completes the order of the
// full sort.  Such runs hold particles closer than 2^-10 of the key domain
// and are tiny in practice; one longer than 64 is left alone and flagged,
// and the build then sorts on all bits.  Threads inside a run read only
// keys with the run's top half, so the reordering cannot move a run start.
constexpr int PREFIX_RUN_MAX = 64;
__global__ void k_fix_prefix_runs(uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                  const uint32_t *__restrict__ ids, int64_t n, DevCounters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t top = (uint32_t)(keys[i] >> 32);
    if (i > 0 && (uint32_t)(keys[i - 1] >> 32) == top) return;
    if (i + 1 >= n || (uint32_t)(keys[i + 1] >> 32) != top) return;
    int64_t e = i + 1;
    while (e < n && (uint32_t)(keys[e] >> 32) == top && e - i <= PREFIX_RUN_MAX) ++e;
    if (e - i > PREFIX_RUN_MAX) { atomicOr(&cnt->err, ERRB_PREFIX_RUN); return; }
    for (int64_t a = i + 1; a < e; ++a) {          // insertion sort on (key, id)
        const uint64_t k = keys[a];
        const uint32_t v = vals[a], idv = ids[v];
        int64_t b = a - 1;
        while (b >= i && (keys[b] > k || (keys[b] == k && ids[vals[b]] > idv))) {
            keys[b + 1] = keys[b];
            vals[b + 1] = vals[b];
            --b;
        }
        keys[b + 1] = k;
        vals[b + 1] = v;
    }
}

// ------------------------------------------------------------------ gather
constexpr int MAX_FIELDS = 24;
struct FieldTable {
    const void *src[MAX_FIELDS];
    void *dst[MAX_FIELDS];
    int size[MAX_FIELDS];
    int nf;
};

// Permute every field: dst_f[i] = src_f[perm[i]] into scratch.
__global__ void k_gather(FieldTable t, const uint32_t *__restrict__ perm, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t p = perm[i];
    for (int f = 0; f < t.nf; ++f) {
        if (t.size[f] == 8) ((double *)t.dst[f])[i] = ((const double *)t.src[f])[p];
        else ((uint32_t *)t.dst[f])[i] = ((const uint32_t *)t.src[f])[p];
    }
}

// two-float split v = hi + lo of a value given in double
__device__ __forceinline__ float2 split2(double v)
{
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// packed pair-kernel sources: {xh, xl, yh, yl} and {zh, zl, m_hi, m_lo} of
// the positions times ls and the masses times ms (powers of two: exact;
// SCALED false: ls = ms = 1, as in mixed mode, without the FP64 multiplies)
template <typename T, bool SCALED>
__global__ void k_pack_pos(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                           const T *__restrict__ m, int64_t n, double ls, double ms, float4 *__restrict__ A,
                           float4 *__restrict__ B)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 sx = split2(SCALED ? x[i] * ls : x[i]), sy = split2(SCALED ? y[i] * ls : y[i]),
                 sz = split2(SCALED ? z[i] * ls : z[i]), sm = split2(SCALED ? (double)m[i] * ms : (double)m[i]);
    A[i] = make_float4(sx.x, sx.y, sy.x, sy.y);
    B[i] = make_float4(sz.x, sz.y, sm.x, sm.y);
}

__global__ void k_copy_back(FieldTable t, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int f = 0; f < t.nf; ++f) {
        if (t.size[f] == 8) ((double *)t.src[f])[i] = ((const double *)t.dst[f])[i];
        else ((uint32_t *)t.src[f])[i] = ((const uint32_t *)t.dst[f])[i];
    }
}

// ------------------------------------------------------------------ near-sorted keys
// Between steps the particles stay in the previous key order and move little,
// so most of the new (key, id) sequence is already in its final order.  An
// element is in place iff every element before it is smaller and every one
// after it is larger: its rank is its position.  The misplaced elements
// occupy the remaining positions in ascending order, so it suffices to rank
// them among themselves (brute force; they are few) and to move only them.
// The result is the (key, id) order of the full sort.
using KI = NsKey;
__device__ __forceinline__ bool ki_lt(const KI &a, const KI &b) { return a.k < b.k || (a.k == b.k && a.i < b.i); }
__device__ __forceinline__ KI ki_max(const KI &a, const KI &b) { return ki_lt(a, b) ? b : a; }
__device__ __forceinline__ KI ki_min(const KI &a, const KI &b) { return ki_lt(a, b) ? a : b; }
__device__ __forceinline__ KI ki_shfl_xor(const KI &a, int o)
{
    KI r;
    r.k = __shfl_xor_sync(0xffffffffu, a.k, o);
    r.i = __shfl_xor_sync(0xffffffffu, a.i, o);
    r.pad = 0;
    return r;
}
__device__ __forceinline__ KI ki_shfl_up(const KI &a, int o)
{
    KI r;
    r.k = __shfl_up_sync(0xffffffffu, a.k, o);
    r.i = __shfl_up_sync(0xffffffffu, a.i, o);
    r.pad = 0;
    return r;
}
__device__ __forceinline__ KI ki_shfl_down(const KI &a, int o)
{
    KI r;
    r.k = __shfl_down_sync(0xffffffffu, a.k, o);
    r.i = __shfl_down_sync(0xffffffffu, a.i, o);
    r.pad = 0;
    return r;
}
__device__ __forceinline__ KI ki_low() { return KI{0ull, 0u, 0u}; }          // keys carry bit 63
__device__ __forceinline__ KI ki_high() { return KI{~0ull, ~0u, 0u}; }

constexpr int NS_THREADS = 256, NS_PER = 4, NS_TILE = NS_THREADS * NS_PER;
constexpr int64_t NS_LIMIT = 32768;   // misplaced elements ranked by brute force at most

// per tile: maximum and minimum element
__global__ void __launch_bounds__(NS_THREADS) k_ns_tiles(const uint64_t *__restrict__ keys,
                                                         const uint32_t *__restrict__ ids, int64_t n,
                                                         NsTile *__restrict__ t)
{
    __shared__ KI smx[NS_THREADS / 32], smn[NS_THREADS / 32];
    const int64_t b0 = (int64_t)blockIdx.x * NS_TILE + NS_PER * threadIdx.x;
    KI mx = ki_low(), mn = ki_high();
#pragma unroll
    for (int u = 0; u < NS_PER; ++u) {
        const int64_t i = b0 + u;
        if (i < n) {
            const KI e{keys[i], ids[i], 0u};
            mx = ki_max(mx, e);
            mn = ki_min(mn, e);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = ki_max(mx, ki_shfl_xor(mx, o));
        mn = ki_min(mn, ki_shfl_xor(mn, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { smx[w] = mx; smn[w] = mn; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < NS_THREADS / 32; ++k) { mx = ki_max(mx, smx[k]); mn = ki_min(mn, smn[k]); }
        t[blockIdx.x].mx = mx;
        t[blockIdx.x].mn = mn;
    }
}

// Block-wide exclusive scan of one KI per thread, with max from the left
// (DIR = +1) or min from the right (DIR = -1); blockDim.x a multiple of 32,
// at most 1024; sh holds 64 entries.
template <int DIR>
__device__ KI ki_block_exscan(KI v, KI ident, KI *sh)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    KI x = v;                                    // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const KI y = DIR > 0 ? ki_shfl_up(x, o) : ki_shfl_down(x, o);
        const bool take = DIR > 0 ? lane >= o : lane + o < 32;
        if (take) x = DIR > 0 ? ki_max(x, y) : ki_min(x, y);
    }
    if (DIR > 0 ? lane == 31 : lane == 0) sh[w] = x;
    __syncthreads();
    if (w == 0) {                                // inclusive scan over the warps
        KI c = lane < nw ? sh[lane] : ident;
        for (int o = 1; o < 32; o <<= 1) {
            const KI y = DIR > 0 ? ki_shfl_up(c, o) : ki_shfl_down(c, o);
            const bool take = DIR > 0 ? lane >= o : lane + o < 32;
            if (take) c = DIR > 0 ? ki_max(c, y) : ki_min(c, y);
        }
        sh[32 + lane] = c;
    }
    __syncthreads();
    KI before = ident;                           // the warps ahead in the scan direction
    if (DIR > 0 && w > 0) before = sh[32 + w - 1];
    if (DIR < 0 && w < nw - 1) before = sh[32 + w + 1];
    KI ex = DIR > 0 ? ki_shfl_up(x, 1) : ki_shfl_down(x, 1);
    if (DIR > 0 ? lane == 0 : lane == 31) ex = ident;
    __syncthreads();                             // sh free for the next call
    return DIR > 0 ? ki_max(before, ex) : ki_min(before, ex);
}

// exclusive prefix maximum and suffix minimum over the tiles (one block)
__global__ void __launch_bounds__(1024) k_ns_prefix(NsTile *__restrict__ t, int nt)
{
    __shared__ KI sh[64];
    const int tid = threadIdx.x;
    const int chunk = (nt + 1023) / 1024;
    const int q0 = min(nt, tid * chunk), q1 = min(nt, q0 + chunk);
    KI mx = ki_low(), mn = ki_high();
    for (int q = q0; q < q1; ++q) { mx = ki_max(mx, t[q].mx); mn = ki_min(mn, t[q].mn); }
    KI run = ki_block_exscan<1>(mx, ki_low(), sh);
    for (int q = q0; q < q1; ++q) { t[q].pre = run; run = ki_max(run, t[q].mx); }
    run = ki_block_exscan<-1>(mn, ki_high(), sh);
    for (int q = q1 - 1; q >= q0; --q) { t[q].suf = run; run = ki_min(run, t[q].mn); }
}

// flag the misplaced elements; count them per tile
__global__ void __launch_bounds__(NS_THREADS) k_ns_mark(const uint64_t *__restrict__ keys,
                                                        const uint32_t *__restrict__ ids, int64_t n,
                                                        NsTile *__restrict__ t, uint8_t *__restrict__ flag)
{
    __shared__ KI sh[64];
    __shared__ int scnt[NS_THREADS / 32];
    const int64_t b0 = (int64_t)blockIdx.x * NS_TILE + NS_PER * threadIdx.x;
    KI e[NS_PER];
#pragma unroll
    for (int u = 0; u < NS_PER; ++u) {
        const int64_t i = b0 + u;
        e[u] = i < n ? KI{keys[i], ids[i], 0u} : ki_high();
    }
    KI tmx = ki_low(), tmn = ki_high();
#pragma unroll
    for (int u = 0; u < NS_PER; ++u) { tmx = ki_max(tmx, e[u]); tmn = ki_min(tmn, e[u]); }
    KI pre = ki_block_exscan<1>(tmx, ki_low(), sh);
    KI suf = ki_block_exscan<-1>(tmn, ki_high(), sh);
    pre = ki_max(pre, t[blockIdx.x].pre);
    suf = ki_min(suf, t[blockIdx.x].suf);
    KI sufs[NS_PER];
#pragma unroll
    for (int u = NS_PER - 1; u >= 0; --u) { sufs[u] = suf; suf = ki_min(suf, e[u]); }
    int c = 0;
#pragma unroll
    for (int u = 0; u < NS_PER; ++u) {
        const int64_t i = b0 + u;
        const bool in_place = ki_lt(pre, e[u]) && ki_lt(e[u], sufs[u]);
        pre = ki_max(pre, e[u]);
        if (i < n) {
            flag[i] = in_place ? 0 : 1;
            c += in_place ? 0 : 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) scnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < NS_THREADS / 32; ++k) tot += scnt[k];
        t[blockIdx.x].cnt = tot;
    }
}

// exclusive scan of the per-tile counts (one block); total -> cnt->ns_total
__global__ void __launch_bounds__(1024) k_ns_offsets(NsTile *__restrict__ t, int nt, DevCounters *cnt)
{
    __shared__ long long sh[1024];
    const int tid = threadIdx.x;
    const int chunk = (nt + 1023) / 1024;
    const int q0 = min(nt, tid * chunk), q1 = min(nt, q0 + chunk);
    long long loc = 0;
    for (int q = q0; q < q1; ++q) loc += t[q].cnt;
    sh[tid] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const long long v = tid >= o ? sh[tid - o] : 0;
        __syncthreads();
        sh[tid] += v;
        __syncthreads();
    }
    long long run = sh[tid] - loc;
    for (int q = q0; q < q1; ++q) { t[q].off = (int32_t)run; run += t[q].cnt; }
    if (tid == 1023) cnt->ns_total = sh[1023];
}

// misplaced elements (key, id, position) in position order
__global__ void __launch_bounds__(NS_THREADS) k_ns_compact(const uint64_t *__restrict__ keys,
                                                           const uint32_t *__restrict__ ids, int64_t n,
                                                           const NsTile *__restrict__ t,
                                                           const uint8_t *__restrict__ flag,
                                                           uint64_t *__restrict__ mk, uint32_t *__restrict__ mi,
                                                           int32_t *__restrict__ mpos, const DevCounters *cnt,
                                                           int limit)
{
    if (cnt->ns_total > limit) return;            // the full sort follows
    __shared__ int sw[NS_THREADS / 32];
    const int64_t b0 = (int64_t)blockIdx.x * NS_TILE + NS_PER * threadIdx.x;
    int f[NS_PER], c = 0;
#pragma unroll
    for (int u = 0; u < NS_PER; ++u) {
        const int64_t i = b0 + u;
        f[u] = (i < n) ? flag[i] : 0;
        c += f[u];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += sw[k];
    int o = t[blockIdx.x].off + before + x - c;
#pragma unroll
    for (int u = 0; u < NS_PER; ++u) {
        if (!f[u]) continue;
        const int64_t i = b0 + u;
        mk[o] = keys[i];
        mi[o] = ids[i];
        mpos[o] = (int32_t)i;
        ++o;
    }
}

// rank of each misplaced element among the misplaced ones (equal (key, id)
// pairs ordered by position); it goes to the rank-th misplaced position.
// The grid covers `limit` elements; the count m = cnt->ns_total is read on
// the device, and above the limit nothing is done (the full sort follows).
constexpr int NS_RANK_T = 256;
__global__ void __launch_bounds__(NS_RANK_T) k_ns_rank(const uint64_t *__restrict__ mk,
                                                       const uint32_t *__restrict__ mi,
                                                       const int32_t *__restrict__ mpos,
                                                       const DevCounters *cnt, int limit,
                                                       uint64_t *__restrict__ keys_out,
                                                       uint32_t *__restrict__ src_pos)
{
    const long long mt = cnt->ns_total;
    if (mt > limit) return;                       // uniform over the block
    const int m = (int)mt;
    __shared__ uint64_t sk[NS_RANK_T];
    __shared__ uint32_t si[NS_RANK_T];
    const int e = blockIdx.x * NS_RANK_T + threadIdx.x;
    const bool valid = e < m;
    const uint64_t ke = valid ? mk[e] : 0;
    const uint32_t ie = valid ? mi[e] : 0;
    int r = 0;
    for (int base = 0; base < m; base += NS_RANK_T) {
        const int f = base + threadIdx.x;
        __syncthreads();
        if (f < m) { sk[threadIdx.x] = mk[f]; si[threadIdx.x] = mi[f]; }
        __syncthreads();
        const int lim = min(NS_RANK_T, m - base);
        for (int k = 0; k < lim; ++k) {
            const uint64_t kf = sk[k];
            const uint32_t jf = si[k];
            r += (kf < ke || (kf == ke && (jf < ie || (jf == ie && base + k < e)))) ? 1 : 0;
        }
    }
    if (valid) {
        const int32_t dest = mpos[r];
        keys_out[dest] = ke;
        src_pos[r] = (uint32_t)mpos[e];
    }
}

// move only the misplaced particles: gather into scratch, then put back
// (grids over `limit` elements, m read on the device as in k_ns_rank)
__global__ void k_ns_gather(FieldTable t, const uint32_t *__restrict__ src_pos, const DevCounters *cnt, int limit)
{
    const long long m = cnt->ns_total;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > limit || k >= m) return;
    const uint32_t p = src_pos[k];
    for (int f = 0; f < t.nf; ++f) {
        if (t.size[f] == 8) ((double *)t.dst[f])[k] = ((const double *)t.src[f])[p];
        else ((uint32_t *)t.dst[f])[k] = ((const uint32_t *)t.src[f])[p];
    }
}

__global__ void k_ns_put(FieldTable t, const int32_t *__restrict__ mpos, const DevCounters *cnt, int limit)
{
    const long long m = cnt->ns_total;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > limit || k >= m) return;
    const int32_t d = mpos[k];
    for (int f = 0; f < t.nf; ++f) {
        if (t.size[f] == 8) ((double *)t.src[f])[d] = ((const double *)t.dst[f])[k];
        else ((uint32_t *)t.src[f])[d] = ((const uint32_t *)t.dst[f])[k];
    }
}

// ------------------------------------------------------------------ leaves and groups
// dlev[i]: octree level at which key i first differs from key i-1
// (1 = top split, 21 = finest; 22 = identical; 0 for i = 0).
__global__ void k_dlev(const uint64_t *__restrict__ keys, int64_t n, uint8_t *__restrict__ dlev)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0) { dlev[0] = 0; return; }
    const uint64_t x = keys[i - 1] ^ keys[i];
    dlev[i] = x ? (uint8_t)(21 - (63 - __clzll((long long)x)) / 3) : (uint8_t)22;
}

// Leaf level of particle i: the shallowest level l whose cell around i holds
// at most S particles.  With B(t) = min dlev[i-t..i] and F(t) = min
// dlev[i+1..i+t] (0 outside [0, n)), the run at level l has at most S
// particles iff max(B(tb), F(S - tb)) <= l for some tb in [0, S).
__global__ void k_leaf_level(const uint8_t *__restrict__ dlev, int64_t n, int S,
                             uint8_t *__restrict__ plev, DevCounters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t F[33];
    uint8_t m = 255;
    for (int t = 1; t <= S; ++t) {
        int64_t j = i + t;
        uint8_t d = j < n ? dlev[j] : 0;
        m = d < m ? d : m;
        F[t] = m;
    }
    uint8_t B = 255, best = 255;
    for (int tb = 0; tb < S; ++tb) {
        int64_t j = i - tb;
        uint8_t d = j >= 0 ? dlev[j] : 0;
        B = d < B ? d : B;
        uint8_t c = B > F[S - tb] ? B : F[S - tb];
        best = c < best ? c : best;
    }
    if (best > 21) { atomicOr(&cnt->err, ERRB_LEAF_DEGENERATE); best = 21; }
    plev[i] = best;
}

// The same for a leaf size S known at compile time: the block's window of
// dlev sits in shared memory and the forward minima in registers.
template <int S>
__global__ void __launch_bounds__(256) k_leaf_level_s(const uint8_t *__restrict__ dlev, int64_t n,
                                                      uint8_t *__restrict__ plev, DevCounters *cnt)
{
    __shared__ uint8_t w[256 + 2 * S];              // w[k] = dlev[base - S + 1 + k], 0 outside [0, n)
    const int64_t base = (int64_t)blockIdx.x * 256;
    for (int k = threadIdx.x; k < 256 + 2 * S - 1; k += 256) {
        const int64_t j = base - S + 1 + k;
        w[k] = (j >= 0 && j < n) ? dlev[j] : (uint8_t)0;
    }
    __syncthreads();
    const int64_t i = base + threadIdx.x;
    if (i >= n) return;
    const int c = threadIdx.x + S - 1;              // w[c] = dlev[i]
    uint8_t F[S + 1];
    uint8_t m = 255;
#pragma unroll
    for (int t = 1; t <= S; ++t) {
        const uint8_t d = w[c + t];
        m = d < m ? d : m;
        F[t] = m;
    }
    uint8_t B = 255, best = 255;
#pragma unroll
    for (int tb = 0; tb < S; ++tb) {
        const uint8_t d = w[c - tb];
        B = d < B ? d : B;
        const uint8_t v = B > F[S - tb] ? B : F[S - tb];
        best = v < best ? v : best;
    }
    if (best > 21) { atomicOr(&cnt->err, ERRB_LEAF_DEGENERATE); best = 21; }
    plev[i] = best;
}

// leaf start flag (itmp0) and sibling-segment start index (itmp1, -1 if none)
__global__ void k_mark(const uint8_t *__restrict__ dlev, const uint8_t *__restrict__ plev, int64_t n,
                       int32_t *__restrict__ leaf_start, int32_t *__restrict__ seg_val)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int L = plev[i], d = dlev[i];
    const bool ls = (i == 0) || d <= L;
    const bool seg = ls && ((i == 0) || d <= L - 1 || plev[i - 1] != L);
    leaf_start[i] = ls ? 1 : 0;
    seg_val[i] = seg ? (int32_t)i : -1;
}

// group start: a sibling-segment start, or every 32nd particle inside one
__global__ void k_mark_groups(int32_t *__restrict__ segbeg_to_flag, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t sb = segbeg_to_flag[i];
    segbeg_to_flag[i] = (((int32_t)i - sb) % SPH_WARP) == 0 ? 1 : 0;
}

// h and m of the first particle in key order: the reference of the units
template <typename T>
__global__ void k_unit_ref(const T *__restrict__ h, const T *__restrict__ m, DevCounters *cnt)
{
    cnt->unit_ref[0] = (double)h[0];
    cnt->unit_ref[1] = (double)m[0];
}

__global__ void k_emit(const int32_t *__restrict__ leaf_start, const int32_t *__restrict__ grp_start,
                       const int32_t *__restrict__ leaf_idx, const int32_t *__restrict__ grp_idx,
                       const uint8_t *__restrict__ plev, int64_t n, int32_t *__restrict__ leaf_begin,
                       int32_t *__restrict__ leaf_level, int32_t *__restrict__ group_begin,
                       DevCounters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (leaf_start[i]) { leaf_begin[leaf_idx[i]] = (int32_t)i; leaf_level[leaf_idx[i]] = plev[i]; }
    if (grp_start[i]) group_begin[grp_idx[i]] = (int32_t)i;
    if (i == n - 1) {
        const int32_t nl = leaf_idx[i] + leaf_start[i];
        const int32_t ng = grp_idx[i] + grp_start[i];
        leaf_begin[nl] = (int32_t)n;
        group_begin[ng] = (int32_t)n;
        cnt->n_leaves = nl;
        cnt->n_groups = ng;
    }
}

// Bounding box of each range [begin[r], begin[r+1]) of at most 32 particles
// from the FP32 high parts of the two-float positions, widened by one ulp
// (x lies within half an ulp of its high part), and the largest coverage
// radius in the range (.w of lo); SEG lanes per range (8 for the leaves,
// whose ranges are short; 32 for the target groups).
template <int SEG>
__global__ void k_range_boxes(const int32_t *__restrict__ begin, int nr, const float4 *__restrict__ A,
                              const float4 *__restrict__ B, const float *__restrict__ cov,
                              float4 *__restrict__ lo4, float4 *__restrict__ hi4)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = (int)(t / SEG);
    const int sl = threadIdx.x & (SEG - 1);
    if (t / 32 * (32 / SEG) >= nr) return;          // whole warps leave together
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    float cm = 0.f;
    if (r < nr) {
        const int b = begin[r], e = begin[r + 1];
        for (int i = b + sl; i < e; i += SEG) {
            const float4 a = A[i];
            const float c[3] = {a.x, a.z, B[i].x};
            for (int d = 0; d < 3; ++d) { mn[d] = fminf(mn[d], c[d]); mx[d] = fmaxf(mx[d], c[d]); }
            cm = fmaxf(cm, cov[i]);
        }
    }
    for (int o = SEG / 2; o > 0; o >>= 1) {
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
        cm = fmaxf(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    }
    if (sl == 0 && r < nr) {
        lo4[r] = make_float4(nextafterf(mn[0], -FLT_MAX), nextafterf(mn[1], -FLT_MAX), nextafterf(mn[2], -FLT_MAX), cm);
        hi4[r] = make_float4(nextafterf(mx[0], FLT_MAX), nextafterf(mx[1], FLT_MAX), nextafterf(mx[2], FLT_MAX), 0.f);
    }
}

// ------------------------------------------------------------------ radix tree over leaves
__device__ __forceinline__ int delta_key(const uint64_t *__restrict__ keys, const int32_t *__restrict__ lb,
                                         int nl, int i, int j)
{
    if (j < 0 || j >= nl) return -1;
    uint64_t a = keys[lb[i]], b = keys[lb[j]];
    if (a == b) return 64 + __clz(i ^ j);
    return __clzll((long long)(a ^ b));
}

// Karras (2012) construction: internal node i covers a leaf range whose
// split is the first differing bit; children with index bit 31 are leaves.
__global__ void k_radix_tree(const uint64_t *__restrict__ keys, const int32_t *__restrict__ lb, int nl,
                             int32_t *__restrict__ child, int32_t *__restrict__ node_parent,
                             int32_t *__restrict__ leaf_parent, int32_t *__restrict__ node_delta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl - 1) return;
    const int d = (delta_key(keys, lb, nl, i, i + 1) - delta_key(keys, lb, nl, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta_key(keys, lb, nl, i, i - d);
    int lmax = 2;
    while (delta_key(keys, lb, nl, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta_key(keys, lb, nl, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta_key(keys, lb, nl, i, j);
    node_delta[i] = dnode;                       // leading key bits the node's leaves share
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta_key(keys, lb, nl, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + (d < 0 ? -1 : 0);
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    int c0, c1;
    if (lo == gamma) { c0 = gamma | (int)0x80000000; leaf_parent[gamma] = i; }
    else { c0 = gamma; node_parent[gamma] = i; }
    if (hi == gamma + 1) { c1 = (gamma + 1) | (int)0x80000000; leaf_parent[gamma + 1] = i; }
    else { c1 = gamma + 1; node_parent[gamma + 1] = i; }
    child[2 * i] = c0;
    child[2 * i + 1] = c1;
    if (i == 0) node_parent[0] = -1;
}

// Start-cell table of the neighbour search: for each level l = 1..CELL_LEVELS
// and each cell of the level-l grid (index x + 2^l (y + 2^l z)), the tree
// node that holds exactly the cell's particles: the internal node whose
// leaves share the cell's 1 + 3 l key bits while its parent's do not, or a
// leaf alone in its cell (leaf | 1 << 31); -1 where the cell holds no
// particle or lies inside a coarser leaf (the lookup then finds that leaf at
// the coarser level).  Cells come from a particle of the node (leaf i's first
// particle lies in internal node i), with the key arithmetic.
__global__ void k_cell_table(int nl, const int32_t *__restrict__ lb, const int32_t *__restrict__ leaf_level,
                             const int32_t *__restrict__ node_parent, const int32_t *__restrict__ leaf_parent,
                             const int32_t *__restrict__ node_delta, const double *__restrict__ x,
                             const double *__restrict__ y, const double *__restrict__ z, int pow2_shift,
                             const DevCounters *cnt, int32_t *__restrict__ table)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * nl - 1) return;
    const bool leaf = t >= nl - 1;
    const int id = leaf ? t - (nl - 1) : t;
    const int dp = leaf ? node_delta[leaf_parent[id]] : (id == 0 ? 0 : node_delta[node_parent[id]]);
    const int dself = leaf ? 1 + 3 * leaf_level[id] : node_delta[id];
    const int p = lb[id];
    uint64_t cx, cy, cz;
    grid_cell(x[p], y[p], z[p], pow2_shift, cnt, cx, cy, cz);
    for (int l = 1; l <= CELL_LEVELS; ++l) {
        if (!(dp < 1 + 3 * l && 1 + 3 * l <= dself)) continue;
        const int sh = 21 - l;
        const int64_t c = (int64_t)(cx >> sh) + ((int64_t)(cy >> sh) << l) + ((int64_t)(cz >> sh) << (2 * l));
        table[cell_table_offset(l) + c] = leaf ? (id | (int)0x80000000) : id;
    }
}

__device__ __forceinline__ void load_box(int c, const float4 *leaf_lo, const float4 *leaf_hi,
                                         const float4 *node_lo, const float4 *node_hi, float4 &lo,
                                         float4 &hi)
{
    if (c < 0) {
        const int id = c & 0x7fffffff;
        lo = __ldcg(leaf_lo + id);
        hi = __ldcg(leaf_hi + id);
    } else {
        lo = __ldcg(node_lo + c);
        hi = __ldcg(node_hi + c);
    }
}

// Bottom-up boxes: the second child to arrive at a node merges both.
__global__ void k_refit(int nl, const int32_t *__restrict__ child, const int32_t *__restrict__ node_parent,
                        const int32_t *__restrict__ leaf_parent, unsigned *__restrict__ visit,
                        const float4 *__restrict__ leaf_lo, const float4 *__restrict__ leaf_hi,
                        float4 *node_lo, float4 *node_hi)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    int node = leaf_parent[l];
    for (int depth = 0; node >= 0 && depth < 4096; ++depth) {
        __threadfence();
        if (atomicAdd(&visit[node], 1u) == 0) return;
        __threadfence();
        float4 alo, ahi, blo, bhi;
        load_box(child[2 * node], leaf_lo, leaf_hi, node_lo, node_hi, alo, ahi);
        load_box(child[2 * node + 1], leaf_lo, leaf_hi, node_lo, node_hi, blo, bhi);
        float4 lo = make_float4(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z), fmaxf(alo.w, blo.w));
        float4 hi = make_float4(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z), 0.f);
        __stcg(node_lo + node, lo);
        __stcg(node_hi + node, hi);
        node = node_parent[node];
    }
}

int boxes_and_refit(sph_ctx *ctx, cudaStream_t s)
{
    const int nl = (int)ctx->n_leaves, ng = (int)ctx->n_groups;
    k_range_boxes<8><<<grid_for((int64_t)nl * 8, 256), 256, 0, s>>>(ctx->leaf_begin, nl, ctx->srcA, ctx->srcB,
                                                                     ctx->cov, ctx->leaf_lo, ctx->leaf_hi);
    SPH_CHECK_LAUNCH();
    k_range_boxes<32><<<grid_for((int64_t)ng * 32, 256), 256, 0, s>>>(ctx->group_begin, ng, ctx->srcA, ctx->srcB,
                                                                      ctx->cov, ctx->group_lo, ctx->group_hi);
    SPH_CHECK_LAUNCH();
    if (nl > 1) {
        SPH_CUDA(cudaMemsetAsync(ctx->node_visit, 0, sizeof(unsigned) * (size_t)(nl - 1), s));
        k_refit<<<grid_for(nl, 256), 256, 0, s>>>(nl, ctx->node_child, ctx->node_parent, ctx->leaf_parent,
                                                  ctx->node_visit, ctx->leaf_lo, ctx->leaf_hi, ctx->node_lo,
                                                  ctx->node_hi);
        SPH_CHECK_LAUNCH();
    }
    return SPH_OK;
}

template <typename T>
void add_field(FieldTable &t, unsigned char *&buf, int64_t nmax, const void *ptr)
{
    if (!ptr) return;
    t.src[t.nf] = ptr;
    t.dst[t.nf] = buf;
    t.size[t.nf] = (int)sizeof(T);
    buf += ((size_t)nmax * sizeof(T) + 255) & ~(size_t)255;
    ++t.nf;
}

template <typename T>
FieldTable make_table(sph_ctx *ctx, const sph_particles *p, bool derived)
{
    FieldTable t{};
    unsigned char *buf = ctx->gbuf;
    const int64_t nm = ctx->n_max;
    add_field<double>(t, buf, nm, p->x);
    add_field<double>(t, buf, nm, p->y);
    add_field<double>(t, buf, nm, p->z);
    const void *tf[] = {p->vx, p->vy, p->vz, p->m, p->h, p->u, p->hprev, p->rho,
                        p->ax, p->ay, p->az, p->dudt, p->divv};
    for (const void *f : tf) add_field<T>(t, buf, nm, f);
    if (derived) {                                 // outputs that a step recomputes before reading
        const void *td[] = {p->omega, p->P, p->c, p->vsig};
        for (const void *f : td) add_field<T>(t, buf, nm, f);
    }
    add_field<int32_t>(t, buf, nm, p->nnb);
    add_field<uint32_t>(t, buf, nm, p->id);
    // the last list lengths, which size the next lists, follow their particles
    if (ctx->lcount_valid) add_field<uint32_t>(t, buf, nm, ctx->lcount);
    return t;
}

// LSD passes over the key bytes first_byte..7 (an even number of passes, so
// the result is back in key_a / val_a)
int radix_sort(sph_ctx *ctx, int64_t n, cudaStream_t s, int first_byte = 0)
{
    // the tile staging needs more than 48 KB (set on the current device)
    SPH_CUDA(cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SCATTER_SMEM));
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    uint64_t *ka = ctx->key_a, *kb = ctx->key_b;
    uint32_t *va = ctx->val_a, *vb = ctx->val_b;
    for (int pass = first_byte; pass < 8; ++pass) {
        const int shift = 8 * pass;
        k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(ka, n, shift, ctx->hist, ntiles);
        SPH_CHECK_LAUNCH();
        SPH_TRY(scan_exclusive_i32(ctx, (const int32_t *)ctx->hist, (int32_t *)ctx->hist,
                                   (int64_t)RS_BINS * ntiles, s));
        k_rs_scatter<<<ntiles, RS_THREADS, RS_SCATTER_SMEM, s>>>(ka, va, kb, vb, n, shift, ctx->hist, ntiles);
        SPH_CHECK_LAUNCH();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return SPH_OK;
}

int compute_domain(sph_ctx *ctx, const sph_particles *p, cudaStream_t s)
{
    const sph_params &q = ctx->prm;
    if (q.periodic) {
        k_domain<<<1, 32, 0, s>>>(nullptr, 0, 1, q.box_lo[0], q.box_lo[1], q.box_lo[2],
                                  q.box_hi[0] - q.box_lo[0], ctx->dcnt);
    } else {
        const int nb = ctx->red_blocks;
        k_bbox_partial<<<nb, 256, 0, s>>>(p->x, p->y, p->z, p->n, ctx->red);
        SPH_CHECK_LAUNCH();
        k_domain<<<1, 32, 0, s>>>(ctx->red, nb, 0, 0, 0, 0, 0, ctx->dcnt);
    }
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

template <typename T>
int keys_impl(sph_ctx *ctx, const sph_particles *p, uint64_t *keys, uint32_t *vals, cudaStream_t s)
{
    SPH_TRY(compute_domain(ctx, p, s));
    // a periodic box at the origin with a power-of-two side: cells by shifts
    int pow2_shift = -1;
    const sph_params &q = ctx->prm;
    if (q.periodic && q.box_lo[0] == 0.0 && q.box_lo[1] == 0.0 && q.box_lo[2] == 0.0) {
        int ex = 0;
        const double fr = std::frexp(q.box_hi[0], &ex);        // L = fr 2^ex, fr in [0.5, 1)
        if (fr == 0.5 && 22 - ex >= 0 && 22 - ex <= 60) pow2_shift = 22 - ex;   // L = 2^(ex - 1)
    }
    ctx->pow2_shift = pow2_shift;
    k_keys<T><<<grid_for(p->n, 256), 256, 0, s>>>(p->x, p->y, p->z, (const T *)p->h, (const T *)p->m, p->n,
                                                  ctx->prm.curve, ctx->prm.dim, pow2_shift, ctx->dcnt, keys, vals);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

// The near-sorted path, launched without a host synchronisation: the
// detection counts the misplaced particles into cnt->ns_total, and when there
// are at most `limit` of them the same launches move them into key order
// (their kernels read the count on the device).  Above the limit nothing
// moves; the caller learns which case it was at its next synchronisation.
void near_sorted(sph_ctx *ctx, sph_particles *p, const FieldTable &t, int limit, cudaStream_t s)
{
    const int64_t n = p->n;
    const int nt = (int)((n + NS_TILE - 1) / NS_TILE);
    k_ns_tiles<<<nt, NS_THREADS, 0, s>>>(ctx->key_a, p->id, n, ctx->ns_tiles);
    k_ns_prefix<<<1, 1024, 0, s>>>(ctx->ns_tiles, nt);
    k_ns_mark<<<nt, NS_THREADS, 0, s>>>(ctx->key_a, p->id, n, ctx->ns_tiles, ctx->dlev);
    k_ns_offsets<<<1, 1024, 0, s>>>(ctx->ns_tiles, nt, ctx->dcnt);
    uint64_t *mk = ctx->key_b;
    uint32_t *mi = ctx->val_b;
    int32_t *mpos = ctx->itmp0;
    uint32_t *src_pos = (uint32_t *)ctx->itmp1;
    k_ns_compact<<<nt, NS_THREADS, 0, s>>>(ctx->key_a, p->id, n, ctx->ns_tiles, ctx->dlev, mk, mi, mpos, ctx->dcnt,
                                            limit);
    k_ns_rank<<<(limit + NS_RANK_T - 1) / NS_RANK_T, NS_RANK_T, 0, s>>>(mk, mi, mpos, ctx->dcnt, limit, ctx->key_a,
                                                                         src_pos);
    k_ns_gather<<<grid_for(limit, 256), 256, 0, s>>>(t, src_pos, ctx->dcnt, limit);
    k_ns_put<<<grid_for(limit, 256), 256, 0, s>>>(t, mpos, ctx->dcnt, limit);
}

// The particle arrays as the scratch copy of the table holds them (the
// fields the table does not permute keep the caller's pointers).
sph_particles scratch_view(const FieldTable &t, const sph_particles *p)
{
    sph_particles v = *p;
    void **fields[] = {(void **)&v.x, (void **)&v.y, (void **)&v.z, &v.vx, &v.vy, &v.vz, &v.m, &v.h, &v.u,
                       &v.hprev, &v.rho, &v.omega, &v.P, &v.c, &v.ax, &v.ay, &v.az, &v.dudt, &v.divv,
                       &v.vsig, (void **)&v.nnb, (void **)&v.id};
    for (void **f : fields)
        for (int k = 0; k < t.nf; ++k)
            if (*f && t.src[k] == *f) { *f = t.dst[k]; break; }
    return v;
}

// full sort, then permute every particle array into key order.  prefix: the
// radix passes cover the top 32 key bits and runs of equal top halves are
// ordered on the device (ERRB_PREFIX_RUN when one is too long for that).
// hook (may be null) runs on the scratch copy between the gather and the
// copy back.
int full_sort(sph_ctx *ctx, sph_particles *p, const FieldTable &t, cudaStream_t s, bool prefix, OrderHook *hook)
{
    const int64_t n = p->n;
    if (prefix) {
        SPH_TRY(radix_sort(ctx, n, s, 4));
        k_fix_prefix_runs<<<grid_for(n, 256), 256, 0, s>>>(ctx->key_a, ctx->val_a, p->id, n, ctx->dcnt);
    } else {
        SPH_TRY(radix_sort(ctx, n, s));
        k_fix_ties<<<grid_for(n, 256), 256, 0, s>>>(ctx->key_a, ctx->val_a, p->id, n, ctx->dcnt);
    }
    SPH_CHECK_LAUNCH();
    k_gather<<<grid_for(n, 256), 256, 0, s>>>(t, ctx->val_a, n);
    SPH_CHECK_LAUNCH();
    if (hook) {
        const sph_particles v = scratch_view(t, p);
        SPH_TRY((*hook)(s, &v));
    }
    k_copy_back<<<grid_for(n, 256), 256, 0, s>>>(t, n);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

// octree leaves and target groups of the keys in key_a (in bounds for any
// order of the keys), then one synchronisation for the counts
template <typename T>
int leaves_impl(sph_ctx *ctx, sph_particles *p, cudaStream_t s)
{
    const int64_t n = p->n;
    k_unit_ref<T><<<1, 1, 0, s>>>((const T *)p->h, (const T *)p->m, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    k_dlev<<<grid_for(n, 256), 256, 0, s>>>(ctx->key_a, n, ctx->dlev);
    SPH_CHECK_LAUNCH();
    if (ctx->prm.leaf_size == 32)
        k_leaf_level_s<32><<<grid_for(n, 256), 256, 0, s>>>(ctx->dlev, n, ctx->plev, ctx->dcnt);
    else
        k_leaf_level<<<grid_for(n, 128), 128, 0, s>>>(ctx->dlev, n, ctx->prm.leaf_size, ctx->plev, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    int32_t *ls = ctx->itmp0, *gs = ctx->itmp1;
    int32_t *lidx = ctx->itmp2, *gidx = ctx->itmp3;
    k_mark<<<grid_for(n, 256), 256, 0, s>>>(ctx->dlev, ctx->plev, n, ls, gs);
    SPH_CHECK_LAUNCH();
    SPH_TRY(scan_inclusive_max_i32(ctx, gs, gs, n, s));
    k_mark_groups<<<grid_for(n, 256), 256, 0, s>>>(gs, n);
    SPH_CHECK_LAUNCH();
    SPH_TRY(scan_exclusive_i32(ctx, ls, lidx, n, s));
    SPH_TRY(scan_exclusive_i32(ctx, gs, gidx, n, s));
    k_emit<<<grid_for(n, 256), 256, 0, s>>>(ls, gs, lidx, gidx, ctx->plev, n, ctx->leaf_begin, ctx->leaf_level,
                                            ctx->group_begin, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    return sync_counters(ctx, s);
}

template <typename T>
int build_impl(sph_ctx *ctx, sph_particles *p, cudaStream_t s, OrderHook *after_order, bool derived)
{
    const int64_t n = p->n;
    ctx->tree_valid = false;
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
    SPH_TRY(keys_impl<T>(ctx, p, ctx->key_a, ctx->val_a, s));
    FieldTable t = make_table<T>(ctx, p, derived);
    // after two full sorts in a row (most keys displaced every step) the
    // detection of a nearly sorted order is skipped for seven builds, then
    // tried again.  The host reads the detection's count before anything
    // else runs, so a failed attempt costs the detection only: the full sort
    // follows at once and the leaves and after_order run once, on the final
    // order.
    int64_t m = -1;                                // >= 0: the near-sorted path moved m particles
    if (ctx->ns_skip > 0) {
        --ctx->ns_skip;
    } else {
        const int limit = (int)std::min<int64_t>(NS_LIMIT, std::max<int64_t>(n / 4, 1024));
        near_sorted(ctx, p, t, limit, s);
        SPH_CHECK_LAUNCH();
        SPH_TRY(sync_counters(ctx, s));
        if (ctx->hcnt->ns_total <= limit) m = ctx->hcnt->ns_total;
        ctx->ns_full_streak = m < 0 ? ctx->ns_full_streak + 1 : 0;
        if (ctx->ns_full_streak >= 2) ctx->ns_skip = 7;
    }
    if (m < 0) SPH_TRY(full_sort(ctx, p, t, s, true, after_order));
    else if (after_order) SPH_TRY((*after_order)(s, p));
    SPH_TRY(leaves_impl<T>(ctx, p, s));
    if (ctx->hcnt->err & ERRB_PREFIX_RUN) {
        // more than 64 particles share the top 32 key bits: the order inside
        // such a run is not final; sort the (now permuted) particles on all
        // bits and build the leaves again
        SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
        if (after_order) SPH_TRY(after_order->join(s));   // its reads of the scratch copy end first
        SPH_TRY(keys_impl<T>(ctx, p, ctx->key_a, ctx->val_a, s));
        SPH_TRY(full_sort(ctx, p, t, s, false, after_order));
        SPH_TRY(leaves_impl<T>(ctx, p, s));
    }
    ctx->ns_moved = m;
    const uint32_t err = ctx->hcnt->err;
    for (int d = 0; d < 4; ++d) ctx->dom[d] = ctx->hcnt->dom[d];
    if (err & ERRB_NONFINITE)
        return sph_fail(ctx, SPH_ERR_NONFINITE, "sph_build_tree: NaN/Inf position, mass or h (or h <= 0)");
    if (err & ERRB_OFF_AXIS)
        return sph_fail(ctx, SPH_ERR_ARG, "sph_build_tree: dim 1 needs y = z = 0 for every particle");
    if (err & (ERRB_LEAF_DEGENERATE | ERRB_TIE_RUN))
        return sph_fail(ctx, SPH_ERR_CAPACITY,
                        "sph_build_tree: more than leaf_size particles share one 63-bit key");
    ctx->n = n;
    ctx->n_leaves = ctx->hcnt->n_leaves;
    ctx->n_groups = ctx->hcnt->n_groups;
    if (ctx->fp64) {
        // 2^kL h and 2^kM m of the first particle in [1, 2)
        const double h0 = ctx->hcnt->unit_ref[0], m0 = ctx->hcnt->unit_ref[1];
        const int kL = (std::isfinite(h0) && h0 > 0.0) ? std::max(-200, std::min(200, -std::ilogb(h0))) : 0;
        const int kM = (std::isfinite(m0) && m0 > 0.0) ? std::max(-200, std::min(200, -std::ilogb(m0))) : 0;
        ctx->len_scale = std::ldexp(1.0, kL);
        ctx->mass_scale = std::ldexp(1.0, kM);
    }
    if (ctx->len_scale != 1.0 || ctx->mass_scale != 1.0)
        k_pack_pos<T, true><<<grid_for(n, 256), 256, 0, s>>>(p->x, p->y, p->z, (const T *)p->m, n, ctx->len_scale,
                                                             ctx->mass_scale, ctx->srcA, ctx->srcB);
    else
        k_pack_pos<T, false><<<grid_for(n, 256), 256, 0, s>>>(p->x, p->y, p->z, (const T *)p->m, n, 1.0, 1.0,
                                                              ctx->srcA, ctx->srcB);
    SPH_CHECK_LAUNCH();
    const int nl = (int)ctx->n_leaves;
    if (nl > 1) {
        k_radix_tree<<<grid_for(nl - 1, 256), 256, 0, s>>>(ctx->key_a, ctx->leaf_begin, nl, ctx->node_child,
                                                           ctx->node_parent, ctx->leaf_parent, ctx->node_delta);
        SPH_CHECK_LAUNCH();
        SPH_CUDA(cudaMemsetAsync(ctx->cell_table, 0xFF, sizeof(int32_t) * (size_t)cell_table_size(), s));
        k_cell_table<<<grid_for(2 * (int64_t)nl - 1, 256), 256, 0, s>>>(
            nl, ctx->leaf_begin, ctx->leaf_level, ctx->node_parent, ctx->leaf_parent, ctx->node_delta, p->x, p->y,
            p->z, ctx->pow2_shift, ctx->dcnt, ctx->cell_table);
        SPH_CHECK_LAUNCH();
    }
    ctx->tree_valid = true;
    ctx->lists_valid = false;
    return SPH_OK;
}

}  // namespace

int tree_build(sph_ctx *ctx, sph_particles *p, cudaStream_t s, OrderHook *after_order, bool derived)
{
    return ctx->fp64 ? build_impl<double>(ctx, p, s, after_order, derived)
                     : build_impl<float>(ctx, p, s, after_order, derived);
}

// Boxes of leaves, groups and radix-tree nodes with the largest coverage
// radius below each (positions of the current tree, coverage of the lists).
int tree_boxes(sph_ctx *ctx, cudaStream_t s) { return boxes_and_refit(ctx, s); }

int tree_keys(sph_ctx *ctx, const sph_particles *p, uint64_t *keys_out, cudaStream_t s)
{
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
    SPH_TRY(ctx->fp64 ? keys_impl<double>(ctx, p, keys_out, nullptr, s) : keys_impl<float>(ctx, p, keys_out, nullptr, s));
    SPH_TRY(sync_counters(ctx, s));
    for (int d = 0; d < 4; ++d) ctx->dom[d] = ctx->hcnt->dom[d];
    if (ctx->hcnt->err & ERRB_NONFINITE)
        return sph_fail(ctx, SPH_ERR_NONFINITE, "sph_morton_keys: NaN/Inf position, mass or h");
    if (ctx->hcnt->err & ERRB_OFF_AXIS)
        return sph_fail(ctx, SPH_ERR_ARG, "sph_morton_keys: dim 1 needs y = z = 0 for every particle");
    return SPH_OK;
}

__global__ void k_iota(uint32_t *v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

int tree_sort(sph_ctx *ctx, int64_t n, const uint64_t *keys, const uint32_t *ids, uint32_t *perm,
              cudaStream_t s)
{
    SPH_CUDA(cudaMemsetAsync(&ctx->dcnt->err, 0, sizeof(uint32_t), s));
    SPH_CUDA(cudaMemcpyAsync(ctx->key_a, keys, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(ctx->val_a, n);
    SPH_CHECK_LAUNCH();
    SPH_TRY(radix_sort(ctx, n, s));
    k_fix_ties<<<grid_for(n, 256), 256, 0, s>>>(ctx->key_a, ctx->val_a, ids, n, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    SPH_CUDA(cudaMemcpyAsync(perm, ctx->val_a, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    SPH_TRY(sync_counters(ctx, s));
    if (ctx->hcnt->err & ERRB_TIE_RUN)
        return sph_fail(ctx, SPH_ERR_CAPACITY, "sph_sort_keys: a run of more than 64 equal keys");
    return SPH_OK;
}
