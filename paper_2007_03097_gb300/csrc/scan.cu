// Device-wide scans (exclusive sum, inclusive max) used by the tree build and
// the neighbour-list allocation: reduce tiles, scan the tile totals
// recursively, then scan each tile with its offset.  Deterministic.
#include <climits>

#include "sph_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct OpAdd {
    template <typename T> __device__ T operator()(T a, T b) const { return a + b; }
    template <typename T> __device__ static T identity() { return T(0); }
};
struct OpMax {
    template <typename T> __device__ T operator()(T a, T b) const { return a > b ? a : b; }
    template <typename T> __device__ static T identity() { return T(INT_MIN); }
};

template <typename T, typename Op>
__device__ T block_scan_incl(T v, T *warp_tot)
{
    Op op;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T nb = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = op(v, nb);
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = warp_tot[lane];    // SCAN_THREADS / 32 == 32 warps
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T nb = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w = op(w, nb);
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = op(warp_tot[warp - 1], v);
    __syncthreads();
    return v;
}

template <typename TIn, typename TOut, typename Op>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const TIn *in, int64_t n, TOut *part)
{
    __shared__ TOut wt[32];
    Op op;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    TOut acc = Op::template identity<TOut>();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < n) acc = op(acc, (TOut)in[base + k]);
    acc = block_scan_incl<TOut, Op>(acc, wt);
    if (threadIdx.x == SCAN_THREADS - 1) part[blockIdx.x] = acc;
}

template <typename TIn, typename TOut, typename Op, bool EXCL>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const TIn *in, TOut *out, int64_t n,
                                                             const TOut *part_incl)
{
    __shared__ TOut wt[32];
    Op op;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    TOut x[SCAN_ITEMS];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        x[k] = (base + k < n) ? (TOut)in[base + k] : Op::template identity<TOut>();
    TOut loc[SCAN_ITEMS];
    TOut run = x[0];
    loc[0] = run;
#pragma unroll
    for (int k = 1; k < SCAN_ITEMS; ++k) { run = op(run, x[k]); loc[k] = run; }
    TOut incl = block_scan_incl<TOut, Op>(run, wt);
    // exclusive prefix of this thread within the block
    TOut prev = __shfl_up_sync(0xffffffffu, incl, 1);
    __shared__ TOut last_of_warp[32];
    if ((threadIdx.x & 31) == 31) last_of_warp[threadIdx.x >> 5] = incl;
    __syncthreads();
    TOut tprefix;
    const bool first_in_block = threadIdx.x == 0;
    if ((threadIdx.x & 31) == 0)
        tprefix = (threadIdx.x >> 5) == 0 ? Op::template identity<TOut>() : last_of_warp[(threadIdx.x >> 5) - 1];
    else
        tprefix = prev;
    TOut boff = (blockIdx.x > 0 && part_incl) ? part_incl[blockIdx.x - 1] : Op::template identity<TOut>();
    bool have = blockIdx.x > 0 && part_incl;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k >= n) break;
        TOut v = loc[k];
        if (!first_in_block) v = op(tprefix, v);
        if (have) v = op(boff, v);
        if (EXCL) v = v - x[k];
        out[base + k] = v;
    }
}

size_t level_bytes(int64_t n, int *levels)
{
    size_t b = 0;
    int l = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        b += ((size_t)m * 8 + 255) & ~(size_t)255;
        ++l;
    }
    if (levels) *levels = l;
    return b;
}

template <typename TIn, typename TOut, typename Op, bool EXCL>
int scan_generic(sph_ctx *ctx, const TIn *in, TOut *out, int64_t n, unsigned char *tmp, cudaStream_t s)
{
    if (n <= 0) return SPH_OK;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_apply<TIn, TOut, Op, EXCL><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        SPH_CHECK_LAUNCH();
        return SPH_OK;
    }
    TOut *part = reinterpret_cast<TOut *>(tmp);
    unsigned char *next = tmp + (((size_t)nb * 8 + 255) & ~(size_t)255);
    k_scan_reduce<TIn, TOut, Op><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, part);
    SPH_CHECK_LAUNCH();
    SPH_TRY((scan_generic<TOut, TOut, Op, false>(ctx, part, part, nb, next, s)));
    k_scan_apply<TIn, TOut, Op, EXCL><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, part);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return level_bytes(n, nullptr) + 256; }

int scan_exclusive_i32(sph_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s)
{
    return scan_generic<int32_t, int32_t, OpAdd, true>(ctx, in, out, n, (unsigned char *)ctx->scan_tmp, s);
}

int scan_exclusive_i64(sph_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    return scan_generic<int32_t, int64_t, OpAdd, true>(ctx, in, out, n, (unsigned char *)ctx->scan_tmp, s);
}

int scan_inclusive_max_i32(sph_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, cudaStream_t s)
{
    return scan_generic<int32_t, int32_t, OpMax, false>(ctx, in, out, n, (unsigned char *)ctx->scan_tmp, s);
}
