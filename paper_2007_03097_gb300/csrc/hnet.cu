// h-predictor network (not part of the paper's method; it only seeds the
// h-rho iteration of Eq. 9, which stays the arbiter of the converged h):
//   y = W3 silu(W2 silu(W1 f + b1) + b2) + b3,  5 -> 64 -> 64 -> 1,
// BF16 weights read by the kernels, FP32 master weights and Adam moments,
// FP32 activations and accumulation (inference: layer 2 on the tensor cores).  The prediction of log(h_next / h) is
// s = f3 * y with f3 = div v * dt: a particle at rest keeps its h exactly, and
// the network learns the gain of the continuity estimate div v dt / 3.
#include <algorithm>
#include <cmath>

#include <cuda_fp16.h>

#include "sph_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int NP = SPH_HNET_NPARAM;
// parameter layout: W1 [64][5] at 0, b1 at 320, W2 [64][64] at 384, b2 at 4480, W3 at 4544, b3 at 4608
constexpr int O_W1 = 0, O_W2 = 384, O_B2 = 4480;
constexpr int H = 64;

// logistic function with the hardware exponential and reciprocal (a few ulp)
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

// SiLU z sigm(z) = z/2 + (z/2) tanh(z/2) with the hardware tanh approximation
// (one special-function operation instead of two; relative error ~2^-11).
// The step's seed uses it: its output y enters the seed as s = f3 y with
// f3 = div v dt, so an error of 1e-3 y moves log h by 1e-3 |s|, about 1e-6 for
// the |s| ~ 1e-3 of a CFL-limited step, far below the first-order Newton bound
// sqrt(h_tol / 10) that decides whether the seed needs a second evaluation.
__device__ __forceinline__ float silu_fast(float z)
{
    const float hz = 0.5f * z;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(hz));
    return fmaf(hz, t, hz);
}

// ---------------------------------------------------------------- features
// f0 = log(h / hbar), hbar = eta (m / rho_ref)^(1/D)
// f1 = log(max(nnb, 1/2) / nbar), nbar = 32 pi eta^3 / 3 (D = 3), 4 eta (D = 1):
//      the particles within 2h at h = eta (m/rho)^(1/D)
// f2 = log(rho h^D / (m eta^D))
// f3 = div v * dt
// f4 = log(h / hprev)  (0 when hprev <= 0)
template <typename T>
struct FeatArgs {
    const T *h, *hprev, *rho, *m, *divv;
    const int32_t *nnb;
    float dt, eta, rho_ref;
    int dim;
};

template <typename T>
__device__ __forceinline__ void features_of(const FeatArgs<T> &fa, int64_t i, float *o)
{
    const float hi = (float)fa.h[i], mi = (float)fa.m[i], ri = (float)fa.rho[i];
    const bool d1 = fa.dim == 1;
    const float etaD = d1 ? fa.eta : fa.eta * fa.eta * fa.eta;
    const float hbar = d1 ? fa.eta * (mi / fa.rho_ref) : fa.eta * cbrtf(mi / fa.rho_ref);
    const float nbar = d1 ? 4.f * fa.eta : 32.f * 3.14159265358979f * etaD / 3.f;
    const float nb = fmaxf((float)fa.nnb[i], 0.5f);
    const float hp = (float)fa.hprev[i];
    o[0] = logf(hi / hbar);
    o[1] = logf(nb / nbar);
    o[2] = logf(ri * (d1 ? hi : hi * hi * hi) / (mi * etaD));
    o[3] = (float)fa.divv[i] * fa.dt;
    o[4] = hp > 0.f ? logf(hi / hp) : 0.f;
}

// features of particles i = k * stride, k < count, into f[5 k ..]
template <typename T>
__global__ void k_features(FeatArgs<T> fa, int64_t stride, int64_t count, float *__restrict__ f)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    float o[5];
    features_of(fa, k * stride, o);
#pragma unroll
    for (int c = 0; c < 5; ++c) f[5 * k + c] = o[c];
}

// ------------------------------------------------- inference, tensor cores
// One warpgroup per tile of 128 samples (a persistent loop over tiles).  Each
// thread owns one sample: it evaluates layer 1 (5 -> 64, FP32) and writes the
// activations to shared memory as the A operand of the layer-2 contraction,
// split into two FP16 terms a = hi + lo (hi = fp16(a), lo = fp16(a - hi)),
// which carry the FP32 activation to about 2^-22 of its value (the SiLU
// activations lie far inside FP16's range).  W2 enters as FP16 too: every
// BF16 weight within FP16's normal range is an FP16 value, so the weights are
// the BF16 ones exactly (a weight below 2^-14 in magnitude rounds to FP16's
// subnormal grid, 2^-24; one beyond 65504 becomes infinite and the seed falls
// back to h).  One thread issues the 8 tcgen05 MMAs (M = 128, N = 64, K = 16
// each; two terms x four K steps) that accumulate z2 = a1 W2^T in FP32 in
// tensor memory; each thread then reads its sample's row back (tcgen05.ld),
// applies b2, SiLU and layer 3 and writes f3 * y.  (Three BF16 terms held
// 48 KB of shared memory per tile and three blocks per SM; two FP16 terms
// hold 32 KB, and four blocks run per SM.)
constexpr int TM = 128;                          // samples per tile (MMA M)
constexpr int NSPLIT = 2;                        // FP16 terms per activation
constexpr uint32_t CM_LBO = 128;                 // K-adjacent core matrices
constexpr uint32_t CM_SBO = (H / 8) * 128;       // next 8 rows: 1024 bytes
constexpr int A_TILE = TM * H * 2;               // 16 KB per term
constexpr int B_TILE = H * H * 2;                // 8 KB
constexpr int B_PAD = 0;                         // A follows B (B_TILE keeps A 1024-aligned)
constexpr int WF = 320 + 64 + 64 + 64 + 1;       // FP32 W1, b1, b2, w3, b3
constexpr uint32_t TM_COLS = 64;                 // TMEM columns: D is 128 x 64 FP32
constexpr uint64_t MMA_WAIT_NS = 1000000000ull;  // give up on an MMA after 1 s

__host__ __device__ constexpr int infer_tc_smem()
{
    return 1024 + B_TILE + B_PAD + NSPLIT * A_TILE + WF * 4 + 16;
}

// byte offset of element (row, k) in a K-major no-swizzle operand of 64 columns
__device__ __forceinline__ uint32_t cm_off(int row, int k)
{
    return (uint32_t)((row >> 3) * CM_SBO + (k >> 3) * CM_LBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_f16(float lo, float hi)
{
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Step-path result: the seed h exp(s) of each particle (h itself, counted as
// a fallback, when s is not finite or changes h by more than a factor 2).
template <typename T>
struct SeedOut {
    T *seed;
};

template <bool FIELDS, typename T>
__global__ void __launch_bounds__(TM) k_infer_tc(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ f,
                                                 FeatArgs<T> fa, int64_t nb, float *__restrict__ y, SeedOut<T> so,
                                                 DevCounters *cnt, int skip_mma)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = base;
    unsigned char *sA = base + B_TILE + B_PAD;
    float *wf = (float *)(sA + NSPLIT * A_TILE);
    float *W1 = wf, *b1 = wf + 320, *b2 = wf + 384, *w3 = wf + 448, *b3 = wf + 512;
    uint64_t *bar = (uint64_t *)(wf + WF + ((WF & 1) ? 1 : 0));
    __shared__ uint32_t tslot;

    const int tid = threadIdx.x, warp = tid >> 5;
    // weights: W2 as the B operand (row n = output unit, K = input unit), the rest FP32
    // eight consecutive K entries of a row are one 16-byte core-matrix row
    // (O_W2 = 384 elements: 16-byte aligned)
    for (int v = tid; v < H * H / 8; v += TM) {
        const int n = v / (H / 8), k = 8 * (v % (H / 8));
        const __nv_bfloat16 *w8 = wb + O_W2 + n * H + k;      // eight BF16 weights -> FP16
        *reinterpret_cast<uint4 *>(sB + cm_off(n, k)) =
            make_uint4(pack_f16(__bfloat162float(w8[0]), __bfloat162float(w8[1])),
                       pack_f16(__bfloat162float(w8[2]), __bfloat162float(w8[3])),
                       pack_f16(__bfloat162float(w8[4]), __bfloat162float(w8[5])),
                       pack_f16(__bfloat162float(w8[6]), __bfloat162float(w8[7])));
    }
    for (int k = tid; k < 320 + 64; k += TM) wf[k] = __bfloat162float(wb[O_W1 + k]);          // W1, b1
    for (int k = tid; k < 64 + 64 + 1; k += TM) wf[384 + k] = __bfloat162float(wb[O_B2 + k]);  // b2, W3, b3
    const uint32_t bar_a = tc::smem_addr(bar);
    if (tid == 0) tc::mbar_init(bar_a, 1);
    if (warp == 0) tc::tmem_alloc(&tslot, TM_COLS);
    tc::fence_async_shared();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tslot;
    const uint32_t sA_a = tc::smem_addr(sA), sB_a = tc::smem_addr(sB);
    constexpr uint32_t IDESC = tc::idesc_f16_f32(TM, H);

    const int64_t ntiles = (nb + TM - 1) / TM;
    uint32_t parity = 0;
    bool failed = false;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t s = tile * TM + tid;
        const bool valid = s < nb;
        float x[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (FIELDS) {
            // a tile of particles at rest (|div v dt| <= 1e-10 for all) keeps h:
            // s = f3 y is then below the FP32 resolution of exp(s) - 1 for any
            // |y| < 300, so the network's seed would be h exactly
            const float f3 = valid ? (float)fa.divv[s] * fa.dt : 0.f;
            if (!__syncthreads_or(valid && fabsf(f3) > 1e-10f)) {
                if (valid) so.seed[s] = fa.h[s];
                continue;
            }
            if (valid) features_of(fa, s, x);
        } else if (valid) {
#pragma unroll
            for (int k = 0; k < 5; ++k) x[k] = f[5 * s + k];
        }
        // layer 1 and the three-term split, 8 units (one 16-byte row of a core matrix) at a time
#pragma unroll 1
        for (int c = 0; c < H / 8; ++c) {
            uint32_t q[NSPLIT][4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float a[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int j = 8 * c + e + u;
                    float z = b1[j];
#pragma unroll
                    for (int k = 0; k < 5; ++k) z += W1[5 * j + k] * x[k];
                    a[u] = FIELDS ? silu_fast(z) : z * sigm(z);
                }
                const __half2 hi = __floats2half2_rn(a[0], a[1]);
                q[0][e / 2] = *reinterpret_cast<const uint32_t *>(&hi);
                q[1][e / 2] = pack_f16(a[0] - __low2float(hi), a[1] - __high2float(hi));
            }
#pragma unroll
            for (int t = 0; t < NSPLIT; ++t)
                *reinterpret_cast<uint4 *>(sA + t * A_TILE + cm_off(tid, 8 * c)) =
                    make_uint4(q[t][0], q[t][1], q[t][2], q[t][3]);
        }
        tc::fence_async_shared();
        __syncthreads();
        // skip_mma (a test hook): nothing is issued, so the bounded wait
        // below runs out and the kernel takes its error path
        if (tid == 0 && !skip_mma) {
            tc::fence_after_sync();
#pragma unroll
            for (int t = 0; t < NSPLIT; ++t)
#pragma unroll
                for (int kk = 0; kk < H / 16; ++kk) {
                    const uint64_t ad = tc::smem_desc(sA_a + t * A_TILE + kk * 2 * CM_LBO, CM_LBO, CM_SBO);
                    const uint64_t bd = tc::smem_desc(sB_a + kk * 2 * CM_LBO, CM_LBO, CM_SBO);
                    tc::mma_bf16(tbase, ad, bd, IDESC, t > 0 || kk > 0);
                }
            tc::mma_commit(bar_a);
        }
        const bool ok = tc::mbar_wait(bar_a, parity, MMA_WAIT_NS);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        // epilogue: this thread's row of z2 (TMEM lane = tid), b2, SiLU, layer 3
        const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
        float out = b3[0];
#pragma unroll
        for (int cc = 0; cc < H / 16; ++cc) {
            float v[16];
            tc::tmem_ld16(trow + 16 * cc, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float z = v[e] + b2[16 * cc + e];
                out += w3[16 * cc + e] * (FIELDS ? silu_fast(z) : z * sigm(z));
            }
        }
        const float sp = x[3] * out;              // s = f3 * y
        if (FIELDS) {
            const bool ok = isfinite(sp) && fabsf(sp) <= 0.69314718f;
            if (valid) {
                const T hs = fa.h[s];
                so.seed[s] = ok ? hs * (T)__expf(sp) : hs;   // a first guess: FP32 exp suffices
            }
            const unsigned fb = __ballot_sync(0xffffffffu, valid && !ok);   // one count per warp
            if (fb && (tid & 31) == 0) atomicAdd(&cnt->hnet_fallback, __popc(fb));
        } else if (valid) {
            y[s] = sp;
        }
        tc::fence_before_sync();
        __syncthreads();                          // TMEM read and A tiles free before the next MMA
    }
    if (failed) {
        // an MMA did not complete in time: report, give it one more bounded
        // wait, then release the tensor memory
        if (tid == 0) {
            atomicOr(&cnt->hnet_err, 1u);
            tc::mbar_wait(bar_a, parity ^ 1u, MMA_WAIT_NS);
        }
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, TM_COLS);
    }
}

// ---------------------------------------------------------------- gradient
// Blocks of GT threads take chunks of GS samples.  Per chunk the three layers
// run as shared-memory products in which each thread owns a 4 x 4 tile
// (4 samples x 4 units): forward z1, a1 = silu(z1), z2 = a1 W2^T + b2,
// a2 = silu(z2), y = w3 . a2 + b3; residual r = f3 y - t, d3 = 2 r f3 / B;
// backward d2 = d3 w3 silu'(z2), d1 = (d2 W2) silu'(z1).  The W2 gradient
// sum_s d2 a1^T accumulates in a 4 x 4 register tile per thread over the
// block's chunks, the 513 smaller entries in up to three registers per
// thread; each block writes its partial gradient once, and the partials are
// reduced in a fixed order.
constexpr int GT = 256;          // threads per block
constexpr int GS = 64;           // samples per chunk
constexpr int ST = 68;           // row stride of the per-sample arrays (16-byte rows)
constexpr int NSMALL = 320 + 64 + 64 + 64 + 1;   // W1, b1, b2, W3, b3

__host__ __device__ constexpr int grad_smem_floats()
{
    return H * ST + 320 + 64 + 64 + 64 + 4 + GS * 8 + 4 * GS * ST + 2 * GS;
}

__global__ void __launch_bounds__(GT) k_grad(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ f,
                                            const float *__restrict__ t, int64_t nb, float *__restrict__ part)
{
    extern __shared__ __align__(16) float sm[];
    float *W2 = sm;                          // [n][ST]: W2[n][k]
    float *W1 = W2 + H * ST;                 // [j][5]
    float *b1 = W1 + 320, *b2 = b1 + 64, *w3 = b2 + 64, *b3 = w3 + 64;
    float *X = b3 + 4;                       // [s][8]
    float *A1 = X + GS * 8;                  // [s][ST]
    float *A2 = A1 + GS * ST;
    float *D2 = A2 + GS * ST;
    float *D1 = D2 + GS * ST;
    float *d3 = D1 + GS * ST;                // [s]
    float *ys = d3 + GS;                     // [s]
    const int tid = threadIdx.x;
    for (int k = tid; k < H * H; k += GT) W2[(k / H) * ST + k % H] = __bfloat162float(wb[O_W2 + k]);
    for (int k = tid; k < 320 + 64; k += GT) W1[k] = __bfloat162float(wb[O_W1 + k]);      // W1, b1
    for (int k = tid; k < 64 + 64 + 1; k += GT) b2[k] = __bfloat162float(wb[O_B2 + k]);  // b2, w3, b3
    __syncthreads();

    const int r0 = 4 * (tid / 16), c0 = 4 * (tid % 16);   // this thread's tile: rows r0.., columns c0..
    float gw2[4][4] = {};                                 // dL/dW2[r0 + i][c0 + j]
    float gsm[3] = {0.f, 0.f, 0.f};                       // small entries q = tid, tid + 256, tid + 512
    float lsum = 0.f;
    const float inv_b = 1.f / (float)nb;
    const int64_t nchunks = (nb + GS - 1) / GS;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t s0 = c * GS;
        for (int k = tid; k < GS * 5; k += GT) {
            const int u = k / 5, q = k % 5;
            X[u * 8 + q] = s0 + u < nb ? f[5 * (s0 + u) + q] : 0.f;
        }
        __syncthreads();
        // layer 1 (tile: samples r0.., units c0..); keep silu'(z1)
        float p1[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = c0 + j;
                float z = b1[u];
#pragma unroll
                for (int q = 0; q < 5; ++q) z += W1[5 * u + q] * X[(r0 + i) * 8 + q];
                const float sg = sigm(z);
                A1[(r0 + i) * ST + u] = z * sg;
                p1[i][j] = sg * (1.f + z * (1.f - sg));
            }
        __syncthreads();
        // layer 2 (tile: samples r0.., units c0..)
        float z2[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) z2[i][j] = b2[c0 + j];
#pragma unroll 4
        for (int k = 0; k < H; k += 4) {
            float4 av[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4 *>(A1 + (r0 + i) * ST + k);
#pragma unroll
            for (int j = 0; j < 4; ++j) wv[j] = *reinterpret_cast<const float4 *>(W2 + (c0 + j) * ST + k);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    z2[i][j] += av[i].x * wv[j].x + av[i].y * wv[j].y + av[i].z * wv[j].z + av[i].w * wv[j].w;
        }
        float p2[4][4], yp[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            yp[i] = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float z = z2[i][j], sg = sigm(z);
                const float a2 = z * sg;
                A2[(r0 + i) * ST + c0 + j] = a2;
                p2[i][j] = sg * (1.f + z * (1.f - sg));
                yp[i] += w3[c0 + j] * a2;
            }
        }
        // y: sum over the 16 threads of a row block (lanes 16 apart share none)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            for (int o = 8; o > 0; o >>= 1) yp[i] += __shfl_xor_sync(0xffffffffu, yp[i], o);
        if ((tid & 15) == 0)
#pragma unroll
            for (int i = 0; i < 4; ++i) ys[r0 + i] = b3[0] + yp[i];
        __syncthreads();
        if (tid < GS) {
            const bool valid = s0 + tid < nb;
            const float f3 = X[tid * 8 + 3];
            const float r = valid ? f3 * ys[tid] - t[s0 + tid] : 0.f;     // prediction f3 * y
            lsum += r * r;
            d3[tid] = 2.f * r * f3 * inv_b;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) D2[(r0 + i) * ST + c0 + j] = p2[i][j] * d3[r0 + i] * w3[c0 + j];
        __syncthreads();
        // backward through W2 (tile: samples r0.., inputs c0..)
        float g1[4][4] = {};
#pragma unroll 4
        for (int n = 0; n < H; n += 4) {
            float4 dv[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) dv[i] = *reinterpret_cast<const float4 *>(D2 + (r0 + i) * ST + n);
#pragma unroll
            for (int m = 0; m < 4; ++m) wv[m] = *reinterpret_cast<const float4 *>(W2 + (n + m) * ST + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                g1[i][0] += dv[i].x * wv[0].x + dv[i].y * wv[1].x + dv[i].z * wv[2].x + dv[i].w * wv[3].x;
                g1[i][1] += dv[i].x * wv[0].y + dv[i].y * wv[1].y + dv[i].z * wv[2].y + dv[i].w * wv[3].y;
                g1[i][2] += dv[i].x * wv[0].z + dv[i].y * wv[1].z + dv[i].z * wv[2].z + dv[i].w * wv[3].z;
                g1[i][3] += dv[i].x * wv[0].w + dv[i].y * wv[1].w + dv[i].z * wv[2].w + dv[i].w * wv[3].w;
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) D1[(r0 + i) * ST + c0 + j] = g1[i][j] * p1[i][j];
        __syncthreads();
        // W2 gradient: tile (outputs n = r0.., inputs k = c0..), sum over the chunk
#pragma unroll 4
        for (int u = 0; u < GS; ++u) {
            const float4 dn = *reinterpret_cast<const float4 *>(D2 + u * ST + r0);
            const float4 ak = *reinterpret_cast<const float4 *>(A1 + u * ST + c0);
            const float dd[4] = {dn.x, dn.y, dn.z, dn.w}, aa[4] = {ak.x, ak.y, ak.z, ak.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) gw2[i][j] += dd[i] * aa[j];
        }
        // the 513 small entries
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int q = tid + GT * e;
            if (q >= NSMALL) break;
            float g = 0.f;
            if (q < 320) {
                const int j = q / 5, qq = q % 5;
                for (int u = 0; u < GS; ++u) g += D1[u * ST + j] * X[u * 8 + qq];
            } else if (q < 384) {
                for (int u = 0; u < GS; ++u) g += D1[u * ST + q - 320];
            } else if (q < 448) {
                for (int u = 0; u < GS; ++u) g += D2[u * ST + q - 384];
            } else if (q < 512) {
                for (int u = 0; u < GS; ++u) g += d3[u] * A2[u * ST + q - 448];
            } else {
                for (int u = 0; u < GS; ++u) g += d3[u];
            }
            gsm[e] += g;
        }
        __syncthreads();
    }
    float *out = part + (int64_t)blockIdx.x * (NP + 1);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[O_W2 + (r0 + i) * H + c0 + j] = gw2[i][j];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int q = tid + GT * e;
        if (q >= NSMALL) break;
        out[q < 384 ? q : O_B2 + (q - 384)] = gsm[e];
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __shared__ float ls[GT / 32];
    if ((tid & 31) == 0) ls[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int k = 0; k < GT / 32; ++k) v += ls[k];
        out[NP] = v;
    }
}

__global__ void k_grad_reduce(const float *__restrict__ part, int nblk, int64_t nb, float *__restrict__ g,
                              DevCounters *cnt)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float v = 0.f;
    for (int b = 0; b < nblk; ++b) v += part[(int64_t)b * (NP + 1) + p];
    if (p < NP) g[p] = v;
    else cnt->loss = v / (float)nb;
}

// the reduction of k_grad_reduce followed by the Adam update of k_adam
__global__ void k_reduce_adam(const float *__restrict__ part, int nblk, int64_t nb, float *__restrict__ g,
                              DevCounters *cnt, float *__restrict__ th, float *__restrict__ m,
                              float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, float lr, float bc1,
                              float bc2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float gi = 0.f;
    for (int b = 0; b < nblk; ++b) gi += part[(int64_t)b * (NP + 1) + p];
    if (p == NP) {
        cnt->loss = gi / (float)nb;
        return;
    }
    g[p] = gi;
    const float mi = 0.9f * m[p] + 0.1f * gi;
    const float vi = 0.999f * v[p] + 0.001f * gi * gi;
    m[p] = mi;
    v[p] = vi;
    const float t = th[p] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    th[p] = t;
    wb[p] = __float2bfloat16_rn(t);
}

__global__ void k_adam(float *__restrict__ th, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, __nv_bfloat16 *__restrict__ wb, float lr, float bc1, float bc2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float gi = g[p];
    const float mi = 0.9f * m[p] + 0.1f * gi;
    const float vi = 0.999f * v[p] + 0.001f * gi * gi;
    m[p] = mi;
    v[p] = vi;
    const float t = th[p] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    th[p] = t;
    wb[p] = __float2bfloat16_rn(t);
}

__global__ void k_to_bf16(const float *__restrict__ th, __nv_bfloat16 *__restrict__ wb)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) wb[p] = __float2bfloat16_rn(th[p]);
}

// targets log(h_new / h_old) of the training samples i = k * stride
template <typename T>
__global__ void k_targets(const T *__restrict__ h, const T *__restrict__ hold, int64_t stride, int64_t nb,
                          float *__restrict__ st)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int64_t i = k * stride;
    st[k] = (float)log((double)h[i] / (double)hold[i]);
}

template <typename T>
FeatArgs<T> feat_args(const sph_ctx *ctx, const sph_particles *p, double dt)
{
    FeatArgs<T> fa{};
    fa.h = (const T *)p->h; fa.hprev = (const T *)p->hprev; fa.rho = (const T *)p->rho; fa.m = (const T *)p->m;
    fa.divv = (const T *)p->divv; fa.nnb = p->nnb;
    fa.dt = (float)dt; fa.eta = (float)ctx->prm.eta; fa.rho_ref = (float)ctx->prm.rho_ref;
    fa.dim = ctx->prm.dim;
    return fa;
}

// training samples of a step: every stride-th particle, at most hnet_batch
void sample_layout(const sph_ctx *ctx, int64_t n, int64_t *nb, int64_t *stride)
{
    *nb = n < ctx->prm.hnet_batch ? n : ctx->prm.hnet_batch;
    *stride = n / *nb;
    if (*stride < 1) *stride = 1;
}

size_t grad_smem() { return sizeof(float) * (size_t)grad_smem_floats(); }

}  // namespace

int hnet_init(sph_ctx *ctx)
{
    SPH_CUDA(cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
    SPH_CUDA(cudaFuncSetAttribute(k_infer_tc<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  infer_tc_smem()));
    SPH_CUDA(cudaFuncSetAttribute(k_infer_tc<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  infer_tc_smem()));
    SPH_CUDA(cudaFuncSetAttribute(k_infer_tc<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  infer_tc_smem()));
    // the persistent inference grid: the blocks that fit on an SM at once,
    // with the SM's memory split in favour of shared memory
    for (const void *f : {(const void *)k_infer_tc<false, float>, (const void *)k_infer_tc<true, float>,
                          (const void *)k_infer_tc<true, double>})
        SPH_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    int sm_smem = 0, reserved = 0;
    SPH_CUDA(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    SPH_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device));
    // what the shared memory holds and what tensor memory holds (512 columns
    // per SM, TM_COLS per block; 128 threads and ~50 registers per block are
    // never the limit), and at most four: the seed runs beside the copy back
    // and the leaf build, which need room on the same SMs (256^3 turbulence,
    // tree phase of a learned step: 5.45 ms with five blocks, 5.05 with four,
    // 5.35 with three); blocks beyond the resident ones only run later
    const int by_smem = sm_smem / (infer_tc_smem() + reserved);
    const int by_tmem = 512 / (int)TM_COLS;
    ctx->infer_per_sm = std::max(1, std::min(4, std::min(by_smem, by_tmem)));
    return SPH_OK;
}

int hnet_features(sph_ctx *ctx, const sph_particles *p, double dt, float *feats, cudaStream_t s)
{
    if (ctx->fp64)
        k_features<double><<<grid_for(p->n, 256), 256, 0, s>>>(feat_args<double>(ctx, p, dt), 1, p->n, feats);
    else
        k_features<float><<<grid_for(p->n, 256), 256, 0, s>>>(feat_args<float>(ctx, p, dt), 1, p->n, feats);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

namespace {
unsigned infer_blocks(const sph_ctx *ctx, int64_t nb)
{
    int64_t blocks = (nb + TM - 1) / TM;
    const int64_t cap = (int64_t)ctx->num_sms * ctx->infer_per_sm;   // the resident blocks
    return (unsigned)(blocks > cap ? cap : blocks);
}
}  // namespace

int hnet_infer(sph_ctx *ctx, const float *feats, int64_t nb, float *y, cudaStream_t s)
{
    if (nb <= 0) return SPH_OK;
    k_infer_tc<false, float><<<infer_blocks(ctx, nb), TM, infer_tc_smem(), s>>>(ctx->hn_bf16, feats, FeatArgs<float>{},
                                                                               nb, y, SeedOut<float>{}, ctx->dcnt,
                                                                               ctx->test_flags & SPH_TEST_SKIP_MMA);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

template <typename T>
int seed_impl(sph_ctx *ctx, const sph_particles *p, double dt, bool train, void *h_seed, cudaStream_t s)
{
    SeedOut<T> so{(T *)h_seed};
    k_infer_tc<true, T><<<infer_blocks(ctx, p->n), TM, infer_tc_smem(), s>>>(
        ctx->hn_bf16, nullptr, feat_args<T>(ctx, p, dt), p->n, nullptr, so, ctx->dcnt,
        ctx->test_flags & SPH_TEST_SKIP_MMA);
    SPH_CHECK_LAUNCH();
    if (train) SPH_TRY(hnet_sample_features(ctx, p, dt, s));
    return SPH_OK;
}

// the step's seed h exp(s) straight from the particle fields (features, network
// and seed in one kernel); with train, the features of the training samples too
int hnet_seed_from_fields(sph_ctx *ctx, const sph_particles *p, double dt, bool train, void *h_seed,
                          cudaStream_t s)
{
    return ctx->fp64 ? seed_impl<double>(ctx, p, dt, train, h_seed, s) : seed_impl<float>(ctx, p, dt, train, h_seed, s);
}

// features of the training samples only (a step that trains without seeding)
int hnet_sample_features(sph_ctx *ctx, const sph_particles *p, double dt, cudaStream_t s)
{
    int64_t nb, stride;
    sample_layout(ctx, p->n, &nb, &stride);
    if (ctx->fp64)
        k_features<double><<<grid_for(nb, 256), 256, 0, s>>>(feat_args<double>(ctx, p, dt), stride, nb, ctx->hn_sample);
    else
        k_features<float><<<grid_for(nb, 256), 256, 0, s>>>(feat_args<float>(ctx, p, dt), stride, nb, ctx->hn_sample);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

int hnet_grad(sph_ctx *ctx, const float *feats, const float *target, int64_t nb, cudaStream_t s)
{
    int64_t blocks = (nb + GS - 1) / GS;
    if (blocks > ctx->hn_part_blocks) blocks = ctx->hn_part_blocks;
    if (blocks < 1) blocks = 1;
    k_grad<<<(unsigned)blocks, GT, grad_smem(), s>>>(ctx->hn_bf16, feats, target, nb, ctx->hn_part);
    SPH_CHECK_LAUNCH();
    k_grad_reduce<<<grid_for(NP + 1, 256), 256, 0, s>>>(ctx->hn_part, (int)blocks, nb, ctx->hn_grad, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

int hnet_adam(sph_ctx *ctx, float lr, cudaStream_t s)
{
    ctx->hn_step += 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)ctx->hn_step));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)ctx->hn_step));
    k_adam<<<grid_for(NP, 256), 256, 0, s>>>(ctx->hn_master, ctx->hn_m, ctx->hn_v, ctx->hn_grad, ctx->hn_bf16, lr,
                                             bc1, bc2);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

int hnet_refresh_bf16(sph_ctx *ctx, cudaStream_t s)
{
    k_to_bf16<<<grid_for(NP, 256), 256, 0, s>>>(ctx->hn_master, ctx->hn_bf16);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

// one online training round on the samples whose features the seeding (or
// hnet_sample_features) recorded, with targets log(h_new / h_old)
int hnet_online(sph_ctx *ctx, const sph_particles *p, cudaStream_t s)
{
    int64_t nb, stride;
    sample_layout(ctx, p->n, &nb, &stride);
    float *sf = ctx->hn_sample, *st = ctx->hn_sample + 5 * (int64_t)ctx->prm.hnet_batch;
    if (ctx->fp64)
        k_targets<double><<<grid_for(nb, 256), 256, 0, s>>>((const double *)p->h, (const double *)ctx->hold, stride,
                                                            nb, st);
    else
        k_targets<float><<<grid_for(nb, 256), 256, 0, s>>>((const float *)p->h, (const float *)ctx->hold, stride,
                                                           nb, st);
    SPH_CHECK_LAUNCH();
    int64_t blocks = (nb + GS - 1) / GS;
    if (blocks > ctx->hn_part_blocks) blocks = ctx->hn_part_blocks;
    if (blocks < 1) blocks = 1;
    for (int it = 0; it < ctx->prm.hnet_iters; ++it) {
        k_grad<<<(unsigned)blocks, GT, grad_smem(), s>>>(ctx->hn_bf16, sf, st, nb, ctx->hn_part);
        SPH_CHECK_LAUNCH();
        ctx->hn_step += 1;
        const float bc1 = (float)(1.0 - std::pow(0.9, (double)ctx->hn_step));
        const float bc2 = (float)(1.0 - std::pow(0.999, (double)ctx->hn_step));
        k_reduce_adam<<<grid_for(NP + 1, 256), 256, 0, s>>>(ctx->hn_part, (int)blocks, nb, ctx->hn_grad, ctx->dcnt,
                                                            ctx->hn_master, ctx->hn_m, ctx->hn_v, ctx->hn_bf16,
                                                            (float)ctx->prm.hnet_lr, bc1, bc2);
        SPH_CHECK_LAUNCH();
    }
    return SPH_OK;
}
