// h-predictor network (not part of the paper's method; it only seeds the
// h-rho iteration of Eq. 9, which stays the judge of the converged h):
//   y = W3 silu(W2 silu(W1 f + b1) + b2) + b3,  5 -> 64 -> 64 -> 1,
// BF16 weights read by the kernels, FP32 master weights and Adam moments,
// FP32 activations and accumulation.  The prediction of log(h_next / h) is
// s = f3 * y with f3 = div v * dt: a particle at rest keeps its h exactly, and
// the network learns the gain of the continuity estimate div v dt / 3.
#include <cmath>

#include "sph_internal.cuh"

namespace {

constexpr int NP = SPH_HNET_NPARAM;
constexpr int O_W1 = 0, O_B1 = 320, O_W2 = 384, O_B2 = 4480, O_W3 = 4544, O_B3 = 4608;
constexpr int H = 64;

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + __expf(-z)); }

__device__ void load_weights(const __nv_bfloat16 *__restrict__ w, float *s)
{
    for (int k = threadIdx.x; k < NP; k += blockDim.x) s[k] = __bfloat162float(w[k]);
    __syncthreads();
}

// ---------------------------------------------------------------- features
// f0 = log(h / hbar), hbar = eta (m / rho_ref)^(1/3)
// f1 = log(max(nnb, 1/2) / nbar), nbar = 32 pi eta^3 / 3
// f2 = log(rho h^3 / (m eta^3))
// f3 = div v * dt
// f4 = log(h / hprev)  (0 when hprev <= 0)
template <typename T>
__global__ void k_features(const T *__restrict__ h, const T *__restrict__ hprev, const int32_t *__restrict__ nnb,
                           const T *__restrict__ rho, const T *__restrict__ m, const T *__restrict__ divv,
                           int64_t n, float dt, float eta, float rho_ref, float *__restrict__ f)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float hi = (float)h[i], mi = (float)m[i], ri = (float)rho[i];
    const float eta3 = eta * eta * eta;
    const float hbar = eta * cbrtf(mi / rho_ref);
    const float nbar = 32.f * 3.14159265358979f * eta3 / 3.f;
    const float nb = fmaxf((float)nnb[i], 0.5f);
    const float hp = (float)hprev[i];
    float *o = f + 5 * i;
    o[0] = logf(hi / hbar);
    o[1] = logf(nb / nbar);
    o[2] = logf(ri * hi * hi * hi / (mi * eta3));
    o[3] = (float)divv[i] * dt;
    o[4] = hp > 0.f ? logf(hi / hp) : 0.f;
}

// ---------------------------------------------------------------- inference
// One thread per sample.  Half of the 64 layer-2 pre-activations at a time
// stay in registers; the layer-1 units are recomputed for each half (5 FMAs
// each) and scattered into them through the transposed W2 held in shared
// memory (float4 broadcast reads).
constexpr int HALF = H / 2;

__global__ void __launch_bounds__(256, 3) k_infer(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ f,
                                                  int64_t nb, float *__restrict__ y)
{
    __shared__ __align__(16) float w[NP + 3];
    for (int k = threadIdx.x; k < NP; k += blockDim.x) {
        int dst = k;
        if (k >= O_W2 && k < O_B2) {              // store W2 transposed: [k][j]
            const int j = (k - O_W2) / H, c = (k - O_W2) % H;
            dst = O_W2 + H * c + j;
        }
        w[dst] = __bfloat162float(wb[k]);
    }
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nb; s += (int64_t)gridDim.x * blockDim.x) {
        float x[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) x[k] = f[5 * s + k];
        float out = w[O_B3];
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            float z2[HALF];
#pragma unroll
            for (int j = 0; j < HALF; ++j) z2[j] = w[O_B2 + half * HALF + j];
#pragma unroll 1
            for (int k = 0; k < H; ++k) {
                float z = w[O_B1 + k];
#pragma unroll
                for (int c = 0; c < 5; ++c) z += w[O_W1 + 5 * k + c] * x[c];
                const float a = z * sigm(z);
                const float4 *col = reinterpret_cast<const float4 *>(w + O_W2 + H * k + half * HALF);
#pragma unroll
                for (int j = 0; j < HALF / 4; ++j) {
                    const float4 r = col[j];
                    z2[4 * j] += r.x * a;
                    z2[4 * j + 1] += r.y * a;
                    z2[4 * j + 2] += r.z * a;
                    z2[4 * j + 3] += r.w * a;
                }
            }
#pragma unroll
            for (int j = 0; j < HALF; ++j) out += w[O_W3 + half * HALF + j] * (z2[j] * sigm(z2[j]));
        }
        y[s] = x[3] * out;                      // s = f3 * y
    }
}

// ---------------------------------------------------------------- gradient
// Each block processes chunks of S samples: one thread per sample runs the
// forward and backward pass and leaves x, a1, a2, d1, d2 (d = dL/dz) in shared
// memory; then every thread accumulates a fixed subset of the 4609 gradient
// entries over the chunk.  Block partials are reduced in a fixed order.
constexpr int GS = 64;           // samples per chunk = threads per block
constexpr int ST = 65;           // row stride (conflict-free)

__global__ void __launch_bounds__(GS) k_grad(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ f,
                                            const float *__restrict__ t, int64_t nb, float *__restrict__ part)
{
    extern __shared__ __align__(16) float sm[];
    float *w = sm;                           // NP (+3)
    float *sx = w + NP + 3;                  // GS x 5
    float *sa1 = sx + GS * 5;                // GS x ST
    float *sa2 = sa1 + GS * ST;
    float *sd1 = sa2 + GS * ST;
    float *sd2 = sd1 + GS * ST;
    float *sd3 = sd2 + GS * ST;              // GS
    load_weights(wb, w);
    const int tid = threadIdx.x;
    // this block's partial row; entries p = tid, tid + GS, ... belong to this thread
    float *out = part + (int64_t)blockIdx.x * (NP + 1);
    for (int p = tid; p < NP; p += GS) out[p] = 0.f;
    float lsum = 0.f;
    const float inv_b = 1.f / (float)nb;
    const int64_t nchunks = (nb + GS - 1) / GS;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t s = c * GS + tid;
        const bool valid = s < nb;
        float x[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) x[k] = valid ? f[5 * s + k] : 0.f;
        float *a1 = sa1 + tid * ST, *a2 = sa2 + tid * ST, *d1 = sd1 + tid * ST, *d2 = sd2 + tid * ST;
        for (int j = 0; j < H; ++j) {
            float z = w[O_B1 + j];
#pragma unroll
            for (int k = 0; k < 5; ++k) z += w[O_W1 + 5 * j + k] * x[k];
            d1[j] = z;                       // keep z1 until the backward pass
            a1[j] = z * sigm(z);
        }
        float y = w[O_B3];
        for (int j = 0; j < H; ++j) {
            float z = w[O_B2 + j];
            for (int k = 0; k < H; ++k) z += w[O_W2 + H * j + k] * a1[k];
            const float sg = sigm(z);
            a2[j] = z * sg;
            d2[j] = sg * (1.f + z * (1.f - sg));   // silu'(z2), scaled below
            y += w[O_W3 + j] * a2[j];
        }
        const float r = valid ? x[3] * y - t[s] : 0.f;      // prediction f3 * y
        lsum += r * r;
        const float d3 = 2.f * r * x[3] * inv_b;
        sd3[tid] = d3;
        for (int j = 0; j < H; ++j) d2[j] *= d3 * w[O_W3 + j];
        for (int k = 0; k < H; ++k) {
            float g = 0.f;
            for (int j = 0; j < H; ++j) g += w[O_W2 + H * j + k] * d2[j];
            const float z = d1[k];
            const float sg = sigm(z);
            d1[k] = g * sg * (1.f + z * (1.f - sg));
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) sx[tid * 5 + k] = x[k];
        __syncthreads();
#pragma unroll 1
        for (int p = tid; p < NP; p += GS) {
            float g = 0.f;
            if (p < O_B1) {                          // W1[j][k]
                const int j = p / 5, k = p % 5;
                for (int u = 0; u < GS; ++u) g += sd1[u * ST + j] * sx[u * 5 + k];
            } else if (p < O_W2) {                   // b1[j]
                const int j = p - O_B1;
                for (int u = 0; u < GS; ++u) g += sd1[u * ST + j];
            } else if (p < O_B2) {                   // W2[j][k]
                const int j = (p - O_W2) / H, k = (p - O_W2) % H;
                for (int u = 0; u < GS; ++u) g += sd2[u * ST + j] * sa1[u * ST + k];
            } else if (p < O_W3) {                   // b2[j]
                const int j = p - O_B2;
                for (int u = 0; u < GS; ++u) g += sd2[u * ST + j];
            } else if (p < O_B3) {                   // W3[0][j]
                const int j = p - O_W3;
                for (int u = 0; u < GS; ++u) g += sd3[u] * sa2[u * ST + j];
            } else {                                 // b3
                for (int u = 0; u < GS; ++u) g += sd3[u];
            }
            out[p] += g;
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    __shared__ float ls[GS / 32];
    if ((tid & 31) == 0) ls[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int k = 0; k < GS / 32; ++k) v += ls[k];
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

// h seed = h exp(y); a non-finite y or a change beyond a factor 2 keeps h.
template <typename T>
__global__ void k_seed(const T *__restrict__ h, const float *__restrict__ y, int64_t n, T *__restrict__ seed,
                       DevCounters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = y[i];
    const bool ok = isfinite(s) && fabsf(s) <= 0.69314718f;
    seed[i] = ok ? (T)((double)h[i] * exp((double)s)) : h[i];
    if (!ok) atomicAdd(&cnt->hnet_fallback, 1);
}

// strided subset of the step's features with targets log(h_new / h_old)
template <typename T>
__global__ void k_sample(const float *__restrict__ feats, const T *__restrict__ h, const T *__restrict__ hold,
                         int64_t n, int64_t stride, int64_t nb, float *__restrict__ sf, float *__restrict__ st)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const int64_t i = (k * stride) % n;
#pragma unroll
    for (int c = 0; c < 5; ++c) sf[5 * k + c] = feats[5 * i + c];
    st[k] = (float)log((double)h[i] / (double)hold[i]);
}

size_t grad_smem() { return sizeof(float) * (NP + 3 + GS * 5 + 4 * GS * ST + GS); }

}  // namespace

int hnet_init(sph_ctx *ctx)
{
    SPH_CUDA(cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem()));
    return SPH_OK;
}

int hnet_features(sph_ctx *ctx, const sph_particles *p, double dt, float *feats, cudaStream_t s)
{
    const float eta = (float)ctx->prm.eta, rr = (float)ctx->prm.rho_ref;
    if (ctx->fp64)
        k_features<double><<<grid_for(p->n, 256), 256, 0, s>>>((const double *)p->h, (const double *)p->hprev, p->nnb,
                                                               (const double *)p->rho, (const double *)p->m,
                                                               (const double *)p->divv, p->n, (float)dt, eta, rr, feats);
    else
        k_features<float><<<grid_for(p->n, 256), 256, 0, s>>>((const float *)p->h, (const float *)p->hprev, p->nnb,
                                                              (const float *)p->rho, (const float *)p->m,
                                                              (const float *)p->divv, p->n, (float)dt, eta, rr, feats);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

int hnet_infer(sph_ctx *ctx, const float *feats, int64_t nb, float *y, cudaStream_t s)
{
    int64_t blocks = (nb + 255) / 256;
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_infer<<<(unsigned)blocks, 256, 0, s>>>(ctx->hn_bf16, feats, nb, y);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

int hnet_grad(sph_ctx *ctx, const float *feats, const float *target, int64_t nb, cudaStream_t s)
{
    int64_t blocks = (nb + GS - 1) / GS;
    if (blocks > ctx->hn_part_blocks) blocks = ctx->hn_part_blocks;
    if (blocks < 1) blocks = 1;
    k_grad<<<(unsigned)blocks, GS, grad_smem(), s>>>(ctx->hn_bf16, feats, target, nb, ctx->hn_part);
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

int hnet_online(sph_ctx *ctx, const sph_particles *p, cudaStream_t s)
{
    const int64_t n = p->n;
    const int64_t nb = n < ctx->prm.hnet_batch ? n : ctx->prm.hnet_batch;
    int64_t stride = n / nb;
    if (stride < 1) stride = 1;
    float *sf = ctx->hn_sample, *st = ctx->hn_sample + 5 * (int64_t)ctx->prm.hnet_batch;
    if (ctx->fp64)
        k_sample<double><<<grid_for(nb, 256), 256, 0, s>>>(ctx->feats, (const double *)p->h, (const double *)ctx->hold,
                                                           n, stride, nb, sf, st);
    else
        k_sample<float><<<grid_for(nb, 256), 256, 0, s>>>(ctx->feats, (const float *)p->h, (const float *)ctx->hold,
                                                          n, stride, nb, sf, st);
    SPH_CHECK_LAUNCH();
    for (int it = 0; it < ctx->prm.hnet_iters; ++it) {
        SPH_TRY(hnet_grad(ctx, sf, st, nb, s));
        SPH_TRY(hnet_adam(ctx, (float)ctx->prm.hnet_lr, s));
    }
    return SPH_OK;
}

int hnet_seed(sph_ctx *ctx, sph_particles *p, const float *y, void *h_seed, cudaStream_t s)
{
    if (ctx->fp64)
        k_seed<double><<<grid_for(p->n, 256), 256, 0, s>>>((const double *)p->h, y, p->n, (double *)h_seed, ctx->dcnt);
    else
        k_seed<float><<<grid_for(p->n, 256), 256, 0, s>>>((const float *)p->h, y, p->n, (float *)h_seed, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}
