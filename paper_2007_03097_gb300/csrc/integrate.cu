// Kick-drift-kick leapfrog around the right-hand side (the paper names no
// integrator), FP64 position update and periodic wrap, and deterministic FP64
// totals: sum m v, sum m a, sum m (v^2/2 + u), sum m (v . a + du/dt) and the
// CFL minimum of h / vsig.
#include <cfloat>
#include <type_traits>

#include "dfloat.cuh"
#include "sph_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ T kinetic(T vx, T vy, T vz) { return T(0.5) * (vx * vx + vy * vy + vz * vz); }

// First half kick and drift.  thermo: du holds de/dt; e = u + v^2/2 gets the
// half kick and u = e - v_half^2/2.
// p wrapped into [0, L) as `if (p >= L) p -= L; else if (p < 0) p += L`
__device__ __forceinline__ double wrap_origin(double p, double L)
{
    const long long b = __double_as_longlong(p);
    if (b >= __double_as_longlong(L)) return p - L;
    if (b < 0 && b != (long long)0x8000000000000000ull) return p + L;
    return p;
}

template <typename T>
__global__ void k_kick_drift(double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             T *__restrict__ vx, T *__restrict__ vy, T *__restrict__ vz, T *__restrict__ u,
                             const T *__restrict__ ax, const T *__restrict__ ay, const T *__restrict__ az,
                             const T *__restrict__ du, int64_t n, double dt, int periodic, double3 lo,
                             double3 hi, int thermo, DevCounters *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the step's h-predictor counters start at zero (this is the step's
    // first kernel; the seeding also zeroes them on its own stream)
    if (i == 0) { cnt->hnet_fallback = 0; cnt->hnet_err = 0; }
    if (i >= n) return;
    const T hdt = (T)(0.5 * dt);
    const T vx0 = vx[i], vy0 = vy[i], vz0 = vz[i];
    const T vxh = vx0 + ax[i] * hdt, vyh = vy0 + ay[i] * hdt, vzh = vz0 + az[i] * hdt;
    vx[i] = vxh; vy[i] = vyh; vz[i] = vzh;
    if (thermo) u[i] = (u[i] + kinetic(vx0, vy0, vz0) + du[i] * hdt) - kinetic(vxh, vyh, vzh);
    else u[i] = u[i] + du[i] * hdt;
    double px = x[i] + (double)vxh * dt, py = y[i] + (double)vyh * dt, pz = z[i] + (double)vzh * dt;
    if (periodic == 2) {
        // box [0, L)^3: the same decisions from the bits (IEEE order is the
        // integer order for non-negative doubles; -0 is not below 0), which
        // keeps the FP64 pipe, 1/64 of the FP32 rate on GB300, for the drift
        px = wrap_origin(px, hi.x);
        py = wrap_origin(py, hi.y);
        pz = wrap_origin(pz, hi.z);
    } else if (periodic) {
        if (px >= hi.x) px -= hi.x - lo.x; else if (px < lo.x) px += hi.x - lo.x;
        if (py >= hi.y) py -= hi.y - lo.y; else if (py < lo.y) py += hi.y - lo.y;
        if (pz >= hi.z) pz -= hi.z - lo.z; else if (pz < lo.z) pz += hi.z - lo.z;
    }
    x[i] = px; y[i] = py; z[i] = pz;
}

// predicted v and u at the end of the step from the old rates (thermo: the
// predicted e = u_half + v_half^2/2 + de dt/2, u_pred = e_pred - v_pred^2/2)
template <typename T>
__global__ void k_predict(const T *__restrict__ vx, const T *__restrict__ vy, const T *__restrict__ vz,
                          const T *__restrict__ u, const T *__restrict__ ax, const T *__restrict__ ay,
                          const T *__restrict__ az, const T *__restrict__ du, int64_t n, double dt,
                          T *__restrict__ px, T *__restrict__ py, T *__restrict__ pz, T *__restrict__ pu,
                          int thermo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T hdt = (T)(0.5 * dt);
    const T vxh = vx[i], vyh = vy[i], vzh = vz[i];
    const T vxp = vxh + ax[i] * hdt, vyp = vyh + ay[i] * hdt, vzp = vzh + az[i] * hdt;
    px[i] = vxp;
    py[i] = vyp;
    pz[i] = vzp;
    if (thermo) pu[i] = (u[i] + kinetic(vxh, vyh, vzh) + du[i] * hdt) - kinetic(vxp, vyp, vzp);
    else pu[i] = u[i] + du[i] * hdt;
}

// closing half kick (thermo: e = u_half + v_half^2/2 + de dt/2, u = e - v^2/2)
template <typename T>
__global__ void k_kick(T *__restrict__ vx, T *__restrict__ vy, T *__restrict__ vz, T *__restrict__ u,
                       const T *__restrict__ ax, const T *__restrict__ ay, const T *__restrict__ az,
                       const T *__restrict__ du, int64_t n, double dt, int thermo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T hdt = (T)(0.5 * dt);
    const T vxh = vx[i], vyh = vy[i], vzh = vz[i];
    const T vx1 = vxh + ax[i] * hdt, vy1 = vyh + ay[i] * hdt, vz1 = vzh + az[i] * hdt;
    vx[i] = vx1;
    vy[i] = vy1;
    vz[i] = vz1;
    if (thermo) u[i] = (u[i] + kinetic(vxh, vyh, vzh) + du[i] * hdt) - kinetic(vx1, vy1, vz1);
    else u[i] = u[i] + du[i] * hdt;
}

constexpr int NT = 9;    // 8 sums + 1 min
constexpr int TB = 256;  // threads per block of the partial-totals kernel

// Per-block partial totals in FP64 (fixed grid, fixed order: deterministic).
// FP64 runs at 1/64 of the FP32 rate, so the kernel spends few FP64
// instructions: the quotient h / v_sig is formed only where it can lower the
// running minimum mn, i.e. where h <= mn v_sig (tested against
// mn (1 + 2^-40) v_sig, which rounding cannot push below the exact mn v_sig),
// and the per-thread sums meet in shared memory, warp k reducing quantity k.
template <typename T>
__global__ void __launch_bounds__(TB) k_totals_partial(
    const T *__restrict__ m, const T *__restrict__ vx, const T *__restrict__ vy, const T *__restrict__ vz,
    const T *__restrict__ u, const T *__restrict__ ax, const T *__restrict__ ay, const T *__restrict__ az,
    const T *__restrict__ du, const T *__restrict__ pvx, const T *__restrict__ pvy, const T *__restrict__ pvz,
    const T *__restrict__ h, const T *__restrict__ vsig, int64_t n, double *__restrict__ part, int thermo)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double mn = DBL_MAX, mnx = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    for (int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        const double mi = m[i], vxi = vx[i], vyi = vy[i], vzi = vz[i];
        const double axi = ax[i], ayi = ay[i], azi = az[i];
        acc[0] += mi * vxi; acc[1] += mi * vyi; acc[2] += mi * vzi;
        acc[3] += mi * axi; acc[4] += mi * ayi; acc[5] += mi * azi;
        acc[6] += mi * (0.5 * (vxi * vxi + vyi * vyi + vzi * vzi) + (double)u[i]);
        const double wx = pvx ? (double)pvx[i] : vxi, wy = pvx ? (double)pvy[i] : vyi, wz = pvx ? (double)pvz[i] : vzi;
        acc[7] += thermo ? mi * (double)du[i] : mi * (wx * axi + wy * ayi + wz * azi + (double)du[i]);
        if (vsig) {
            const double v = vsig[i], hi = h[i];
            if (v > 0 && hi <= mnx * v) {
                mn = fmin(mn, hi / v);
                mnx = mn * (1.0 + 0x1p-40);
            }
        }
    }
    __shared__ double s[NT][TB];
    for (int k = 0; k < 8; ++k) s[k][threadIdx.x] = acc[k];
    s[8][threadIdx.x] = mn;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < NT; k += TB / 32) {
        double v = s[k][lane];
        for (int j = lane + 32; j < TB; j += 32) v = k < 8 ? v + s[k][j] : fmin(v, s[k][j]);
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = k < 8 ? v + w : fmin(v, w);
        }
        if (lane == 0) part[blockIdx.x * NT + k] = v;
    }
}

// SPH_MIXED partial totals: every field is FP32, so each product is exact as
// a two-float (two_prod) and the per-thread sums run in double-float on the
// FP32 pipes (~2^-44 relative per addition, FP64 would take 1/64 of the FP32
// rate); the thread sums meet in FP64 in shared memory as in
// k_totals_partial, and the quotient h / v_sig is FP64 where it can lower the
// running minimum.
__global__ void __launch_bounds__(TB) k_totals_partial_f32(
    const float *__restrict__ m, const float *__restrict__ vx, const float *__restrict__ vy,
    const float *__restrict__ vz, const float *__restrict__ u, const float *__restrict__ ax,
    const float *__restrict__ ay, const float *__restrict__ az, const float *__restrict__ du,
    const float *__restrict__ pvx, const float *__restrict__ pvy, const float *__restrict__ pvz,
    const float *__restrict__ h, const float *__restrict__ vsig, int64_t n, double *__restrict__ part, int thermo)
{
    df acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = df{0.f, 0.f};
    double mn = DBL_MAX, mnx = __longlong_as_double(0x7ff0000000000000ll);   // +inf
    float mnf = __int_as_float(0x7f800000);                                    // +inf
    for (int64_t i = (int64_t)blockIdx.x * TB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TB) {
        const float mi = m[i], vxi = vx[i], vyi = vy[i], vzi = vz[i];
        const float axi = ax[i], ayi = ay[i], azi = az[i];
        acc[0] = df_add(acc[0], two_prod(mi, vxi));
        acc[1] = df_add(acc[1], two_prod(mi, vyi));
        acc[2] = df_add(acc[2], two_prod(mi, vzi));
        acc[3] = df_add(acc[3], two_prod(mi, axi));
        acc[4] = df_add(acc[4], two_prod(mi, ayi));
        acc[5] = df_add(acc[5], two_prod(mi, azi));
        // m (v^2/2 + u) from the exact squares
        const df v2 = df_add(df_add(two_prod(vxi, vxi), two_prod(vyi, vyi)), two_prod(vzi, vzi));
        acc[6] = df_add(acc[6], df_mul_f(df_add_f(df_scale(v2, 0.5f), u[i]), mi));
        const float wx = pvx ? pvx[i] : vxi, wy = pvx ? pvy[i] : vyi, wz = pvx ? pvz[i] : vzi;
        if (thermo) {
            acc[7] = df_add(acc[7], two_prod(mi, du[i]));
        } else {
            const df wa = df_add(df_add(two_prod(wx, axi), two_prod(wy, ayi)), two_prod(wz, azi));
            acc[7] = df_add(acc[7], df_mul_f(df_add_f(wa, du[i]), mi));
        }
        if (vsig) {
            // an FP32 screen (the threshold grown by 2^-20, far beyond the
            // FP32 product's rounding) keeps the FP64 test and quotient for
            // the few particles that can lower the minimum
            const float vf = vsig[i], hf = h[i];
            if (vf > 0.f && hf <= mnf * vf) {
                const double v = vf, hi = hf;
                if (hi <= mnx * v) {
                    mn = fmin(mn, hi / v);
                    mnx = mn * (1.0 + 0x1p-40);
                    mnf = (float)mnx * (1.f + 0x1p-20f);
                }
            }
        }
    }
    __shared__ double s[NT][TB];
    for (int k = 0; k < 8; ++k) s[k][threadIdx.x] = (double)acc[k].hi + (double)acc[k].lo;
    s[8][threadIdx.x] = mn;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int k = threadIdx.x >> 5; k < NT; k += TB / 32) {
        double v = s[k][lane];
        for (int j = lane + 32; j < TB; j += 32) v = k < 8 ? v + s[k][j] : fmin(v, s[k][j]);
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = k < 8 ? v + w : fmin(v, w);
        }
        if (lane == 0) part[blockIdx.x * NT + k] = v;
    }
}

// Block partials combined in a fixed order: warp k sums quantity k over the
// partials with a strided loop and a shuffle tree (deterministic).
__global__ void k_totals_final(const double *__restrict__ part, int nb, DevCounters *cnt)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= NT) return;
    double v = k < 8 ? 0.0 : DBL_MAX;
    for (int b = lane; b < nb; b += 32) v = k < 8 ? v + part[b * NT + k] : fmin(v, part[b * NT + k]);
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = k < 8 ? v + w : fmin(v, w);
    }
    if (lane == 0) {
        if (k < 8) cnt->totals[k] = v;
        else cnt->min_dt = v;
    }
}

template <typename T>
int kd_impl(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s)
{
    const sph_params &q = ctx->prm;
    k_kick_drift<T><<<grid_for(p->n, 256), 256, 0, s>>>(
        p->x, p->y, p->z, (T *)p->vx, (T *)p->vy, (T *)p->vz, (T *)p->u, (const T *)p->ax, (const T *)p->ay,
        (const T *)p->az, (const T *)p->dudt, p->n, dt,
        q.periodic ? (q.box_lo[0] == 0.0 && q.box_lo[1] == 0.0 && q.box_lo[2] == 0.0 ? 2 : 1) : 0,
        make_double3(q.box_lo[0], q.box_lo[1], q.box_lo[2]),
        make_double3(q.box_hi[0], q.box_hi[1], q.box_hi[2]), q.energy == SPH_ENERGY_TOTAL, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

template <typename T>
int pred_impl(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s)
{
    k_predict<T><<<grid_for(p->n, 256), 256, 0, s>>>(
        (const T *)p->vx, (const T *)p->vy, (const T *)p->vz, (const T *)p->u, (const T *)p->ax, (const T *)p->ay,
        (const T *)p->az, (const T *)p->dudt, p->n, dt, (T *)ctx->vpx, (T *)ctx->vpy, (T *)ctx->vpz, (T *)ctx->upred,
        ctx->prm.energy == SPH_ENERGY_TOTAL);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

template <typename T>
int kick_impl(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s)
{
    k_kick<T><<<grid_for(p->n, 256), 256, 0, s>>>((T *)p->vx, (T *)p->vy, (T *)p->vz, (T *)p->u, (const T *)p->ax,
                                                  (const T *)p->ay, (const T *)p->az, (const T *)p->dudt, p->n, dt,
                                                  ctx->prm.energy == SPH_ENERGY_TOTAL);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

template <typename T>
int totals_impl(sph_ctx *ctx, const sph_particles *p, const void *pvx, const void *pvy, const void *pvz,
                const void *u, cudaStream_t s)
{
    const int nb = ctx->red_blocks;
    if constexpr (std::is_same<T, float>::value)
        k_totals_partial_f32<<<nb, TB, 0, s>>>(p->m ? (const float *)p->m : nullptr, (const float *)p->vx,
                                                (const float *)p->vy, (const float *)p->vz, (const float *)u,
                                                (const float *)p->ax, (const float *)p->ay, (const float *)p->az,
                                                (const float *)p->dudt, (const float *)pvx, (const float *)pvy,
                                                (const float *)pvz, (const float *)p->h, (const float *)p->vsig,
                                                p->n, ctx->red, ctx->prm.energy == SPH_ENERGY_TOTAL);
    else
        k_totals_partial<T><<<nb, TB, 0, s>>>((const T *)p->m, (const T *)p->vx, (const T *)p->vy, (const T *)p->vz,
                                               (const T *)u, (const T *)p->ax, (const T *)p->ay, (const T *)p->az,
                                               (const T *)p->dudt, (const T *)pvx, (const T *)pvy, (const T *)pvz,
                                               (const T *)p->h, (const T *)p->vsig, p->n, ctx->red,
                                               ctx->prm.energy == SPH_ENERGY_TOTAL);
    SPH_CHECK_LAUNCH();
    k_totals_final<<<1, 32 * NT, 0, s>>>(ctx->red, nb, ctx->dcnt);
    SPH_CHECK_LAUNCH();
    return SPH_OK;
}

}  // namespace

int kick_drift(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s)
{
    return ctx->fp64 ? kd_impl<double>(ctx, p, dt, s) : kd_impl<float>(ctx, p, dt, s);
}

int predict(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s)
{
    return ctx->fp64 ? pred_impl<double>(ctx, p, dt, s) : pred_impl<float>(ctx, p, dt, s);
}

int kick(sph_ctx *ctx, sph_particles *p, double dt, cudaStream_t s)
{
    return ctx->fp64 ? kick_impl<double>(ctx, p, dt, s) : kick_impl<float>(ctx, p, dt, s);
}

// totals of p with u; power uses the predicted velocities (pvx..) when given
int totals_run(sph_ctx *ctx, const sph_particles *p, const void *pvx, const void *pvy, const void *pvz,
               const void *u, cudaStream_t s)
{
    return ctx->fp64 ? totals_impl<double>(ctx, p, pvx, pvy, pvz, u, s)
                     : totals_impl<float>(ctx, p, pvx, pvy, pvz, u, s);
}

int sync_counters(sph_ctx *ctx, cudaStream_t s)
{
    SPH_CUDA(cudaMemcpyAsync(ctx->hcnt, ctx->dcnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    return SPH_OK;
}
