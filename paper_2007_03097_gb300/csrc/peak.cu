// FP32 pipe calibration: the rate of independent fused multiply-add chains
// on this GPU, the measured ceiling of the pair kernels (which are bound by
// the FP32 pipe and by instruction issue, not by memory).  The paper has no
// counterpart; it is a measurement of the hardware the library runs on.
#include <cuda_runtime.h>

#include "sph.h"

namespace {

constexpr int CHAINS = 8;       // independent chains per thread (covers the FMA latency)
constexpr int THREADS = 256;
constexpr int BLOCKS_PER_SM = 8;

// each chain iterates v <- v * b + c, whose fixed point c / (1 - b) = 1 keeps
// the values bounded; one store per thread keeps the chains alive
__global__ void __launch_bounds__(THREADS) k_fma_chains(float *out, int iters, float b, float c)
{
    float v[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) v[j] = 1.0f + 1e-3f * (float)j + 1e-7f * (float)threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CHAINS; ++j) v[j] = fmaf(v[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) s += v[j];
    out[(size_t)blockIdx.x * THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" int sph_peak_fp32(double *tflops, double *ms_out, void *stream)
{
    if (!tflops) return SPH_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SPH_ERR_CUDA;
    const int blocks = sms * BLOCKS_PER_SM;
    const int iters = 1 << 15;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = SPH_OK;
    double best = 0.0, best_ms = 0.0;
    if (cudaMalloc(&out, (size_t)blocks * THREADS * sizeof(float)) != cudaSuccess) return SPH_ERR_CUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        status = SPH_ERR_CUDA;
    } else {
        // one warm-up launch, then the best of five timed ones
        for (int rep = 0; rep < 6 && status == SPH_OK; ++rep) {
            cudaEventRecord(e0, s);
            k_fma_chains<<<blocks, THREADS, 0, s>>>(out, iters, 0.999f, 0.001f);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                status = SPH_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double flops = 2.0 * CHAINS * (double)iters * (double)blocks * THREADS;
            const double tf = flops / (ms * 1e-3) / 1e12;
            if (rep > 0 && tf > best) {
                best = tf;
                best_ms = ms;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (status != SPH_OK) return status;
    *tflops = best;
    if (ms_out) *ms_out = best_ms;
    return SPH_OK;
}
