// peak.cu -- measured throughput of the CUDA-core pipes the path runs on, the
// denominators of its roofline fractions: FP32 fused multiply-add (the
// inlier scoring, Eq. 3) and the ex2 special-function unit (the conductance
// of Eq. 1).  Each kernel issues only that instruction, in independent
// chains, on every SM at full occupancy, and is timed with CUDA events.
// Nothing here changes a clock, a power limit or any other device setting.
#include <cuda_runtime.h>

#include "pm_internal.cuh"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 8;        // independent dependency chains per thread
constexpr int UNROLL = 16;

// Keeps the results live without a store per thread.
__device__ float g_peak_sink;

__global__ void __launch_bounds__(PEAK_THREADS) k_ffma_peak(int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
        x[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k)
                x[k] = __fmaf_rn(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
        s += x[k];
    if (s == -1.0f)   // never true for these inputs; the compiler cannot know
        g_peak_sink = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) k_ex2_peak(int iters)
{
    float x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
        x[k] = 0.5f + 1e-4f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k)
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[k]) : "f"(-x[k]));
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k)
        s += x[k];
    if (s == -1.0f)
        g_peak_sink = s;
}

}  // namespace

extern "C" pm_status pm_measure_peaks(double *fp32_tflops, double *ex2_tops, int *sm_count,
                                      void *stream)
{
    using pm::set_last_error;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma_peak, PEAK_THREADS, 0);
    if (e != cudaSuccess)
        return set_last_error(PM_ERR_CUDA, cudaGetErrorString(e));
    if (sm_count)
        *sm_count = sms;
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const double threads = (double)blocks * PEAK_THREADS;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess)
        e = cudaEventCreate(&ev[1]);
    // each measurement: one untimed launch, then the best of three timed ones
    auto timed = [&](bool ffma, int iters, float *best_ms) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        *best_ms = 0.0f;
        for (int rep = 0; rep < 4 && r == cudaSuccess; ++rep) {
            r = cudaEventRecord(ev[0], s);
            if (r != cudaSuccess)
                break;
            if (ffma)
                k_ffma_peak<<<blocks, PEAK_THREADS, 0, s>>>(iters, 0.9999999f, 1e-7f);
            else
                k_ex2_peak<<<blocks, PEAK_THREADS, 0, s>>>(iters);
            if ((r = cudaGetLastError()) != cudaSuccess || (r = cudaEventRecord(ev[1], s)) != cudaSuccess ||
                (r = cudaEventSynchronize(ev[1])) != cudaSuccess)
                break;
            float ms = 0.0f;
            r = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (rep > 0 && (*best_ms == 0.0f || ms < *best_ms))
                *best_ms = ms;
        }
        return r;
    };
    const int f_iters = 1 << 14, x_iters = 1 << 11;
    float f_ms = 0.0f, x_ms = 0.0f;
    if (e == cudaSuccess)
        e = timed(true, f_iters, &f_ms);
    if (e == cudaSuccess)
        e = timed(false, x_iters, &x_ms);
    for (cudaEvent_t x : ev)
        if (x)
            cudaEventDestroy(x);
    if (e != cudaSuccess)
        return set_last_error(PM_ERR_CUDA, cudaGetErrorString(e));
    const double per_thread_f = (double)f_iters * UNROLL * CHAINS;
    const double per_thread_x = (double)x_iters * UNROLL * CHAINS;
    if (fp32_tflops)
        *fp32_tflops = f_ms > 0 ? 2.0 * per_thread_f * threads / (f_ms * 1e-3) / 1e12 : 0.0;
    if (ex2_tops)
        *ex2_tops = x_ms > 0 ? per_thread_x * threads / (x_ms * 1e-3) / 1e12 : 0.0;
    return PM_OK;
}
