// ts_peaks.cu -- measured arithmetic peaks of this GPU (FP32 and FP64 fused multiply-add
// throughput), the denominators of the pair kernel's roofline. Every thread runs independent
// chains of FMA (explicit fmaf / fma, so the count is exact whatever the contraction flags) over
// a grid that fills every SM; the time comes from CUDA events around the launch.
#include "ts_internal.cuh"

namespace ts {

void note_launches(unsigned long long n);

namespace {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_loop(int iters, T a, T b, T *out)
{
    T v[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; c++) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < PEAK_CHAINS; c++) v[c] = fma(v[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; c++) s += v[c];
    // the chains are kept: one store per thread, only when the sum takes an impossible value
    if (s == (T)-12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
ts_status time_fma(int blocks, int iters, double *tflops)
{
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TS_CUDA(cudaMalloc((void **)&out, sizeof(T) * (size_t)blocks * PEAK_THREADS));
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; err == cudaSuccess && rep < 4; rep++) {  // the first run warms up
        err = cudaEventRecord(e0, 0);
        if (err != cudaSuccess) break;
        k_fma_loop<T><<<blocks, PEAK_THREADS>>>(iters, (T)0.999999, (T)1e-6, out);
        note_launches(1);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return cuda_status(err, "alu peak measurement");
    const double flops = 2.0 * PEAK_CHAINS * (double)iters * (double)blocks * PEAK_THREADS;
    *tflops = best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
    return TS_OK;
}

}  // namespace

ts_status measure_alu_peaks(double *fp32_tflops, double *fp64_tflops)
{
    int dev = 0, sms = 0;
    TS_CUDA(cudaGetDevice(&dev));
    TS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;  // 8 blocks of 256 threads per SM: 64 warps resident
    // 2 x 8 chains x iters x 311,296 threads: ~33 ms per launch at the nominal rates (FP32 ~80,
    // FP64 ~1.25 TFLOP/s)
    TS_CHECK(time_fma<float>(blocks, 1 << 19, fp32_tflops));
    TS_CHECK(time_fma<double>(blocks, 1 << 13, fp64_tflops));
    return TS_OK;
}

}  // namespace ts
