// ts_peaks.cu -- diagnostics: measured arithmetic peaks of this GPU (FP32 and FP64 fused
// multiply-add throughput), the denominators of the pair kernel's roofline, and an evaluation of
// the exact test's refined reciprocal and square root beside the CUDA runtime's.
//
// Peaks: every thread runs independent chains of FMA (explicit fmaf / fma, so the count is exact
// whatever the contraction flags) over a grid that fills every SM; the time comes from CUDA
// events around the launch.
#include "ts_device.cuh"

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

// The exact test's refined estimates (rcp_nr, sqrt_nr) and the CUDA runtime's correctly rounded
// 1/x and sqrt(x) of the same inputs; NaN where x is outside the estimates' range.
__global__ void k_eval_estimates(const double *x, uint64_t n, double *out)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const bool in = nr_range(v);
    out[i] = in ? rcp_nr(v) : NAN;
    out[n + i] = in && v > 0.0 ? sqrt_nr(v) : NAN;
    out[2 * n + i] = 1.0 / v;
    out[3 * n + i] = sqrt(v);
}

}  // namespace

ts_status eval_estimates(const double *x, uint64_t n, double *rcp_est, double *sqrt_est,
                         double *rcp_ref, double *sqrt_ref)
{
    if (n == 0) return TS_OK;
    double *d = nullptr;
    TS_CUDA(cudaMalloc((void **)&d, sizeof(double) * 5 * n));
    cudaError_t e = cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_eval_estimates<<<(unsigned)((n + 255) / 256), 256>>>(d, n, d + n);
        note_launches(1);
        e = cudaGetLastError();
    }
    double *outs[4] = {rcp_est, sqrt_est, rcp_ref, sqrt_ref};
    for (int k = 0; k < 4 && e == cudaSuccess; k++)
        e = cudaMemcpy(outs[k], d + (uint64_t)(k + 1) * n, sizeof(double) * n,
                       cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_status(e, "eval_estimates");
    return TS_OK;
}

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
