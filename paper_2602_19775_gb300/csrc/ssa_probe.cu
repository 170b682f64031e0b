// ssa_probe.cu -- ssa_pipe_rates: throughput of the instruction classes an SSA step is made of,
// measured on the current GPU, as the basis of the issue-slot roofline of the SSA kernels.
//
// Each probe kernel runs four independent dependency chains per thread at full occupancy, so the
// result is a throughput, reported as operations per SM per clock (clock = the device's maximum
// SM clock). The chains depend on the thread index, so nothing folds at compile time.
#include <cmath>

#include "ssa_internal.cuh"

namespace {

constexpr int kIters = 2048;

__global__ void probe_ffma(float *out)
{
    float a = threadIdx.x * 1e-3f, c = a + 1.0f, d = a + 2.0f, e = a + 3.0f;
    for (int i = 0; i < kIters; ++i) {
        a = fmaf(a, 1.0001f, 1e-7f);
        c = fmaf(c, 1.0001f, 1e-7f);
        d = fmaf(d, 1.0001f, 1e-7f);
        e = fmaf(e, 1.0001f, 1e-7f);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = a + c + d + e;
}

__global__ void probe_dadd(float *out)
{
    double a = threadIdx.x * 1e-3, c = a + 1.0, d = a + 2.0, e = a + 3.0;
    for (int i = 0; i < kIters; ++i) {
        a += 1.000000001;
        c += 1.000000001;
        d += 1.000000001;
        e += 1.000000001;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)(a + c + d + e);
}

__global__ void probe_logf(float *out)
{
    float a = 0.3f + threadIdx.x * 1e-6f, c = 0.5f, d = 0.6f, e = 0.7f, s = 0.0f;
    for (int i = 0; i < kIters; ++i) {
        s += ssa::neg_log_unit(a) + ssa::neg_log_unit(c) + ssa::neg_log_unit(d) + ssa::neg_log_unit(e);
        a += 1e-7f;
        c += 1e-7f;
        d += 1e-7f;
        e += 1e-7f;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_imad(float *out)
{
    unsigned a = threadIdx.x, c = a + 1, d = a + 2, e = a + 3;
    for (int i = 0; i < kIters; ++i) {
        a = __umulhi(a, 0xD2511F53u) ^ (a * 0xCD9E8D57u);
        c = __umulhi(c, 0xD2511F53u) ^ (c * 0xCD9E8D57u);
        d = __umulhi(d, 0xD2511F53u) ^ (d * 0xCD9E8D57u);
        e = __umulhi(e, 0xD2511F53u) ^ (e * 0xCD9E8D57u);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)(a + c + d + e);
}

__global__ void probe_lg2(float *out)
{
    float a = 0.3f + threadIdx.x * 1e-6f, c = 0.5f, d = 0.6f, e = 0.7f, s = 0.0f;
    for (int i = 0; i < kIters; ++i) {
        s += __log2f(a) + __log2f(c) + __log2f(d) + __log2f(e);
        a += 1e-7f;
        c += 1e-7f;
        d += 1e-7f;
        e += 1e-7f;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

namespace ssa {
ssa_status set_error(ssa_status code, const char *text);
}

extern "C" ssa_status ssa_pipe_rates(double *host_rates, double *host_sm_clock_mhz, int32_t *host_sm_count)
{
    if (!host_rates) return ssa::set_error(SSA_ERR_INVALID_ARG, "host_rates is NULL");
    int dev = 0, sms = 0, clk_khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return ssa::set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
    const int blocks = sms * 8, threads = 256;
    float *buf = nullptr;
    e = cudaMalloc(&buf, sizeof(float) * blocks * threads);
    if (e != cudaSuccess) return ssa::set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    void (*kernels[5])(float *) = {probe_ffma, probe_dadd, probe_logf, probe_imad, probe_lg2};
    const double ops_per_iter[5] = {4, 4, 4, 8, 4};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
        kernels[k]<<<blocks, threads>>>(buf);  // warm-up
        cudaEventRecord(t0);
        kernels[k]<<<blocks, threads>>>(buf);
        cudaEventRecord(t1);
        e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        const double ops = (double)blocks * threads * kIters * ops_per_iter[k];
        host_rates[k] = ops / (ms * 1e-3) / sms / (clk_khz * 1e3);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(buf);
    if (e != cudaSuccess) return ssa::set_error(SSA_ERR_CUDA, cudaGetErrorString(e));
    if (host_sm_clock_mhz) *host_sm_clock_mhz = clk_khz / 1e3;
    if (host_sm_count) *host_sm_count = sms;
    return SSA_OK;
}
