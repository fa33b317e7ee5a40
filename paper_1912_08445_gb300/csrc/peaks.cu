// Throughput of the FP32 pipes that bound the mixed-precision formal solve, measured on
// the device (the roofline denominators of the FP32 sweep): scalar FFMA, packed FFMA2,
// and the MUFU operations ex2.approx and rcp.approx. Each kernel runs independent
// dependency chains (8 per thread) over a grid of 8 CTAs of 256 threads per SM (full
// occupancy, enough operations in flight to cover the pipe latencies), timed with CUDA
// events after a warm-up launch.
#include <cstring>
#include "common.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_ffma(float *out, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = threadIdx.x * 1e-7f + c;
    for (int i = 0; i < kIters; i++)
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == 1.2345f) out[0] = s;   // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_ffma2(float *out, float a, float b) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = make_float2(threadIdx.x * 1e-7f + c, c * 0.5f);
    for (int i = 0; i < kIters; i++)
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c].x + x[c].y;
    if (s == 1.2345f) out[0] = s;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ex2 chains: x <- ex2(-x) stays in (0, 1].
__global__ void __launch_bounds__(256) k_ex2(float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 0.25f + threadIdx.x * 1e-6f + c * 0.01f;
    for (int i = 0; i < kIters; i++)
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = ex2_approx(-x[c]);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == 1.2345f) out[0] = s;
}

// rcp chains: x <- rcp(x + 1) converges to the golden ratio's inverse; the add keeps
// the compiler from folding rcp(rcp(x)) into x (the add runs on the FMA pipe, which has
// eight times the MUFU rate).
__global__ void __launch_bounds__(256) k_rcp(float *out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 1.5f + threadIdx.x * 1e-6f + c * 0.01f;
    for (int i = 0; i < kIters; i++)
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = rcp_approx(x[c] + 1.0f);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == 1.2345f) out[0] = s;
}

}  // namespace

/* Measured pipe rates (see the header): rates[0] FFMA flops/s (2 per FMA), rates[1]
 * FFMA2 flops/s (4 per packed FMA), rates[2] ex2 results/s, rates[3] rcp results/s. */
namespace {
// Restores the calling thread's current device on every return path.
struct DeviceRestore {
    int prev = -1;
    DeviceRestore() {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceRestore() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" int mg_measure_pipe_rates(int32_t device, double *rates) {
    if (!rates) return MG_ERR_ARG;
    DeviceRestore keep;
    if (cudaSetDevice(device) != cudaSuccess) return MG_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MG_ERR_CUDA;
    float *d = nullptr;
    if (cudaMalloc(&d, 16) != cudaSuccess) return MG_ERR_OOM;
    cudaStream_t st;
    cudaEvent_t e0, e1;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaFree(d); return MG_ERR_CUDA; }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const unsigned grid = 8u * (unsigned)sms, threads = 256;
    const double work = (double)grid * threads * kChains * kIters;
    double res[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; k++) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; rep++) {   // the first launch warms up
            cudaEventRecord(e0, st);
            if (k == 0) k_ffma<<<grid, threads, 0, st>>>(d, 0.999f, 1e-3f);
            else if (k == 1) k_ffma2<<<grid, threads, 0, st>>>(d, 0.999f, 1e-3f);
            else if (k == 2) k_ex2<<<grid, threads, 0, st>>>(d);
            else k_rcp<<<grid, threads, 0, st>>>(d);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        const double per = k == 0 ? 2.0 : (k == 1 ? 4.0 : 1.0);
        res[k] = work * per / (best * 1e-3);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(d);
    if (err != cudaSuccess) return MG_ERR_CUDA;
    std::memcpy(rates, res, sizeof(res));
    return MG_OK;
}
