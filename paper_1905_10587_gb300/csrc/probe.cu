// Throughput probes for the roofline denominators of the ALU-bound kernels:
// FP32 FFMA, MUFU ex2 and FP64 DFMA issue rates of the whole GPU.  Each thread
// runs eight independent dependency chains so the pipe, not latency, limits.
#include "internal.cuh"

namespace krr {

constexpr int PR_THREADS = 256;
constexpr int PR_UNROLL = 16;

__global__ void __launch_bounds__(PR_THREADS) k_probe_ffma(int iters, float a, float b, float* sink) {
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PR_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == 1234.5f) sink[0] = s;
}

__global__ void __launch_bounds__(PR_THREADS) k_probe_ex2(int iters, float* sink) {
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = -(threadIdx.x & 7) * 0.01f - c * 0.1f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PR_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = -0.5f * ex2f(x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == 1234.5f) sink[0] = s;
}

__global__ void __launch_bounds__(PR_THREADS) k_probe_dfma(int iters, double a, double b, double* sink) {
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PR_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    if (s == 1234.5) sink[0] = s;
}

// out[i] = 2^t[i] by the hardware approximation the products use (method 0), the FMA-pipe
// polynomial of the accurate product form (method 1), or the hardware approximation on the
// reduced argument t - round(t) (method 2).
__global__ void k_exp2_probe(const float* __restrict__ t, long long n, int method, float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = method == 0 ? ex2f(t[i]) : method == 1 ? exp2_poly(t[i]) : ex2_reduced(t[i]);
}

}  // namespace krr

using namespace krr;

extern "C" int krr_exp2_probe(const float* t, long long n, int method, float* out, void* stream) {
    if (!t || !out || n < 1 || method < 0 || method > 2) return KRR_E_INVAL;
    k_exp2_probe<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(t, n, method, out);
    return cudaGetLastError() == cudaSuccess ? KRR_OK : KRR_E_CUDA;
}

extern "C" int krr_peak_probe(int kind, double* ops_per_s, void* stream_v) {
    if (!ops_per_s || kind < 0 || kind > 2) return KRR_E_INVAL;
    cudaStream_t stream = (cudaStream_t)stream_v;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return KRR_E_CUDA;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return KRR_E_NOMEM;
    const int blocks = sms * 8;
    const int iters = kind == 2 ? 64 : kind == 1 ? 512 : 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
        cudaEventRecord(e0, stream);
        if (kind == 0) k_probe_ffma<<<blocks, PR_THREADS, 0, stream>>>(iters, 0.999f, 1e-3f, (float*)sink);
        else if (kind == 1) k_probe_ex2<<<blocks, PR_THREADS, 0, stream>>>(iters, (float*)sink);
        else k_probe_dfma<<<blocks, PR_THREADS, 0, stream>>>(iters, 0.999, 1e-3, (double*)sink);
        cudaEventRecord(e1, stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || ms <= 0.f) return KRR_E_CUDA;
    const double ops = (double)blocks * PR_THREADS * iters * PR_UNROLL * 8;
    *ops_per_s = ops / (ms * 1e-3);
    return KRR_OK;
}
