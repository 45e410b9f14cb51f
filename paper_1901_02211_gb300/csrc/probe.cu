// Arithmetic peaks of the GPU, measured: the denominators of the ALU rooflines
// that the float-float and FP64 solver kernels are reported against.  Not part
// of the paper's method; the measured counterpart of "SMs x lanes x clock".
//
// Each thread runs 8 independent fused multiply-add chains (enough independent
// work to fill the pipes), 8 resident blocks of 256 threads per SM.  The
// multiplier and addend are kernel arguments, so nothing folds at compile time;
// the values stay bounded (|m| < 1) and one guarded store keeps the chains live.
#include <algorithm>

#include "smpq_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(int iters, float m, float c, float *out) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

// the packed two-lane form (one instruction, two FP32 lanes)
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma2(int iters, float m, float c, float *out) {
    float2 a[PROBE_CHAINS];
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k].x + a[k].y;
    if (s == 1234.5f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int iters, double m, double c, float *out) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], m, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    if (s == 1234.5) out[blockIdx.x] = (float)s;
}

} // namespace

extern "C" int smpq_alu_peak(int device, int kind, double *ops_per_s) {
    if (!ops_per_s || kind < 0 || kind > 2) return SMPQ_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SMPQ_ECUDA;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    // about 2e10 lane operations per FP32 launch, 2.5e9 per FP64 launch
    const int iters = kind == 2 ? 1 << 10 : 1 << 13;
    const double lanes = (kind == 1 ? 2.0 : 1.0) * PROBE_CHAINS;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, blocks * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreate(&st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) { // the first launch is a warm-up
        cudaEventRecord(e0, st);
        if (kind == 0) k_probe_ffma<<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999999f, 1e-7f, out);
        else if (kind == 1) k_probe_ffma2<<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999999f, 1e-7f, out);
        else k_probe_dfma<<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999999, 1e-7, out);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0) {
            const double ops = (double)blocks * PROBE_THREADS * iters * lanes;
            best = std::max(best, ops / (ms * 1e-3));
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SMPQ_ECUDA;
    }
    *ops_per_s = best;
    return SMPQ_OK;
}
