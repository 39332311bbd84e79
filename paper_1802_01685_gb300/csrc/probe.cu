// Measured FP32 and FP64 FMA rates of the device: the denominators of the
// rooflines of the ALU-bound kernels (the FP32 SIMT correlation, the FFT
// route, the FP64 phase of the template synthesis).  The paper has no
// counterpart.
//
// Each thread runs CHAINS independent FMA chains a = a * b + c (b and c are
// kernel arguments, so nothing folds; |b| < 1 keeps the values normal), with
// the loop body unrolled UNROLL times so the loop's own counter and branch are
// a few percent of the issued instructions.  The grid fills every SM with
// as many 512-thread blocks as fit at once (one wave), enough warps to cover
// the FMA latency on all four schedulers.
// The rate counts two flops per FMA and nothing for the loop overhead, so it
// reads slightly below the pipe's true peak.
#include <algorithm>

#include "bf_internal.h"
#include "runtime.h"

namespace bfi {

namespace {

constexpr int CHAINS = 16;
constexpr int UNROLL = 4;
constexpr int PROBE_T = 512;
constexpr int PROBE_MAX_BLOCKS_PER_SM = 4;    // the output buffer's size

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(PROBE_T) k_fma_rate(T b, T c, uint32_t iters, T* __restrict__ out)
{
    T a[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = (T)(threadIdx.x & 63) * (T)1e-3 + (T)i;
    for (uint32_t n = 0; n < iters; ++n) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) a[i] = fma_t(a[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += a[i];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// best of `reps` timed launches (after one untimed), in TFLOP/s
template <typename T>
cudaError_t time_rate(int n_sm, uint32_t iters, int reps, cudaStream_t st, T* out, double* tflops)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate<T>, PROBE_T, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)(n_sm * std::min(per_sm, PROBE_MAX_BLOCKS_PER_SM));
    const T b = (T)0.999, c = (T)1e-3;
    cudaEvent_t e0, e1;
    e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    double best_ms = 1e30;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, st);
        count_launches(1);
        k_fma_rate<T><<<grid, PROBE_T, 0, st>>>(b, c, iters, out);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0) best_ms = std::min(best_ms, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * CHAINS * UNROLL * (double)iters * grid * PROBE_T;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_probe_alu_peaks(int device, double* fp32_tflops, double* fp64_tflops)
{
    if (!fp32_tflops && !fp64_tflops) { set_error("NULL argument"); return BF_EINVAL; }
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    cudaStream_t st = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    void* out = nullptr;
    const size_t n_out = (size_t)n_sm * PROBE_MAX_BLOCKS_PER_SM * PROBE_T;
    if (e == cudaSuccess) e = cudaMalloc(&out, n_out * sizeof(double));
    // about 35 ms per FP32 launch and 40 ms per FP64 launch at the nominal rates
    if (e == cudaSuccess && fp32_tflops)
        e = time_rate<float>(n_sm, 1u << 16, 3, st, static_cast<float*>(out), fp32_tflops);
    if (e == cudaSuccess && fp64_tflops)
        e = time_rate<double>(n_sm, 1u << 10, 3, st, static_cast<double*>(out), fp64_tflops);
    if (out) cudaFree(out);
    if (st) cudaStreamDestroy(st);
    cudaSetDevice(prev);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "FMA rate probe");
}
