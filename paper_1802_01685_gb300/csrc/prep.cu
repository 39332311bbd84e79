// Series preparation on the device.
//
// (1) Split rows for the tensor-core path.  Row w holds the eight samples
//     x[w .. w+7] rounded to bf16 (hi) and the bf16 rounding of the remainder
//     x - hi (lo; x - hi is exact in FP32).  Consecutive rows overlap by seven
//     samples, so the 8-row x 8-sample core matrix that starts at row w is the
//     Hankel block x[w + i + c] (i, c < 8) stored as 128 contiguous bytes: the
//     correlation kernel feeds it to tcgen05.mma as the lag operand with 16-byte
//     row pitch and no gather.  Rows past the series read zeros.
// (2) Inverse window norms.  S[n] = sum_{i<n} x[i]^2 in FP64 (every x^2 of an
//     FP32 sample is exact in FP64), nu(tau) = S[tau+M] - S[tau], and
//     inv(tau) = 1 / sqrt(nu) rounded to FP32.  A window without a nonzero
//     sample gets exactly 0 (rho := 0 there): an exact count prefix C[n] of
//     nonzero samples decides it, because the block-wise scan sums the energy
//     prefix in different orders on either side of a block edge, so S may
//     differ by rounding across an all-zero window.
#include <algorithm>

#include "bf_internal.h"

namespace bfi {

__global__ void k_split_rows(const float* __restrict__ x, uint64_t N, uint64_t rows,
                             uint4* __restrict__ yhi, uint4* __restrict__ ylo)
{
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < rows;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            float v0 = (w + c < N) ? x[w + c] : 0.f;
            float v1 = (w + c + 1 < N) ? x[w + c + 1] : 0.f;
            __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
            __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
            __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
            h[c / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            l[c / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        yhi[w] = make_uint4(h[0], h[1], h[2], h[3]);
        ylo[w] = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// max |x| as float bits (non-negative floats order like unsigned integers)
__global__ void k_absmax(const float* __restrict__ x, uint64_t N, uint32_t* __restrict__ xmax)
{
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(x[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(xmax, m);
}

// Split rows as k_split_rows, in FP16 of x 2^s: hi = fp16(x 2^s), lo =
// fp16(x 2^s - hi) (exact difference in FP32), s from the series' max |x|.
__global__ void k_split_rows_f16(const float* __restrict__ x, uint64_t N, uint64_t rows,
                                 uint4* __restrict__ yhi, uint4* __restrict__ ylo,
                                 const uint32_t* __restrict__ xmax)
{
    const float scale = ldexpf(1.f, f16_series_shift(*xmax));
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < rows;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
            const float v0 = ((w + c < N) ? x[w + c] : 0.f) * scale;
            const float v1 = ((w + c + 1 < N) ? x[w + c + 1] : 0.f) * scale;
            const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
            const __half l0 = __float2half_rn(v0 - __half2float(h0));
            const __half l1 = __float2half_rn(v1 - __half2float(h1));
            h[c / 2] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
            l[c / 2] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
        }
        yhi[w] = make_uint4(h[0], h[1], h[2], h[3]);
        ylo[w] = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

cudaError_t launch_split_rows_f16(const float* x, uint64_t N, uint64_t rows, uint4* yhi, uint4* ylo,
                                  uint32_t* xmax, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(xmax, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    uint64_t b1 = std::min<uint64_t>((N + 255) / 256, 1024);
    uint64_t blocks = (rows + 255) / 256;
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    if (blocks == 0) blocks = 1;
    count_launches(2);
    k_absmax<<<(unsigned)std::max<uint64_t>(b1, 1), 256, 0, s>>>(x, N, xmax);
    k_split_rows_f16<<<(unsigned)blocks, 256, 0, s>>>(x, N, rows, yhi, ylo, xmax);
    return cudaGetLastError();
}

cudaError_t launch_split_rows(const float* x, uint64_t N, uint64_t rows, uint4* yhi, uint4* ylo,
                              cudaStream_t s)
{
    uint64_t blocks = (rows + 255) / 256;
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    if (blocks == 0) blocks = 1;
    count_launches(1);
    k_split_rows<<<(unsigned)blocks, 256, 0, s>>>(x, N, rows, yhi, ylo);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 scan
constexpr int SCAN_T = 512;              // threads per scan block
constexpr int SCAN_E = 4;                // elements per thread
constexpr int SCAN_B = SCAN_T * SCAN_E;  // elements per block

// block-sum scratch (doubles): energies and nonzero counts of every scan block
uint64_t inv_norm_scratch_blocks(uint64_t N) { return 2 * ((N + SCAN_B - 1) / SCAN_B + 1); }

__device__ __forceinline__ double block_excl_scan(double v, double* sh, double* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        double s = lane < (SCAN_T / 32) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < SCAN_T / 32) sh[lane] = s;
    }
    __syncthreads();
    double base = wid > 0 ? sh[wid - 1] : 0.0;
    if (total) *total = sh[SCAN_T / 32 - 1];
    return base + inc - v;
}

// Per-block sums of x^2 (FP64) and of the count of nonzero samples (an exact
// integer in FP64): bsum[0, nb) and bsum[nb, 2 nb).
__global__ void __launch_bounds__(SCAN_T) k_block_sq(const float* __restrict__ x, uint64_t N, uint64_t nb,
                                                     double* __restrict__ bsum)
{
    __shared__ double sh[SCAN_T / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_B + (uint64_t)threadIdx.x * SCAN_E;
    double v = 0.0, c = 0.0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e)
        if (base + e < N) {
            double d = x[base + e];
            v += d * d;
            c += d != 0.0 ? 1.0 : 0.0;
        }
    double tot, ctot;
    block_excl_scan(v, sh, &tot);
    __syncthreads();
    block_excl_scan(c, sh, &ctot);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = tot;
        bsum[nb + blockIdx.x] = ctot;
    }
}

// exclusive scan of the n block sums of one lane, in place (one block)
__global__ void __launch_bounds__(SCAN_T) k_scan_sums(double* __restrict__ bsum, uint64_t n)
{
    __shared__ double sh[SCAN_T / 32];
    double* lane_sums = bsum + blockIdx.x * n;        // block 0: energies, block 1: counts
    double carry = 0.0;
    for (uint64_t c = 0; c < n; c += SCAN_T) {
        uint64_t i = c + threadIdx.x;
        double v = i < n ? lane_sums[i] : 0.0;
        double tot;
        double ex = block_excl_scan(v, sh, &tot);
        __syncthreads();
        if (i < n) lane_sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
}

// S[t] = sum_{i < t} x_i^2 and C[t] = #{i < t : x_i != 0}, t = 0..N
__global__ void __launch_bounds__(SCAN_T) k_prefix(const float* __restrict__ x, uint64_t N, uint64_t nb,
                                                   const double* __restrict__ boff,
                                                   double* __restrict__ S, uint32_t* __restrict__ C)
{
    __shared__ double sh[SCAN_T / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_B + (uint64_t)threadIdx.x * SCAN_E;
    double v[SCAN_E];
    uint32_t nz[SCAN_E];
    double t = 0.0, c = 0.0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        double d = base + e < N ? (double)x[base + e] : 0.0;
        v[e] = d * d;
        nz[e] = d != 0.0 ? 1u : 0u;
        t += v[e];
        c += (double)nz[e];
    }
    double ex = block_excl_scan(t, sh, nullptr) + boff[blockIdx.x];
    __syncthreads();
    uint32_t cx = (uint32_t)(block_excl_scan(c, sh, nullptr) + boff[nb + blockIdx.x]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S[0] = 0.0;
        C[0] = 0u;
    }
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        ex += v[e];
        cx += nz[e];
        if (base + e < N) {
            S[base + e + 1] = ex;
            C[base + e + 1] = cx;
        }
    }
}

// 1 / |window|, and exactly 0 for a window without a nonzero sample (rho := 0
// there).  The count decides emptiness: a difference of FP64 prefix sums
// formed in different orders need not vanish over an all-zero window.
// The prefix difference S[t+M] - S[t] carries an absolute rounding error of a
// few ulps of S[t+M]; where the window holds less than 2^-30 of the energy
// before it (a quiet stretch after loud data) that would be a relative error
// above ~5e-6, so such windows are summed directly (x^2 is exact in FP64).
// The first thread also reports a non-finite series: the FP64 total of x^2
// (at most 2^32 squares of floats, far below the FP64 range) is finite
// exactly when every sample is.
__global__ void k_inv_norm(const float* __restrict__ x, const double* __restrict__ S,
                           const uint32_t* __restrict__ C, uint64_t L, uint32_t M,
                           float* __restrict__ inv, unsigned int* __restrict__ status)
{
    if (status && blockIdx.x == 0 && threadIdx.x == 0 && !isfinite(S[L + M - 1])) atomicOr(status, 1u);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < L;
         t += (uint64_t)gridDim.x * blockDim.x) {
        double nu = S[t + M] - S[t];
        const bool any = C[t + M] != C[t];
        if (any && nu < S[t + M] * 0x1p-30) {
            double acc = 0.0;
            for (uint32_t m = 0; m < M; ++m) {
                const double v = (double)x[t + m];
                acc = fma(v, v, acc);
            }
            nu = acc;
        }
        inv[t] = (any && nu > 0.0) ? (float)(1.0 / sqrt(nu)) : 0.f;
    }
}

size_t prefix_bytes(uint64_t N) { return (N + 1) * (sizeof(double) + sizeof(uint32_t)); }

cudaError_t launch_inv_norm(const float* x, uint64_t N, uint32_t M, double* prefix,
                            double* block_scratch, uint64_t n_blocks_cap, float* inv,
                            cudaStream_t s, unsigned int* status)
{
    uint64_t nb = (N + SCAN_B - 1) / SCAN_B;
    if (nb == 0 || 2 * nb > n_blocks_cap || N < M) return cudaErrorInvalidValue;
    uint32_t* counts = reinterpret_cast<uint32_t*>(prefix + N + 1);
    count_launches(4);
    k_block_sq<<<(unsigned)nb, SCAN_T, 0, s>>>(x, N, nb, block_scratch);
    k_scan_sums<<<2, SCAN_T, 0, s>>>(block_scratch, nb);
    k_prefix<<<(unsigned)nb, SCAN_T, 0, s>>>(x, N, nb, block_scratch, prefix, counts);
    uint64_t L = N - M + 1;
    uint64_t blocks = (L + 255) / 256;
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    k_inv_norm<<<(unsigned)blocks, 256, 0, s>>>(x, prefix, counts, L, M, inv, status);
    return cudaGetLastError();
}

}  // namespace bfi
