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

// split rows of series s = blockIdx.y: row w holds x[w .. w+7] (zero past N)
__global__ void k_split_rows(const __grid_constant__ PrepBatch b)
{
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const float* x = b.x[s];
    const uint64_t N = b.N[s], rows = b.rows[s];
    uint4* yhi = b.yhi[s];
    uint4* ylo = b.ylo[s];
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

// max |x| of series blockIdx.y as float bits (non-negative floats order like
// unsigned integers), into *xmax (zeroed by k_block_sq)
__global__ void k_absmax(const __grid_constant__ PrepBatch b)
{
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const float* x = b.x[s];
    const uint64_t N = b.N[s];
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(x[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(b.xmax[s], m);
}

// Split rows as k_split_rows, in FP16 of x 2^s: hi = fp16(x 2^s), lo =
// fp16(x 2^s - hi) (exact difference in FP32), s from the series' max |x|.
__global__ void k_split_rows_f16(const __grid_constant__ PrepBatch b)
{
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const float* x = b.x[s];
    const uint64_t N = b.N[s], rows = b.rows[s];
    uint4* yhi = b.yhi[s];
    uint4* ylo = b.ylo[s];
    const float scale = ldexpf(1.f, f16_series_shift(*b.xmax[s]));
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
// integer in FP64) of series s = blockIdx.y: bsum[0, nb) and bsum[nb, 2 nb).
// The same launch zeroes the series' padding x[N, xcap) and its max |x| word.
__global__ void __launch_bounds__(SCAN_T) k_block_sq(const __grid_constant__ PrepBatch b)
{
    __shared__ double sh[SCAN_T / 32];
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const float* x = b.x[s];
    const uint64_t N = b.N[s], nb = b.nb[s];
    for (uint64_t i = N + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < b.xcap[s];
         i += (uint64_t)gridDim.x * blockDim.x)
        b.x[s][i] = 0.f;
    if (b.mode == 2 && blockIdx.x == 0 && threadIdx.x == 0) *b.xmax[s] = 0u;
    if (blockIdx.x >= nb) return;
    double* bsum = b.bsum[s];
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

// exclusive scan of the nb block sums of one lane of series blockIdx.y, in
// place (block x = 0: energies, 1: counts)
__global__ void __launch_bounds__(SCAN_T) k_scan_sums(const __grid_constant__ PrepBatch b)
{
    __shared__ double sh[SCAN_T / 32];
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const uint64_t n = b.nb[s];
    double* lane_sums = b.bsum[s] + blockIdx.x * n;
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

// S[t] = sum_{i < t} x_i^2 and C[t] = #{i < t : x_i != 0}, t = 0..N, of
// series blockIdx.y
__global__ void __launch_bounds__(SCAN_T) k_prefix(const __grid_constant__ PrepBatch b)
{
    __shared__ double sh[SCAN_T / 32];
    const int s = blockIdx.y;
    if (s >= b.n || blockIdx.x >= b.nb[s]) return;
    const float* x = b.x[s];
    const uint64_t N = b.N[s], nb = b.nb[s];
    const double* boff = b.bsum[s];
    double* S = b.S[s];
    uint32_t* C = reinterpret_cast<uint32_t*>(S + N + 1);
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
// The first thread of a series also reports a non-finite series: the FP64
// total of x^2 (at most 2^32 squares of floats, far below the FP64 range) is
// finite exactly when every sample is.
__global__ void k_inv_norm(const __grid_constant__ PrepBatch b)
{
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const float* x = b.x[s];
    const uint32_t M = b.M;
    const uint64_t N = b.N[s], L = N - M + 1;
    const double* S = b.S[s];
    const uint32_t* C = reinterpret_cast<const uint32_t*>(S + N + 1);
    float* inv = b.inv[s];
    if (b.status[s] && blockIdx.x == 0 && threadIdx.x == 0 && !isfinite(S[N])) atomicOr(b.status[s], 1u);
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

uint64_t prep_scan_blocks(uint64_t N) { return (N + SCAN_B - 1) / SCAN_B; }

cudaError_t launch_prep(const PrepBatch& b, cudaStream_t st)
{
    if (b.n <= 0 || b.n > MAX_PREP) return cudaErrorInvalidValue;
    uint64_t nb = 0, lmax = 0, rmax = 0, nmax = 0;
    for (int i = 0; i < b.n; ++i) {
        if (b.N[i] < b.M || b.nb[i] != prep_scan_blocks(b.N[i]) || b.nb[i] == 0) return cudaErrorInvalidValue;
        nb = std::max(nb, b.nb[i]);
        lmax = std::max(lmax, b.N[i] - b.M + 1);
        rmax = std::max(rmax, b.rows[i]);
        nmax = std::max(nmax, b.N[i]);
    }
    auto grid_x = [](uint64_t work) {
        return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, 65535ull * 16));
    };
    const unsigned ny = (unsigned)b.n;
    count_launches(4);
    k_block_sq<<<dim3((unsigned)nb, ny), SCAN_T, 0, st>>>(b);
    k_scan_sums<<<dim3(2, ny), SCAN_T, 0, st>>>(b);
    k_prefix<<<dim3((unsigned)nb, ny), SCAN_T, 0, st>>>(b);
    k_inv_norm<<<dim3(grid_x(lmax), ny), 256, 0, st>>>(b);
    if (b.mode == 1) {
        count_launches(1);
        k_split_rows<<<dim3(grid_x(rmax), ny), 256, 0, st>>>(b);
    } else if (b.mode == 2) {
        count_launches(2);
        k_absmax<<<dim3((unsigned)std::min<uint64_t>((nmax + 255) / 256, 1024), ny), 256, 0, st>>>(b);
        k_split_rows_f16<<<dim3(grid_x(rmax), ny), 256, 0, st>>>(b);
    }
    return cudaGetLastError();
}

}  // namespace bfi
