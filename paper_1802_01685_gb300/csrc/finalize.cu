// Reductions after the correlation kernels.
//   finalize: unpack the per-template max key into max |rho| and its argmax,
//             sigma = sqrt(sum rho^2 / L), histogram of the maxima (Fig. 2:
//             distributions of maxima of the filter output), and the
//             per-template mean of the maxima over all series (Fig. 1: the
//             spectrum averaged over 42 light curves).
//   paint:    the chirp-based spectrogram of Sect. 2.1.  Every tail (k, tau)
//             with |rho| >= threshold paints the track f(t) of template k,
//             placed at lag tau, onto cells of dt x df by maximum.  A time cell
//             b is painted when its centre (b + 1/2) dt lies in the template's
//             support [(tau + a_k) / fs, (tau + a_k + M_D) / fs); the frequency
//             is the ascending track at the local time t (ascending templates)
//             or at D - t (descending), clamped to [0, D], binned by floor(f/df).
//             Bin arithmetic is FP64.
#include "bf_internal.h"

namespace bfi {

__global__ void k_finalize(const __grid_constant__ FinalizeParams p, uint32_t K, uint32_t nbins)
{
    const uint64_t total = (uint64_t)p.n * K;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = (uint32_t)(i / K), k = (uint32_t)(i % K);
        const FinalizeSeries& f = p.ser[s];
        const unsigned long long key = f.packed[k];
        const float a = __uint_as_float((uint32_t)(key >> 32));
        const uint32_t tau = ~(uint32_t)(key & 0xFFFFFFFFull);
        f.vmax[k] = a;
        f.argmax[k] = (int32_t)tau;
        f.sigma[k] = (float)sqrt(f.sumsq[k] / (double)f.L);
        if (f.hist) {
            int b = (int)floorf(a * (float)nbins);
            b = b < 0 ? 0 : (b > (int)nbins - 1 ? (int)nbins - 1 : b);
            atomicAdd(f.hist + b, 1u);
        }
    }
}

// vmax is [n_series][K]; the mean runs over series in a fixed order
__global__ void k_mean_max(const float* __restrict__ vmax, uint32_t n_series, uint32_t K,
                           float* __restrict__ mean)
{
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (uint32_t s = 0; s < n_series; ++s) acc += (double)vmax[(size_t)s * K + k];
        mean[k] = (float)(acc / (double)n_series);
    }
}

cudaError_t launch_finalize(const FinalizeParams& p, uint32_t K, uint32_t nbins, cudaStream_t s)
{
    uint64_t total = (uint64_t)p.n * K;
    uint64_t blocks = (total + 255) / 256;
    if (blocks > 65535ull * 32) blocks = 65535ull * 32;
    if (blocks == 0) return cudaSuccess;
    count_launches(1);
    k_finalize<<<(unsigned)blocks, 256, 0, s>>>(p, K, nbins);
    return cudaGetLastError();
}

cudaError_t launch_mean_max(const float* vmax, uint32_t n_series, uint32_t K, float* mean,
                            cudaStream_t s)
{
    unsigned b = (K + 255) / 256;
    if (b == 0) return cudaSuccess;
    count_launches(1);
    k_mean_max<<<b, 256, 0, s>>>(vmax, n_series, K, mean);
    return cudaGetLastError();
}

// Moments of the maxima for the skew-normal fit (Fig. 2: the distributions
// of maxima of the filter output are left-truncated skewed Gaussians).  Two
// FP64 passes over v[0, n): pass 0 sums v into acc[0]; pass 1 sums the
// squared and cubed deviations from mean = acc[0] / n into acc[1], acc[2].
__global__ void k_moments(const float* __restrict__ v, uint64_t n, int pass, double* __restrict__ acc)
{
    const double mean = pass ? acc[0] / (double)n : 0.0;
    double a = 0.0, b = 0.0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double x = (double)v[i];
        if (pass == 0) {
            a += x;
        } else {
            const double d = x - mean, d2 = d * d;
            a += d2;
            b += d2 * d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    __shared__ double sa[32], sb[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = (int)(blockDim.x >> 5);
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            atomicAdd(acc + (pass ? 1 : 0), a);
            if (pass) atomicAdd(acc + 2, b);
        }
    }
}

// Method-of-moments skew-normal parameters (Azzalini 1985) from the sums of
// k_moments: sample skewness g, clipped to the family's range, gives
// |delta| = sqrt(pi/2 |g|^(2/3) / (|g|^(2/3) + ((4 - pi)/2)^(2/3))) with the
// sign of g, then alpha = delta / sqrt(1 - delta^2), omega = sd /
// sqrt(1 - 2 delta^2 / pi) and xi = mean - omega delta sqrt(2 / pi).
// out = {n, mean, sd, skewness, xi, omega, alpha}.
__global__ void k_skewnorm_close(const double* __restrict__ acc, uint64_t n, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double pi = 3.14159265358979323846;
    const double dn = (double)n;
    const double mean = acc[0] / dn, var = acc[1] / dn, m3 = acc[2] / dn;
    const double sd = sqrt(var);
    double g = var > 0.0 ? m3 / (var * sd) : 0.0;
    const double gmax = 0.99527;
    g = fmin(fmax(g, -gmax), gmax);
    const double a = pow(fabs(g), 2.0 / 3.0);
    const double c = pow((4.0 - pi) / 2.0, 2.0 / 3.0);
    const double delta = copysign(sqrt(pi / 2.0 * a / (a + c)), g);
    out[0] = dn;
    out[1] = mean;
    out[2] = sd;
    out[3] = g;
    const double omega = sd / sqrt(1.0 - 2.0 * delta * delta / pi);
    out[4] = mean - omega * delta * sqrt(2.0 / pi);
    out[5] = omega;
    out[6] = delta / sqrt(1.0 - delta * delta);
}

// Pseudo-spectra of tails of two detectors (Fig. 6: counts of rho > kappa
// sigma against frequency, independently and simultaneously in both
// detectors with frequency pairs within delta f).  A cell (t, c) of a map is
// occupied when a tail painted it (value > 0).  out = [4][nf]: independent
// counts of a and b, then the counts of occupied cells of a (of b) that have
// an occupied cell of the other map within dt time cells and w frequency
// cells.  Tails are sparse, so the window is searched only at occupied cells.
__device__ __forceinline__ bool any_occupied(const float* __restrict__ m, uint32_t nf, uint32_t t0,
                                             uint32_t t1, uint32_t c0, uint32_t c1)
{
    for (uint32_t t = t0; t <= t1; ++t)
        for (uint32_t c = c0; c <= c1; ++c)
            if (m[(size_t)t * nf + c] > 0.f) return true;
    return false;
}

__global__ void k_coincidence(const float* __restrict__ A, const float* __restrict__ B, uint32_t nt,
                              uint32_t nf, uint32_t w, uint32_t dt, unsigned int* __restrict__ out)
{
    const uint64_t total = (uint64_t)nt * nf;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const bool oa = A[i] > 0.f, ob = B[i] > 0.f;
        if (!oa && !ob) continue;
        const uint32_t t = (uint32_t)(i / nf), c = (uint32_t)(i % nf);
        const uint32_t t0 = t > dt ? t - dt : 0, t1 = min(t + dt, nt - 1);
        const uint32_t c0 = c > w ? c - w : 0, c1 = min(c + w, nf - 1);
        if (oa) {
            atomicAdd(out + c, 1u);
            if (any_occupied(B, nf, t0, t1, c0, c1)) atomicAdd(out + 2 * nf + c, 1u);
        }
        if (ob) {
            atomicAdd(out + nf + c, 1u);
            if (any_occupied(A, nf, t0, t1, c0, c1)) atomicAdd(out + 3 * nf + c, 1u);
        }
    }
}

// out: 4 nf counters, zeroed here
cudaError_t launch_coincidence(const float* A, const float* B, uint32_t nt, uint32_t nf, uint32_t w,
                               uint32_t dt, unsigned int* out, int n_sm, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 4 * (size_t)nf * sizeof(unsigned int), s);
    const uint64_t total = (uint64_t)nt * nf;
    if (e != cudaSuccess || total == 0) return e;
    const unsigned blocks = (unsigned)std::min<uint64_t>((total + 255) / 256, 8ull * n_sm);
    count_launches(1);
    k_coincidence<<<blocks, 256, 0, s>>>(A, B, nt, nf, w, dt, out);
    return cudaGetLastError();
}

// acc: 3 doubles (zeroed here); out: 7 doubles, both device memory
cudaError_t launch_skewnorm_fit(const float* v, uint64_t n, double* acc, double* out, int n_sm,
                                cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(acc, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const uint64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, 4ull * n_sm));
    count_launches(3);
    k_moments<<<blocks, 256, 0, s>>>(v, n, 0, acc);
    k_moments<<<blocks, 256, 0, s>>>(v, n, 1, acc);
    k_skewnorm_close<<<1, 32, 0, s>>>(acc, n, out);
    return cudaGetLastError();
}

// v^(-3/8) for v in (0, 1]: the FP32 powf value, then one Newton step on
// y^8 v^3 = 1 in FP64 (relative error ~1e-7 squared), as GB300 runs a full
// FP64 pow at a small fraction of its FP32 rate; very small v (a sweep over
// more than ~30x in frequency near its end) takes the FP64 pow
__device__ __forceinline__ double pow_m3_8(double v)
{
    if (v < 1e-4) return pow(v, -0.375);
    const double y = (double)powf((float)v, -0.375f);
    const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    const double e = fma(y8, v * v * v, -1.0);          // y^8 v^3 - 1, near 0
    return y * fma(-e, 0.125, 1.0);                     // y - (y^8 v^3 - 1) / (8 y^7 v^3)
}

// A template's track in cell units, per candidate: q(u) = a + b u (linear) or
// a (1 - b u)^(-3/8) (power law), i.e. f(u) / df with the divisions by D, t_c
// and df taken once, not per cell (GB300 divides in FP64 at a small fraction
// of its FP32 rate).
struct TrackCells {
    double a, b;
};

__device__ __forceinline__ TrackCells track_cells(const ChirpDev& p, double df)
{
    if (p.track == BF_LINEAR) return {p.f_lo / df, (p.f_hi - p.f_lo) / (p.D * df)};
    return {p.f_lo / df, 1.0 / p.tc};
}

// Frequency cell of the ascending track at local time u (the map paints f(t)).
// The end of the sweep (u clamped to D) takes its defined value f(D) = f_hi
// exactly: through the formula it lands within an ulp of f_hi, and where
// f_hi / df is a whole number the cell would hang on that ulp.  Elsewhere the
// fast value is within ~1e-13 of f / df; where f / df lies that close to a
// cell edge the cell is decided by the defining formula in FP64, with its
// divisions, as the oracle evaluates it.
__device__ __forceinline__ int64_t track_cell(const ChirpDev& p, const TrackCells& c, double u, double df)
{
    if (u >= p.D) return (int64_t)floor(p.f_hi / df);
    const bool lin = p.track == BF_LINEAR;
    const double q = lin ? fma(c.b, u, c.a) : c.a * pow_m3_8(fma(-u, c.b, 1.0));
    if (fabs(q - rint(q)) > 1e-9 * fabs(q)) return (int64_t)floor(q);
    const double f = lin ? p.f_lo + (p.f_hi - p.f_lo) * u / p.D : p.f_lo * pow(1.0 - u / p.tc, -0.375);
    return (int64_t)floor(f / df);
}

// one warp per candidate, lanes over time cells
__global__ void k_paint(const Candidate* __restrict__ cand, const unsigned int* __restrict__ count,
                        unsigned int cap, const ChirpDev* __restrict__ params,
                        const __grid_constant__ FinalizeParams fp, uint32_t M, double fs,
                        double dt, double df, uint32_t nf)
{
    const unsigned int n = min(*count, cap);
    const unsigned int lane = threadIdx.x & 31;
    const unsigned int warps = (gridDim.x * blockDim.x) >> 5;
    for (unsigned int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += warps) {
        const Candidate cd = cand[c];
        if (cd.series < fp.s0 || cd.series >= fp.s0 + fp.n) continue;
        if (!BF_BOUNDS(fp.err, cd.k < fp.n_chirps)) continue;
        const ChirpDev p = params[cd.k];
        const TrackCells tcells = track_cells(p, df);
        const FinalizeSeries& f = fp.ser[cd.series - fp.s0];
        const float a = fabsf(cd.rho);
        // a superposed template paints both of its tracks
        for (int pass = 0; pass < (p.sense == BF_BOTH ? 2 : 1); ++pass) {
        const int sense = p.sense == BF_BOTH ? (pass == 0 ? BF_ASC : BF_DESC) : p.sense;
        const int64_t first = sense == BF_ASC ? p.first : (int64_t)M - p.first - p.MD;
        const double t0 = (double)((int64_t)cd.tau + first) / fs;
        const double t1 = (double)((int64_t)cd.tau + first + p.MD) / fs;
        int64_t b_lo = (int64_t)floor(t0 / dt - 0.5);
        const int64_t b_hi = (int64_t)ceil(t1 / dt);
        if (b_lo < 0) b_lo = 0;
        for (int64_t b = b_lo + lane; b <= b_hi && b < (int64_t)f.nt; b += 32) {
            const double tb = ((double)b + 0.5) * dt;
            if (!(tb >= t0 && tb < t1)) continue;
            const double t = tb - t0;
            double u = sense == BF_ASC ? t : p.D - t;
            if (u < 0.0) u = 0.0;
            if (u > p.D) u = p.D;
            const int64_t fb = track_cell(p, tcells, u, df);
            if (fb < 0 || fb >= (int64_t)nf) continue;
            atomicMax(reinterpret_cast<int*>(f.map + (size_t)b * nf + fb), __float_as_int(a));
        }
        }
    }
}

cudaError_t launch_paint(const Candidate* cand, const unsigned int* count, unsigned int cap,
                         const ChirpDev* params, const FinalizeParams& fp, uint32_t M, double fs,
                         double dt, double df, uint32_t nf, unsigned int n_sm, cudaStream_t s)
{
    count_launches(1);
    k_paint<<<n_sm * 8, 256, 0, s>>>(cand, count, cap, params, fp, M, fs, dt, df, nf);
    return cudaGetLastError();
}

// ---- Painted cells of a time-frequency map, in increasing cell index.
// Three launches over the map's CELL_BLK-cell blocks: the nonzero count of
// each block, an exclusive scan of those counts (one CTA; it also writes the
// total), then each block writes its nonzero cells at its offset, in cell
// order.  The outputs may be mapped page-locked host memory: only the painted
// cells cross to the host.
constexpr int CELL_T = 256;
constexpr int CELL_IT = 32;                         // cells per thread per block
constexpr uint32_t CELL_BLK = CELL_T * CELL_IT;     // 8192 cells per block

uint64_t map_cell_blocks(uint64_t n_cells) { return (n_cells + CELL_BLK - 1) / CELL_BLK; }

__global__ void __launch_bounds__(CELL_T) k_cells_count(const float* __restrict__ map, uint64_t n,
                                                        uint32_t* __restrict__ counts)
{
    __shared__ uint32_t red[CELL_T / 32];
    const uint64_t base = (uint64_t)blockIdx.x * CELL_BLK;
    uint32_t c = 0;
#pragma unroll 4
    for (int it = 0; it < CELL_IT; ++it) {
        const uint64_t i = base + (uint64_t)it * CELL_T + threadIdx.x;
        if (i < n && map[i] != 0.f) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < CELL_T / 32; ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}

// exclusive scan of counts[0, nb) in place, and the total into *total
__global__ void __launch_bounds__(1024) k_cells_scan(uint32_t* __restrict__ counts, uint64_t nb,
                                                     uint32_t* __restrict__ total)
{
    __shared__ uint32_t sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (uint64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
        const uint64_t i = c0 + threadIdx.x;
        const uint32_t v = i < nb ? counts[i] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) sh[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint32_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            sh[lane] = w;
        }
        __syncthreads();
        const uint32_t before = (wid > 0 ? sh[wid - 1] : 0u) + inc - v;
        if (i < nb) counts[i] = carry + before;
        carry += sh[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(CELL_T) k_cells_write(const float* __restrict__ map, uint64_t n,
                                                        const uint32_t* __restrict__ offsets,
                                                        uint32_t* __restrict__ cell, float* __restrict__ value,
                                                        uint64_t cap)
{
    __shared__ uint32_t wsum[CELL_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * CELL_BLK;
    uint64_t at = offsets[blockIdx.x];
    for (int it = 0; it < CELL_IT; ++it) {
        const uint64_t i = base + (uint64_t)it * CELL_T + threadIdx.x;
        const float v = i < n ? map[i] : 0.f;
        const bool hit = v != 0.f;
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wsum[wid] = __popc(m);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < CELL_T / 32; ++w) {
            before += w < wid ? wsum[w] : 0u;
            total += wsum[w];
        }
        const uint64_t slot = at + before + __popc(m & ((1u << lane) - 1u));
        if (hit && slot < cap) {
            cell[slot] = (uint32_t)i;
            value[slot] = v;
        }
        at += total;
        __syncthreads();                            // wsum read before the next iteration writes it
    }
}

cudaError_t launch_map_cells(const float* map, uint64_t n_cells, uint32_t* counts, uint32_t* cell, float* value,
                             uint64_t cap, uint32_t* total, cudaStream_t s)
{
    const uint64_t nb = map_cell_blocks(n_cells);
    if (nb == 0) return cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
    if (nb > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    count_launches(3);
    k_cells_count<<<(unsigned)nb, CELL_T, 0, s>>>(map, n_cells, counts);
    k_cells_scan<<<1, 1024, 0, s>>>(counts, nb, total);
    k_cells_write<<<(unsigned)nb, CELL_T, 0, s>>>(map, n_cells, counts, cell, value, cap);
    return cudaGetLastError();
}

}  // namespace bfi
