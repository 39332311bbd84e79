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

__device__ __forceinline__ double track_freq(const ChirpDev& p, double u)
{
    if (p.track == BF_LINEAR) return p.f_lo + (p.f_hi - p.f_lo) * u / p.D;
    return p.f_lo * pow(1.0 - u / p.tc, -0.375);
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
        const ChirpDev p = params[cd.k];
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
            const int64_t fb = (int64_t)floor(track_freq(p, u) / df);
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

}  // namespace bfi
