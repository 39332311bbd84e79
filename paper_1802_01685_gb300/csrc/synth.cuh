// Template synthesis shared by the bank (bank.cu) and the FFT route's direct
// fixup of low-energy lags (corr_fft.cu): one bank row into shared memory.
//
// One CTA of 256 threads per row.  The phase in cycles is evaluated in FP64 and
// reduced to [-1/2, 1/2) before the cosine, which runs in FP32 (the reduction
// is where FP64 is needed; after it FP32 holds the phase to ~1e-7 of a cycle).
// The taper is sin^2(pi (j + 1/2) / M_D) in FP32; the unit norm is an FP64 sum.
// GB300 runs FP64 at a small fraction of its FP32 rate, so FP64 is spent once
// per group of 8 samples (synth_group), and the power-law phase avoids a full
// FP64 pow: (1 - t/t_c)^(5/8) starts from the FP32 powf value and takes one
// Newton step on y^8 = u^5 in float-float arithmetic (relative error ~1e-7
// squared).
#pragma once

#include "bf_internal.h"

namespace bfi {

// Float-float (double-single) helpers: error-free FP32 products and sums
// (Dekker; the product's error from one FMA).  The _rn intrinsics keep the
// compiler from contracting a rounded product into a later addition, which
// would break the error terms.
__device__ __forceinline__ float2 ff_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return make_float2(p, __fmaf_rn(a, b, -p));
}

// a + b as (sum, error) for |a| >= |b|
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ float2 ff_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return ff_fast_two_sum(p, e);
}

// u^(5/8) for u in (0, 1]: the FP32 powf value y, then one Newton step on
// y^8 = u^5, y <- y (1 + (u^5 / y^8 - 1) / 8), with u^5 and y^8 in float-float
// (about 46 bits: the difference u^5 - y^8 needs them to well below FP32's
// resolution, not to FP64's); the result's error is ~1e-14, far inside what
// the phase anchor needs, at a third of an FP64 Newton step's FP64
// operations.  Very small u (a sweep over more than ~30x in frequency) would
// underflow y^8 in FP32 and takes the FP64 pow instead.
__device__ __forceinline__ double pow_5_8(double u)
{
    if (u < 1e-4) return pow(u, 0.625);
    const float uh = (float)u;
    const float2 uu = make_float2(uh, (float)(u - (double)uh));
    const float y0 = powf(uh, 0.625f);
    const float2 y2 = ff_two_prod(y0, y0);
    const float2 y4 = ff_mul(y2, y2);
    const float2 y8 = ff_mul(y4, y4);
    const float2 u2 = ff_mul(uu, uu);
    const float2 u4 = ff_mul(u2, u2);
    const float2 u5 = ff_mul(u4, uu);
    // the heads agree to within a factor of 2, so their difference is exact
    const float d = __fadd_rn(__fsub_rn(u5.x, y8.x), __fsub_rn(u5.y, y8.y));
    const float e = __fdividef(d, y8.x);                    // u^5 / y^8 - 1, near 0
    return (double)y0 + (double)__fmul_rn(y0, 0.125f * e);
}

// Samples are made in groups of SYN_G consecutive template indices j0 + dir q.
// The phase is evaluated in FP64 once per group, at an anchor sample j_a in
// the group (clamped into the support), and carried to the others by the
// exact phase difference over the short step d = (j - j_a) / fs, evaluated in
// FP32 without cancellation:
//   linear:    c(t_a + d) - c(t_a) = d (f(t_a) + k2 d);
//   power law: c(t_a + d) - c(t_a) = k1 u_a^(5/8) (1 - (1 - d / (t_c - t_a))^(5/8))
//              = -k1 u_a^(5/8) expm1(5/8 log1p(-d / (t_c - t_a))),
// with u_a = 1 - t_a / t_c.  |d| <= SYN_G/2 samples keeps the difference
// below ~2 cycles, where FP32 holds it to a few 1e-7 of a cycle.
constexpr int SYN_G = 8;

__device__ __forceinline__ void synth_group(float (&v)[SYN_G], int j0, int dir, float sign,
                                            const ChirpDev& p, double k1, double k2, float k2f,
                                            double inv_fs, float inv_fs_f, float inv_md, bool sine)
{
    const int j_lo = dir > 0 ? j0 : j0 - (SYN_G - 1);            // the group's index range
    if (j_lo + SYN_G - 1 < 0 || j_lo >= p.MD) return;             // all outside the support
    const int j_a = min(max(j0 + dir * (SYN_G / 2), 0), p.MD - 1);
    const double t_a = (double)j_a * inv_fs;
    double c_a;
    float lin_f = 0.f, pw_amp = 0.f, pw_rate = 0.f;
    if (p.track == BF_LINEAR) {
        c_a = t_a * fma(k2, t_a, k1);
        lin_f = (float)fma(2.0 * k2, t_a, k1);                    // f(t_a)
    } else {
        const double u_a = fma(-t_a, k2, 1.0);
        const double pw = pow_5_8(u_a);
        c_a = k1 * (1.0 - pw);
        pw_amp = (float)(k1 * pw);
        pw_rate = k2f / (float)u_a;                               // 1 / (t_c - t_a)
    }
    const float fr_a = (float)(c_a - rint(c_a));                  // [-1/2, 1/2]
#pragma unroll
    for (int q = 0; q < SYN_G; ++q) {
        const int j = j0 + dir * q;
        if (j < 0 || j >= p.MD) continue;
        const float d = (float)(j - j_a) * inv_fs_f;
        float dc = p.track == BF_LINEAR ? d * fmaf(k2f, d, lin_f)
                                        : -pw_amp * expm1f(0.625f * log1pf(-d * pw_rate));
        dc -= rintf(dc);                                          // exact
        float fr = fr_a + dc;
        fr -= rintf(fr);
        const float f2 = 2.f * fr;                                // exact doubling
        const float cs = sine ? sinpif(f2) : cospif(f2);
        const float sn = sinpif(((float)j + 0.5f) * inv_md);
        v[q] = fmaf(sign * sn * sn, cs, v[q]);
    }
}

// Bank row `row` (in a quadrature bank, chirp row / 2, odd rows holding the
// partner) into g[0, M_s) of shared memory, before normalisation (zero past M;
// M_s is a multiple of SYN_G), returning the factor 1 / |g| that gives it unit
// norm (0 for an all-zero row).  valid = false makes a zero row.  Called by all
// 256 threads of the CTA; red holds 8 doubles of shared scratch.  Ends with a
// CTA barrier, after which g is complete and red may be reused.  The row's
// FP64 constants (two divisions) and its norm (a square root and a division)
// are computed once, by thread 0, and shared: the FP64 pipe is the bound.
__device__ __forceinline__ float synth_row(const ChirpDev* __restrict__ params, uint32_t row, int quad,
                                           bool valid, uint32_t M, uint32_t M_s, double fs, float* g,
                                           double* red)
{
    __shared__ double s_c[3];           // k1, k2, 1/fs of this row
    __shared__ float s_inv;             // 1/|g|
    const bool sine = quad && (row & 1u);
    ChirpDev p{};
    if (valid) p = params[quad ? row >> 1 : row];

    if (threadIdx.x == 0) {
        double c1 = 0.0, c2 = 0.0;
        if (valid) {
            if (p.track == BF_LINEAR) {
                c1 = p.f_lo;
                c2 = (p.f_hi - p.f_lo) / (2.0 * p.D);
            } else {
                c1 = 1.6 * p.f_lo * p.tc;
                c2 = 1.0 / p.tc;
            }
        }
        s_c[0] = c1;
        s_c[1] = c2;
        s_c[2] = 1.0 / fs;
    }
    __syncthreads();
    const double k1 = s_c[0], k2 = s_c[1], inv_fs = s_c[2];
    const float inv_md = valid ? 1.0f / (float)p.MD : 0.f;
    const float inv_fs_f = (float)inv_fs;
    const float k2f = (float)k2;
    double part = 0.0;
    for (uint32_t m0 = SYN_G * threadIdx.x; m0 < M_s; m0 += SYN_G * blockDim.x) {
        float v[SYN_G];
#pragma unroll
        for (int q = 0; q < SYN_G; ++q) v[q] = 0.f;
        if (valid && m0 < M) {
            // ascending-template sample index of m0 (later samples count up),
            // and of its mirror M-1-m0 (later samples count down)
            const float rev = sine ? -1.f : 1.f;       // the reversed part of a partner is negated
            if (p.sense != BF_DESC)
                synth_group(v, (int)m0 - p.first, 1, 1.f, p, k1, k2, k2f, inv_fs, inv_fs_f, inv_md, sine);
            if (p.sense != BF_ASC)
                synth_group(v, (int)(M - 1 - m0) - p.first, -1, rev, p, k1, k2, k2f, inv_fs, inv_fs_f,
                            inv_md, sine);
        }
        float gs = 0.f;                 // the group's sum of squares (8 terms, FP32)
#pragma unroll
        for (int q = 0; q < SYN_G; ++q) {
            g[m0 + q] = v[q];
            gs = fmaf(v[q], v[q], gs);
        }
        part += (double)gs;
    }
    // block sum of g^2 in FP64
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        s_inv = tot > 0.0 ? (float)(1.0 / sqrt(tot)) : 0.f;
    }
    __syncthreads();
    return s_inv;
}

}  // namespace bfi
