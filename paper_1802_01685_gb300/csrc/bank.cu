// Template synthesis on the device (arXiv:1802.01685 Sect. 2.1: banks of up to
// 8.64 million ascending and descending chirps of ~1 s).
//
// One CTA builds one template: the phase in cycles is evaluated in FP64 and
// reduced to [-1/2, 1/2) before the cosine, which then runs in FP32 (the
// reduction is where FP64 is needed; after it FP32 holds the phase to ~1e-7
// of a cycle).  The taper is sin^2(pi (j + 1/2) / M_D) in FP32; the unit norm is
// an FP64 sum over the template, applied in FP32, where the hi/lo split of
// the tensor-core layout is made too.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so FP64 is spent once
// per group of 8 samples (synth_group below), and the power-law phase avoids
// a full FP64 pow: (1 - t/t_c)^(5/8) starts from the FP32 powf value and
// takes one Newton step on y^8 = u^5 in FP64 (relative error ~1e-7 squared),
// whose reciprocal comes from an FP32 seed and one Newton-Raphson step.  Outputs, as requested:
//   f32: row-major [K_pad][M_pad] float (SIMT path),
//   hi/lo: the tensor-core operand layout (below), hi = bf16(h), lo = bf16(h - hi).
//
// Tensor-core operand layout ("A" operand of tcgen05.mma, K-major, no swizzle):
// templates are grouped in tiles of 128 (tt = k / 128, r = k % 128) and samples
// in blocks of 64 (kb = m / 64, c = m % 64).  Each (tt, kb) block is 16 KiB,
// stored contiguously at ((tt * n_kb + kb) * 16384) so one bulk copy stages it;
// inside, the 8x8 core matrix (r / 8, c / 8) is 128 contiguous bytes at
// (r / 8) * 1024 + (c / 8) * 128, row r % 8 at +16 * (r % 8), element c % 8 at +2.
// Hence LBO (next 8 samples) = 128 B and SBO (next 8 templates) = 1024 B.
#include <algorithm>

#include "bf_internal.h"

namespace bfi {

// u^(5/8) for u in (0, 1]; very small u (a sweep over more than ~30x in
// frequency) would underflow y^8 in FP32 and takes the FP64 pow instead
__device__ __forceinline__ double pow_5_8(double u)
{
    if (u < 1e-4) return pow(u, 0.625);
    const double y = (double)powf((float)u, 0.625f);
    const double u2 = u * u, u5 = u2 * u2 * u;
    const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    double r = (double)(1.0f / (float)y8);              // 1/y^8, then one refinement
    r = r * fma(-y8, r, 2.0);
    const double qv = u5 * r;                           // u^5 / y^8, close to 1
    return y * fma(qv - 1.0, 0.125, 1.0);               // y - (y^8 - u^5) / (8 y^7)
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

__device__ __forceinline__ size_t tc_offset(uint32_t k, uint32_t m, uint32_t n_kb)
{
    uint32_t tt = k >> 7, r = k & 127, kb = m >> 6, c = m & 63;
    return ((size_t)tt * n_kb + kb) * TILE_BYTES_A + (r >> 3) * 1024 + (c >> 3) * 128 +
           (r & 7) * 16 + (c & 7) * 2;
}

// Row k of the output is bank row row0 + k.  In a quadrature bank row r is
// chirp r / 2, and odd rows hold the quadrature partner: the Hilbert
// transform of the template, i.e. sin(2 pi c(t)) in place of the cosine with
// time-reversed parts negated (ascending g_s[m], descending -g_s[M-1-m], both
// g_s[m] - g_s[M-1-m]), at unit norm of its own.
__global__ void __launch_bounds__(256) k_bank_synth(const ChirpDev* __restrict__ params,
                                                    uint32_t row0, int quad, uint32_t K,
                                                    uint32_t M, uint32_t M_pad,
                                                    double fs, float* __restrict__ f32,
                                                    uint8_t* __restrict__ hi,
                                                    uint8_t* __restrict__ lo,
                                                    uint8_t* __restrict__ hi16,
                                                    uint8_t* __restrict__ lo16)
{
    extern __shared__ float g[];        // the first M_s = round64(M) samples of the row
    __shared__ double red[8];
    const uint32_t k = blockIdx.x;
    const uint32_t n_kb = M_pad / TC_BK;
    const bool valid = k < K;
    const uint32_t row = row0 + k;
    const bool sine = quad && (row & 1u);
    ChirpDev p{};
    if (valid) p = params[quad ? row >> 1 : row];

    const double inv_fs = 1.0 / fs;
    double k1 = 0.0, k2 = 0.0;
    float inv_md = 0.f;
    if (valid) {
        if (p.track == BF_LINEAR) {
            k1 = p.f_lo;
            k2 = (p.f_hi - p.f_lo) / (2.0 * p.D);
        } else {
            k1 = 1.6 * p.f_lo * p.tc;
            k2 = 1.0 / p.tc;
        }
        inv_md = 1.0f / (float)p.MD;
    }
    const uint32_t M_s = min(M_pad, (M + 63u) & ~63u);      // a multiple of SYN_G
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
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    // the samples g are FP32, so scaling and splitting them in FP32 loses only
    // the last ulp of h (the split's own error is 2^-17); GB300's FP64 rate is
    // kept for the phase
    const float inv = tot > 0.0 ? (float)(1.0 / sqrt(tot)) : 0.f;

    for (uint32_t m = threadIdx.x; m < M_pad; m += blockDim.x) {
        const float h = m < M_s ? g[m] * inv : 0.f;
        if (f32) f32[(size_t)k * M_pad + m] = h;
        if (hi) {
            __nv_bfloat16 bh = __float2bfloat16_rn(h);
            __nv_bfloat16 bl = __float2bfloat16_rn(h - __bfloat162float(bh));   // exact difference
            size_t off = tc_offset(k, m, n_kb);
            *reinterpret_cast<__nv_bfloat16*>(hi + off) = bh;
            *reinterpret_cast<__nv_bfloat16*>(lo + off) = bl;
        }
        if (hi16) {
            // FP16 split of 2^8 h: the scale keeps the lo parts normal
            const float hs = h * TEMPLATE_F16_SCALE;
            const __half fh = __float2half_rn(hs);
            const __half fl = __float2half_rn(hs - __half2float(fh));       // exact difference
            size_t off = tc_offset(k, m, n_kb);
            *reinterpret_cast<__half*>(hi16 + off) = fh;
            *reinterpret_cast<__half*>(lo16 + off) = fl;
        }
    }
}

cudaError_t launch_bank_synth(const ChirpDev* params, uint32_t row0, int quad, uint32_t K, uint32_t K_pad, uint32_t M,
                              uint32_t M_pad, double fs, float* f32, uint8_t* hi, uint8_t* lo,
                              cudaStream_t s, uint8_t* hi16, uint8_t* lo16)
{
    size_t smem = (size_t)std::min(M_pad, (M + 63u) & ~63u) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bank_synth,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    count_launches(1);
    k_bank_synth<<<K_pad, 256, smem, s>>>(params, row0, quad, K, M, M_pad, fs, f32, hi, lo, hi16, lo16);
    return cudaGetLastError();
}

}  // namespace bfi
