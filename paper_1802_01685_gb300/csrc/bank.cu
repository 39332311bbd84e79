// Template synthesis on the device (arXiv:1802.01685 Sect. 2.1: banks of up to
// 8.64 million ascending and descending chirps of ~1 s).
//
// One CTA builds one template with synth_row (synth.cuh: FP64 phase anchors
// per group of 8 samples, FP32 cosine, FP64 norm), scales it to unit norm in
// FP32 and writes the layouts the bank keeps, where the hi/lo splits of the
// tensor-core layouts are made too.  Outputs, as requested:
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

#include "synth.cuh"

namespace bfi {

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
    const uint32_t M_s = min(M_pad, (M + 63u) & ~63u);      // a multiple of SYN_G
    // the samples g are FP32, so scaling and splitting them in FP32 loses only
    // the last ulp of h (the split's own error is 2^-17); GB300's FP64 rate is
    // kept for the phase
    const float inv = synth_row(params, row, quad, valid, M, M_s, fs, g, red);

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
