// FP32 SIMT correlation with the fused epilogue: the plain single-precision
// GPU path (FP32 operands, FP32 FMA accumulation).  It is the baseline the
// tensor-core path is measured against and the arithmetic of BF_FP32.
//
// Block tile: 64 templates x 256 lags, 256 threads.  Warp w owns templates
// 8w .. 8w+7 of the tile; lane l owns the eight consecutive lags 8l .. 8l+7, so
// one 32-sample chunk of the series (40 values per thread, held in registers)
// slides under the eight template rows: 64 FMAs per template value pair and no
// re-read of the series.  Templates come from the row-major FP32 layout.
#include "corr_common.cuh"

namespace bfi {

__global__ void __launch_bounds__(SIMT_THREADS, 2) k_corr_simt(const __grid_constant__ CorrParams p)
{
    __shared__ __align__(16) float sh_t[SIMT_TILE_T][SIMT_BK];
    __shared__ __align__(16) float sh_x[SIMT_TILE_L + SIMT_BK + 16];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (uint64_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
        const Seg& s = p.seg[find_seg(p, t)];
        const uint64_t local = t - s.tile_begin;
        const uint32_t tt = s.tt0 + (uint32_t)(local / s.n_lag_tiles);
        const uint32_t lag0 = (uint32_t)(local % s.n_lag_tiles) * SIMT_TILE_L;
        const uint32_t k0 = tt * SIMT_TILE_T;
        if (!BF_BOUNDS(p.err, k0 >= s.bank_k0 && lag0 < s.L)) continue;      // the same for the whole CTA
        const float* __restrict__ bank = s.bank_f32 + (size_t)(k0 - s.bank_k0) * s.M_pad;
        const float* __restrict__ xs = s.x + lag0;

        float acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

        // the 64-sample blocks of the 128-row tile holding this 64-row tile
        // outside which all its rows are zero (SIMT_BK divides 64)
        uint32_t m_lo = 0, m_hi = s.M_pad;
        if (s.tile_kb) {
            const uint32_t r = s.tile_kb[k0 / TC_TILE_T];
            m_lo = (r & 0xffffu) * TC_BK;
            m_hi = min((r >> 16) * TC_BK, s.M_pad);
        }
        for (uint32_t m0 = m_lo; m0 < m_hi; m0 += SIMT_BK) {
            __syncthreads();
            for (int i = tid; i < SIMT_TILE_T * SIMT_BK / 4; i += SIMT_THREADS) {
                int row = i / (SIMT_BK / 4), c4 = i % (SIMT_BK / 4);
                float4 v = *reinterpret_cast<const float4*>(bank + (size_t)row * s.M_pad + m0 + 4 * c4);
                *reinterpret_cast<float4*>(&sh_t[row][4 * c4]) = v;
            }
            if (tid < (SIMT_TILE_L + SIMT_BK + 16) / 4) {
                float4 v = *reinterpret_cast<const float4*>(xs + m0 + 4 * tid);
                *reinterpret_cast<float4*>(&sh_x[4 * tid]) = v;
            }
            __syncthreads();

            float xr[40];
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                float4 v = *reinterpret_cast<const float4*>(&sh_x[8 * lane + 4 * q]);
                xr[4 * q + 0] = v.x;
                xr[4 * q + 1] = v.y;
                xr[4 * q + 2] = v.z;
                xr[4 * q + 3] = v.w;
            }
#pragma unroll
            for (int mm = 0; mm < SIMT_BK; mm += 4) {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    float4 hv = *reinterpret_cast<const float4*>(&sh_t[8 * warp + a][mm]);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        acc[a][b] = fmaf(hv.x, xr[b + mm + 0], acc[a][b]);
                        acc[a][b] = fmaf(hv.y, xr[b + mm + 1], acc[a][b]);
                        acc[a][b] = fmaf(hv.z, xr[b + mm + 2], acc[a][b]);
                        acc[a][b] = fmaf(hv.w, xr[b + mm + 3], acc[a][b]);
                    }
                }
            }
        }

        // fused epilogue: normalise, max/argmax, sum of squares, tails
        float inv[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            uint32_t tau = lag0 + 8 * lane + b;
            inv[b] = tau < s.L ? s.inv_norm[tau] : 0.f;
        }
        if (s.quad) {
            // rows (a, a + 1) are a quadrature pair: output sqrt(rho_cos^2 + rho_sin^2)
#pragma unroll
            for (int a = 0; a < 8; a += 2) {
                const uint32_t k = k0 + 8 * warp + a;
                const bool keep = k >= s.k_begin && k < s.k_end;
                const uint32_t o = (k - s.k_begin) >> 1;
                const float thr = !keep ? INFINITY : (s.sigma_pred ? s.kappa * s.sigma_pred[o] : p.thr);
                unsigned long long best = 0ull;
                float ss = 0.f;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    uint32_t tau = lag0 + 8 * lane + b;
                    if (tau < s.L) {
                        const float r = sqrtf(acc[a][b] * acc[a][b] + acc[a + 1][b] * acc[a + 1][b]) * inv[b];
                        if (s.rho && keep) s.rho[(size_t)o * s.L + tau] = r;
                        unsigned long long key = pack_max(r, tau);
                        best = key > best ? key : best;
                        ss = fmaf(r, r, ss);
                        if (r >= thr) push_candidate(p, s.series_id, k >> 1, tau, r);
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, off);
                    best = ob > best ? ob : best;
                    ss += __shfl_xor_sync(0xffffffffu, ss, off);
                }
                if (lane == 0 && keep) {
                    atomicMax(s.vmax + o, best);
                    atomicAdd(s.sumsq + o, (double)ss);
                }
            }
            continue;
        }
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const uint32_t k = k0 + 8 * warp + a;
            const bool keep = k >= s.k_begin && k < s.k_end;
            const float thr = !keep ? INFINITY
                                    : (s.sigma_pred ? s.kappa * s.sigma_pred[k - s.k_begin] : p.thr);
            unsigned long long best = 0ull;
            float ss = 0.f;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                uint32_t tau = lag0 + 8 * lane + b;
                if (tau < s.L) {
                    float r = acc[a][b] * inv[b];
                    float ar = fabsf(r);
                    if (s.rho && keep) s.rho[(size_t)(k - s.k_begin) * s.L + tau] = r;
                    unsigned long long key = pack_max(ar, tau);
                    best = key > best ? key : best;
                    ss = fmaf(r, r, ss);
                    if (ar >= thr) push_candidate(p, s.series_id, k, tau, r);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                best = ob > best ? ob : best;
                ss += __shfl_xor_sync(0xffffffffu, ss, o);
            }
            if (lane == 0 && keep) {
                atomicMax(s.vmax + (k - s.k_begin), best);
                atomicAdd(s.sumsq + (k - s.k_begin), (double)ss);
            }
        }
    }
}

cudaError_t launch_corr_simt(const CorrParams& p, cudaStream_t st)
{
    if (p.total_tiles == 0) return cudaSuccess;
    uint64_t grid = p.total_tiles;
    if (grid > (1ull << 30)) grid = 1ull << 30;
    count_launches(1);
    k_corr_simt<<<(unsigned)grid, SIMT_THREADS, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace bfi
