// Helpers shared by the two correlation kernels: tile lookup over segments and
// the reductions of the fused epilogue (arXiv:1802.01685 Sect. 2.1-2.2 and
// Fig. 2: per-template maxima of the filter output, sigma of the output, and
// the tails |rho| >= threshold that paint the chirp-based spectrogram).
#pragma once
#include "bf_internal.h"

namespace bfi {

// Locates the segment owning global tile t (segments are sorted by tile_begin).
__device__ __forceinline__ int find_seg(const CorrParams& p, uint64_t t)
{
    int lo = 0, hi = p.n_seg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (p.seg[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Max key of |rho| with ties resolved to the smallest lag: |rho| >= 0, so its
// float bits order like unsigned integers; the low word is ~tau.
__device__ __forceinline__ unsigned long long pack_max(float a, uint32_t tau)
{
    return ((unsigned long long)__float_as_uint(a) << 32) | (unsigned long long)(~tau);
}

__device__ __forceinline__ void push_candidate(const CorrParams& p, uint32_t series,
                                               uint32_t k, uint32_t tau, float rho)
{
    unsigned int i = atomicAdd(p.cand_count, 1u);
    if (i < p.cand_cap) p.cand[i] = Candidate{series, k, tau, rho};
}

}  // namespace bfi
