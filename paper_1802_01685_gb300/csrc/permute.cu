// Time-randomised control (arXiv:1802.01685 Sect. 2.2 and Fig. 2): the series
// with its samples permuted, which keeps the sample histogram exactly and
// destroys all phase coherence.  The permutation is the argsort of the pairs
// (splitmix64(seed ^ i), i) -- a counter-based draw, so it does not depend on
// the device or thread count -- computed by a bitonic sort of 64-bit keys with
// 32-bit indices (pads sort last), followed by a gather out[j] = in[pi(j)].
// splitmix64 is the published generator of Steele, Lea and Flood (2014).
#include "bf_internal.h"

namespace bfi {

constexpr int SORT_CHUNK = 2048;          // elements per shared-memory block
constexpr int SORT_THREADS = SORT_CHUNK / 2;

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool pair_greater(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib)
{
    return ka > kb || (ka == kb && ia > ib);
}

__global__ void k_perm_keys(uint64_t* __restrict__ keys, uint32_t* __restrict__ idx, uint64_t n,
                            uint64_t P, uint64_t seed)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < P;
         i += (uint64_t)gridDim.x * blockDim.x) {
        keys[i] = i < n ? splitmix64(seed ^ i) : ~0ull;
        idx[i] = i < n ? (uint32_t)i : 0xFFFFFFFFu;
    }
}

// one compare-exchange step (k, j) over the whole array
__global__ void k_bitonic_global(uint64_t* __restrict__ keys, uint32_t* __restrict__ idx,
                                 uint64_t P, uint64_t j, uint64_t k)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < P / 2;
         t += (uint64_t)gridDim.x * blockDim.x) {
        // t-th pair: i has bit j clear
        uint64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        uint64_t l = i | j;
        bool asc = (i & k) == 0;
        uint64_t ka = keys[i], kb = keys[l];
        uint32_t ia = idx[i], ib = idx[l];
        if (pair_greater(ka, ia, kb, ib) == asc) {
            keys[i] = kb; keys[l] = ka;
            idx[i] = ib; idx[l] = ia;
        }
    }
}

// all steps with j < chunk for stages k in [k_lo, k_hi], in shared memory;
// the first stage starts at j_start
__global__ void __launch_bounds__(SORT_THREADS) k_bitonic_shared(uint64_t* __restrict__ keys,
                                                                 uint32_t* __restrict__ idx,
                                                                 uint64_t chunk, uint64_t k_lo,
                                                                 uint64_t k_hi, uint64_t j_start)
{
    __shared__ uint64_t sk[SORT_CHUNK];
    __shared__ uint32_t si[SORT_CHUNK];
    const uint64_t base = (uint64_t)blockIdx.x * chunk;
    for (uint64_t e = threadIdx.x; e < chunk; e += blockDim.x) {
        sk[e] = keys[base + e];
        si[e] = idx[base + e];
    }
    __syncthreads();
    for (uint64_t k = k_lo; k <= k_hi; k <<= 1) {
        for (uint64_t j = (k == k_lo ? j_start : k >> 1); j > 0; j >>= 1) {
            for (uint64_t t = threadIdx.x; t < chunk / 2; t += blockDim.x) {
                uint64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                uint64_t l = i | j;
                bool asc = ((base + i) & k) == 0;
                if (pair_greater(sk[i], si[i], sk[l], si[l]) == asc) {
                    uint64_t tk = sk[i]; sk[i] = sk[l]; sk[l] = tk;
                    uint32_t ti = si[i]; si[i] = si[l]; si[l] = ti;
                }
            }
            __syncthreads();
        }
    }
    for (uint64_t e = threadIdx.x; e < chunk; e += blockDim.x) {
        keys[base + e] = sk[e];
        idx[base + e] = si[e];
    }
}

__global__ void k_gather(const float* __restrict__ in, const uint32_t* __restrict__ idx,
                         uint64_t n, float* __restrict__ out)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x)
        out[j] = in[idx[j]];
}

static uint64_t pow2_at_least(uint64_t n)
{
    uint64_t P = 1;
    while (P < n) P <<= 1;
    return P < 2 ? 2 : P;
}

size_t permute_scratch_bytes(uint64_t n)
{
    uint64_t P = pow2_at_least(n);
    return (size_t)P * (sizeof(uint64_t) + sizeof(uint32_t)) + 256;
}

static unsigned grid_for(uint64_t work)
{
    uint64_t b = (work + 255) / 256;
    if (b > 65535ull * 16) b = 65535ull * 16;
    return (unsigned)(b ? b : 1);
}

// Loads the code of the permutation kernels on the current device.  Under
// CUDA's lazy module loading a kernel's module (and the device memory it
// takes) is otherwise loaded at the kernel's first launch; asking for the
// kernels' attributes loads it now.
cudaError_t preload_permute()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_perm_keys);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_bitonic_shared);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_bitonic_global);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_gather);
    return e;
}

cudaError_t launch_permute(const float* in, uint64_t n, uint64_t seed, float* out, void* scratch,
                           cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t P = pow2_at_least(n);
    uint64_t* keys = reinterpret_cast<uint64_t*>(scratch);
    uint32_t* idx = reinterpret_cast<uint32_t*>(keys + P);
    count_launches(1);
    k_perm_keys<<<grid_for(P), 256, 0, s>>>(keys, idx, n, P, seed);
    const uint64_t chunk = P < (uint64_t)SORT_CHUNK ? P : (uint64_t)SORT_CHUNK;
    const unsigned nchunks = (unsigned)(P / chunk);
    count_launches(1);
    k_bitonic_shared<<<nchunks, SORT_THREADS, 0, s>>>(keys, idx, chunk, 2, chunk, 1);
    for (uint64_t k = chunk << 1; k <= P; k <<= 1) {
        for (uint64_t j = k >> 1; j >= chunk; j >>= 1) {
            count_launches(1);
            k_bitonic_global<<<grid_for(P / 2), 256, 0, s>>>(keys, idx, P, j, k);
        }
        count_launches(1);
        k_bitonic_shared<<<nchunks, SORT_THREADS, 0, s>>>(keys, idx, chunk, k, k, chunk >> 1);
    }
    count_launches(1);
    k_gather<<<grid_for(n), 256, 0, s>>>(in, idx, n, out);
    return cudaGetLastError();
}

}  // namespace bfi
