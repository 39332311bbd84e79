// Predictor of the noise level of the filter output (arXiv:1802.01685,
// Sect. 2.2 and Fig. 5 caption: sigma of rho is computed in a predictor step
// by Parseval's theorem, on the GPU, and only the tails rho > kappa sigma are
// kept).  Before the search:
//
//   sigma_k^2 = sum_f P_x(f) |H_k(f)|^2 / (F^2 M sigma_x^2),   F = 2M,
//
// with P_x the averaged periodogram of the series over rectangular F-sample
// segments at hop F/2 (a series shorter than F: one zero-padded segment
// scaled by F/N), H_k the F-point DFT of template k and sigma_x^2 the mean of
// x^2 (from the FP64 prefix of the series preparation).  For white noise this
// is exactly 1/M.  The template power spectra depend only on the bank and are
// computed once per bank (templates re-synthesised into zero-padded FFT rows,
// batched cuFFT R2C); the per-series work is one batched R2C, a reduction over
// segments and a dot product per template.
#include <cufft.h>

#include "runtime.h"

namespace bfi {

namespace {

constexpr size_t PH_CHUNK = 4096;          // templates per power-spectrum batch

bf_status cufft_fail(cufftResult r, const char* what)
{
    set_error("%s: cuFFT error %d", what, (int)r);
    return BF_ECUDA;
}

// one-sided |X(f)|^2, weighted 2 except at f = 0 and f = F/2, for `rows` rows
__global__ void k_power_rows(const cufftComplex* __restrict__ X, uint32_t rows, uint32_t nf,
                             float* __restrict__ out)
{
    const uint64_t total = (uint64_t)rows * nf;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t f = (uint32_t)(i % nf);
        const cufftComplex z = X[i];
        const float w = (f == 0 || f == nf - 1) ? 1.f : 2.f;
        out[i] = w * (z.x * z.x + z.y * z.y);
    }
}

// P(f) = scale / S * sum_s |X_s(f)|^2 (unweighted), FP64 sum over segments
__global__ void k_welch_mean(const cufftComplex* __restrict__ X, uint32_t S, uint32_t nf,
                             double scale, float* __restrict__ P)
{
    for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (uint32_t s = 0; s < S; ++s) {
            const cufftComplex z = X[(size_t)s * nf + f];
            acc += (double)z.x * z.x + (double)z.y * z.y;
        }
        P[f] = (float)(acc * scale / (double)S);
    }
}

// sigma_k for k in [k_begin, k_end): one warp per template; the rows of a
// quadrature pair add (E rho_q^2 = E rho_cos^2 + E rho_sin^2)
__global__ void k_sigma_dot(const float* __restrict__ ph, uint32_t nf, const float* __restrict__ P,
                            uint32_t k_begin, uint32_t k_end, int quad, const double* __restrict__ prefix,
                            uint64_t N, uint32_t M, float* __restrict__ sigma)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    const double sx2 = prefix[N] / (double)N;
    const double F = 2.0 * M;
    for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k_begin + w < k_end; w += warps) {
        const uint32_t k = k_begin + w;
        float acc = 0.f;
        for (int q = 0; q <= quad; ++q) {
            const float* row = ph + (size_t)(quad ? 2 * k + q : k) * nf;
            for (uint32_t f = lane; f < nf; f += 32) acc = fmaf(P[f], row[f], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0)
            sigma[w] = sx2 > 0.0 ? (float)sqrt((double)acc / (F * F * (double)M * sx2)) : 0.f;
    }
}

}  // namespace

// Weighted one-sided template power spectra [K_pad][M+1], computed once per bank.
bf_status bank_power_spectra(bf_ctx* ctx, bf_bank* bank, cudaStream_t st)
{
    if (bank->ph) return BF_OK;
    const uint32_t M = bank->M, F = 2 * M, nf = M + 1;
    Allocator& mem = *ctx->mem;
    float* ph = static_cast<float*>(mem.alloc(bank->K_pad * (size_t)nf * sizeof(float)));
    const size_t chunk = std::min<size_t>(PH_CHUNK, bank->K_pad);
    float* rows = static_cast<float*>(mem.alloc(chunk * F * sizeof(float)));
    cufftComplex* spec = static_cast<cufftComplex*>(mem.alloc(chunk * nf * sizeof(cufftComplex)));
    auto cleanup = [&]() {
        mem.release(rows);
        mem.release(spec);
    };
    if (!ph || !rows || !spec) {
        mem.release(ph);
        cleanup();
        set_error("out of device memory for the template power spectra");
        return BF_ENOMEM;
    }
    cufftHandle plan;
    int n = (int)F;
    cufftResult r = cufftPlanMany(&plan, 1, &n, nullptr, 1, (int)F, nullptr, 1, (int)nf, CUFFT_R2C,
                                  (int)chunk);
    if (r != CUFFT_SUCCESS) {
        mem.release(ph);
        cleanup();
        return cufft_fail(r, "power-spectrum plan");
    }
    cufftSetStream(plan, st);
    cudaError_t e = cudaSuccess;
    for (size_t k0 = 0; k0 < bank->K_pad && e == cudaSuccess && r == CUFFT_SUCCESS; k0 += chunk) {
        const size_t kc = std::min(chunk, bank->rows - std::min(k0, bank->rows));
        // rows of F samples: the template followed by zeros (rows past the bank are zero)
        e = launch_bank_synth(bank->d_params, (uint32_t)std::min(k0, bank->rows), bank->quad, (uint32_t)kc,
                              (uint32_t)chunk, M, F, bank->fs, rows, nullptr, nullptr, st);
        if (e == cudaSuccess) r = cufftExecR2C(plan, rows, spec);
        if (e == cudaSuccess && r == CUFFT_SUCCESS) {
            const uint32_t nrow = (uint32_t)std::min(chunk, bank->K_pad - k0);
            uint64_t total = (uint64_t)nrow * nf;
            unsigned blocks = (unsigned)std::min<uint64_t>((total + 255) / 256, 65535ull * 8);
            count_launches(1);
            k_power_rows<<<blocks, 256, 0, st>>>(spec, nrow, nf, ph + k0 * nf);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && r == CUFFT_SUCCESS) e = cudaStreamSynchronize(st);
    cufftDestroy(plan);
    cleanup();
    if (r != CUFFT_SUCCESS || e != cudaSuccess) {
        mem.release(ph);
        return r != CUFFT_SUCCESS ? cufft_fail(r, "power spectra") : cuda_fail(e, "power spectra");
    }
    bank->ph = ph;
    return BF_OK;
}

// sigma_k of one prepared series for templates [k_begin, k_end) into out[]
bf_status predict_sigma(bf_ctx* ctx, const bf_bank* bank, const PreparedSeries& ps, size_t k_begin,
                        size_t k_end, float* out, std::vector<void*>& scratch, cudaStream_t st)
{
    const uint32_t M = bank->M, F = 2 * M, nf = M + 1;
    const uint64_t N = ps.N;
    Allocator& mem = *ctx->mem;
    const float* src = ps.x;
    uint32_t S = 1;
    double scale = 1.0;
    int idist = (int)F;
    if (N >= F) {
        S = (uint32_t)((N - F) / (F / 2) + 1);
        idist = (int)(F / 2);
    } else {
        // one segment: the series zero-padded to F samples, scaled by F/N
        float* pad = static_cast<float*>(mem.alloc((size_t)F * sizeof(float)));
        if (!pad) { set_error("out of device memory (predictor)"); return BF_ENOMEM; }
        scratch.push_back(pad);
        cudaError_t e = cudaMemsetAsync(pad, 0, (size_t)F * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pad, ps.x, N * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "predictor input");
        src = pad;
        scale = (double)F / (double)N;
    }
    cufftComplex* spec = static_cast<cufftComplex*>(mem.alloc((size_t)S * nf * sizeof(cufftComplex)));
    float* P = static_cast<float*>(mem.alloc((size_t)nf * sizeof(float)));
    if (!spec || !P) {
        mem.release(spec);
        mem.release(P);
        set_error("out of device memory (predictor)");
        return BF_ENOMEM;
    }
    scratch.push_back(spec);
    scratch.push_back(P);
    cufftHandle plan;
    int n = (int)F;
    int inembed = (int)F, onembed = (int)nf;
    cufftResult r = cufftPlanMany(&plan, 1, &n, &inembed, 1, idist, &onembed, 1, (int)nf,
                                  CUFFT_R2C, (int)S);
    if (r != CUFFT_SUCCESS) return cufft_fail(r, "periodogram plan");
    cufftSetStream(plan, st);
    r = cufftExecR2C(plan, const_cast<float*>(src), spec);
    cudaError_t e = cudaSuccess;
    if (r == CUFFT_SUCCESS) {
        count_launches(2);
        k_welch_mean<<<(nf + 255) / 256, 256, 0, st>>>(spec, S, nf, scale, P);
        const uint32_t K = (uint32_t)(k_end - k_begin);
        const unsigned blocks = std::max(1u, std::min((K + 7) / 8, 65535u * 8));
        k_sigma_dot<<<blocks, 256, 0, st>>>(bank->ph, nf, P, (uint32_t)k_begin, (uint32_t)k_end,
                                            bank->quad ? 1 : 0, ps.prefix, N, M, out);
        e = cudaGetLastError();
    }
    // the plan's work area must outlive the transform; synchronising here keeps
    // the plan's lifetime local (the predictor runs once per series per call)
    if (r == CUFFT_SUCCESS && e == cudaSuccess) e = cudaStreamSynchronize(st);
    cufftDestroy(plan);
    if (r != CUFFT_SUCCESS) return cufft_fail(r, "periodogram");
    if (e != cudaSuccess) return cuda_fail(e, "predictor");
    return BF_OK;
}

}  // namespace bfi
