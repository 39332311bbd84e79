// Predictor of the noise level of the filter output (arXiv:1802.01685,
// Sect. 2.2 and Fig. 5 caption: sigma of rho is computed in a predictor step
// by Parseval's theorem, on the GPU, and only the tails rho > kappa sigma are
// kept).  Before the search:
//
//   sigma_k^2 = sum_f P_x(f) |H_k(f)|^2 / (F^2 M sigma_x^2),   F = 16384,
//
// the sum over all F bins, with P_x the averaged periodogram of the series
// over rectangular F-sample segments at hop F/2 (a series shorter than F: one
// zero-padded segment scaled by F/N), H_k the F-point DFT of template k and
// sigma_x^2 the mean of x^2 (from the FP64 prefix of the series preparation).
// For white noise its expectation is 1/M.  F is the FFT route's real segment
// length, so both steps run on the library's own 16384-point real transform
// (corr_fft.cu); the template power spectra are made per call, chunk by chunk,
// from the chirp parameters, so nothing is kept per bank.  The work splits
// into predict_prepare (allocations, twiddle tables) and predict_launch
// (kernels only), so that a plan can capture the second in its graph.  Every
// sum runs in a fixed order: the prediction of a series is the same alone, in
// a batch, in a plan or in the serving loop, bit for bit.
#include <algorithm>

#include "runtime.h"

namespace bfi {

// one launch of the final step: up to MAX_FFT_SER series
struct SigmaBatch {
    int n;
    uint32_t s0;                           // first series of the batch (row of D)
    const double* prefix[MAX_FFT_SER];
    uint64_t N[MAX_FFT_SER];
    float* out[MAX_FFT_SER];
};

namespace {

constexpr size_t PRED_CHUNK = 4096;        // template rows synthesised per chunk

// sigma of output j (a template, or the pair of rows 2j, 2j + 1 of a
// quadrature bank, whose squares add: E rho_q^2 = E rho_cos^2 + E rho_sin^2)
// of each series of the batch, from the power dot products D[s][row]
__global__ void k_sigma_final(const __grid_constant__ SigmaBatch b, const float* __restrict__ D,
                              uint32_t d_stride, uint32_t n_out, int quad, uint32_t M)
{
    const int s = blockIdx.y;
    if (s >= b.n) return;
    const double sx2 = b.prefix[s][b.N[s]] / (double)b.N[s];
    const double F = (double)PRED_F;
    const float* d = D + (size_t)(b.s0 + s) * d_stride;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_out; j += gridDim.x * blockDim.x) {
        const double v = quad ? (double)d[2 * j] + (double)d[2 * j + 1] : (double)d[j];
        b.out[s][j] = sx2 > 0.0 && v > 0.0 ? (float)sqrt(v / (F * F * (double)M * sx2)) : 0.f;
    }
}

}  // namespace

bf_status predict_prepare(bf_ctx* ctx, const bf_bank* bank, const std::vector<const PreparedSeries*>& ps,
                          size_t k_begin, size_t k_end, float* out, size_t out_stride,
                          std::vector<void*>& scratch, cudaStream_t st, PredictCall* c)
{
    if (bank->M > (uint32_t)PRED_F / 2) {
        set_error("the Parseval predictor takes templates of at most %d samples (this bank: %u)",
                  PRED_F / 2, bank->M);
        return BF_ENOTSUP;
    }
    const float2* tw = nullptr;
    cudaError_t e = fft_tables(ctx, st, &tw);
    if (e != cudaSuccess) return cuda_fail(e, "FFT tables");
    Allocator& mem = *ctx->mem;
    auto grab = [&](size_t bytes) -> void* {
        void* p = mem.alloc(bytes);
        if (p) scratch.push_back(p);
        return p;
    };
    c->tw = tw;
    c->row_begin = (uint32_t)bank_row(bank, k_begin);
    c->row_end = (uint32_t)bank_row(bank, k_end);
    c->n_out = (uint32_t)(k_end - k_begin);
    c->n_series = (uint32_t)ps.size();
    const uint32_t n_rows = c->row_end - c->row_begin;
    c->chunk = (uint32_t)std::min<size_t>(PRED_CHUNK, n_rows);
    c->rows = static_cast<float*>(grab((size_t)c->chunk * FFT_POINTS * sizeof(float)));
    c->D = static_cast<float*>(grab((size_t)c->n_series * n_rows * sizeof(float)));
    c->P = static_cast<float*>(grab((size_t)c->n_series * PRED_BINS * sizeof(float)));
    if (!c->rows || !c->D || !c->P) {
        set_error("out of device memory (predictor)");
        return BF_ENOMEM;
    }
    for (size_t s0 = 0; s0 < ps.size(); s0 += MAX_FFT_SER) {
        const int n = (int)std::min<size_t>(MAX_FFT_SER, ps.size() - s0);
        WelchBatch b{};
        SigmaBatch sb{};
        b.n = sb.n = n;
        b.tw = tw;
        sb.s0 = (uint32_t)s0;
        uint32_t total = 0;
        for (int i = 0; i < n; ++i) {
            const PreparedSeries& p = *ps[s0 + i];
            b.x[i] = p.x;
            b.N[i] = p.N;
            b.seg_begin[i] = total;
            total += welch_segments(p.N);
            sb.prefix[i] = p.prefix;
            sb.N[i] = p.N;
            sb.out[i] = out + (s0 + i) * out_stride;
        }
        b.seg_begin[n] = total;
        b.pseg = static_cast<float*>(grab((size_t)total * PRED_BINS * sizeof(float)));
        if (!b.pseg) {
            set_error("out of device memory (predictor periodograms)");
            return BF_ENOMEM;
        }
        b.P = c->P + s0 * PRED_BINS;
        c->welch.push_back(b);
        c->sigma.push_back(new SigmaBatch(sb));
    }
    return BF_OK;
}

cudaError_t predict_launch(bf_ctx* ctx, const bf_bank* bank, const PredictCall& c, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    // the averaged periodogram of every series
    for (const WelchBatch& b : c.welch)
        if (e == cudaSuccess) e = launch_welch(b, ctx->n_sm, st);
    // template power spectra, chunk by chunk, dotted with every periodogram
    const uint32_t n_rows = c.row_end - c.row_begin;
    for (uint32_t q0 = 0; q0 < n_rows && e == cudaSuccess; q0 += c.chunk) {
        const uint32_t kc = std::min(c.chunk, n_rows - q0);
        e = launch_bank_synth(bank->d_params, c.row_begin + q0, bank->quad, kc, kc, bank->M, FFT_POINTS,
                              bank->fs, c.rows, nullptr, nullptr, st);
        if (e == cudaSuccess)
            e = launch_template_power_dot(c.rows, kc, c.tw, c.P, c.n_series, c.D, n_rows, q0, ctx->n_sm, st);
    }
    for (const SigmaBatch* sb : c.sigma) {
        if (e != cudaSuccess) break;
        count_launches(1);
        const unsigned bx = std::max(1u, std::min((c.n_out + 255) / 256, 1024u));
        k_sigma_final<<<dim3(bx, (unsigned)sb->n), 256, 0, st>>>(*sb, c.D, n_rows, c.n_out,
                                                                bank->quad ? 1 : 0, bank->M);
        e = cudaGetLastError();
    }
    return e;
}

PredictCall::~PredictCall()
{
    for (SigmaBatch* s : sigma) delete s;
}

}  // namespace bfi
