// Host runtime pieces shared by the C ABI (api.cu) and the serving scheduler
// (serve.cu): series preparation, segment building, launches, results.
#pragma once
#include "bf_internal.h"

namespace bfi {

bf_status cuda_fail(cudaError_t e, const char* what);
uint32_t template_len(double T, double fs);
void map_shape(size_t N, double fs, double dt, double df, uint32_t* nt, uint32_t* nf);

// A series resident on the device in the layouts the kernels read.
struct PreparedSeries {
    size_t N = 0;
    uint32_t L = 0;
    float* x = nullptr;             // padded FP32 samples
    float* inv = nullptr;           // [L] inverse window norms
    uint4* yhi = nullptr;           // split rows (tensor-core path)
    uint4* ylo = nullptr;
    double* prefix = nullptr;       // FP64 prefix of x^2, then the uint32 nonzero counts (scratch)
    uint32_t* xmax = nullptr;       // split-FP16 rows: float bits of max |x|
    double* bsum = nullptr;         // scan block sums (scratch)
    uint64_t xcap = 0, nb = 0, rows = 0;
    unsigned int* status = nullptr; // the result's status word (non-finite samples)
    std::vector<void*> owned;       // every buffer, prefix scratch included
    void release(Allocator& mem);
};

bf_status prepare_series(bf_ctx* ctx, const float* src, size_t N, uint32_t M, uint32_t M_pad,
                         int precision, cudaStream_t st, PreparedSeries* out, unsigned int* status);
// the two halves of prepare_series: buffers, then the kernels that fill them
// from ps.x[0..N)
bf_status prepare_series_alloc(bf_ctx* ctx, size_t N, uint32_t M, uint32_t M_pad, int precision,
                               PreparedSeries* out);
cudaError_t prepare_series_kernels(const PreparedSeries& ps, uint32_t M, int precision,
                                   cudaStream_t st);
// the same kernels for many series, one launch per kernel for MAX_PREP series
cudaError_t prepare_series_batch(const std::vector<const PreparedSeries*>& ps, uint32_t M, int precision,
                                 cudaStream_t st);
// prepare_series_alloc, then the copy of src into ps.x (no kernels)
bf_status prepare_series_copy(bf_ctx* ctx, const float* src, size_t N, uint32_t M, uint32_t M_pad,
                              int precision, cudaStream_t st, PreparedSeries* out, unsigned int* status);
void build_segments(const std::vector<PreparedSeries*>& ser, const std::vector<uint32_t>& ids,
                    const bf_bank* bank, size_t k_begin, size_t k_end, int precision,
                    unsigned long long* packed, double* sumsq, size_t K, std::vector<Seg>& segs);
bool is_device_ptr(const void* p);
uint64_t ceil_div(uint64_t a, uint64_t b);
cudaError_t clear_result(bf_result* r, cudaStream_t st);
size_t prepared_series_bytes(size_t N, uint32_t M, uint32_t M_pad, int precision);

// Template-tile geometry of a precision's kernel.
inline uint32_t tile_templates(int precision) { return precision == BF_FP32 ? SIMT_TILE_T : TC_TILE_T; }
inline uint32_t tile_lags(int precision) { return precision == BF_FP32 ? SIMT_TILE_L : TC_TILE_L; }
// first template row of chirp k (quadrature banks hold two rows per chirp)
inline size_t bank_row(const bf_bank* b, size_t k) { return b->quad ? 2 * k : k; }
// the tensor-core precisions read the series as bf16 split rows
inline bool uses_split_rows(int precision)
{
    return precision == BF_BF16 || precision == BF_SPLIT_BF16 || precision == BF_SPLIT_FP16;
}

// One segment: series `ps` (result slot series_id) against template tiles
// [tt_first, tt_first + tt_count), keeping outputs of templates [k_begin, k_end).
Seg make_segment(const PreparedSeries& ps, uint32_t series_id, const bf_bank* bank, size_t k_begin,
                 size_t k_end, uint32_t tt_first, uint32_t tt_count, int precision,
                 unsigned long long* packed_s, double* sumsq_s, float* rho = nullptr);

// lt: lags per tensor-core tile (256 or 512), 0 = autotuned; ignored by FP32
cudaError_t launch_segments(bf_ctx* ctx, const std::vector<Seg>& segs, int precision, float thr,
                            Candidate* cand, unsigned int* cand_count, unsigned int cand_cap,
                            cudaStream_t st, uint64_t* tiles_out, int lt = 0);
// The autotuner: lags per tile for this precision and template length, timed
// once per context on a synthetic problem over the segment's template tiles.
int choose_lag_tile(bf_ctx* ctx, const Seg& g, int precision, cudaStream_t st);

bf_status resolve_opts(const bf_bank* bank, const bf_opts* in, bf_opts* o);
bf_status alloc_result(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o,
                       const std::vector<size_t>& lengths, double fs, cudaStream_t st,
                       bf_result** out);
size_t result_bytes(const bf_bank* bank, const bf_opts& o, size_t N, double fs, size_t max_cand);
bf_status finalize_result(bf_ctx* ctx, const bf_bank* bank, bf_result* r, cudaStream_t st);
bf_status check_device_status(bf_ctx* ctx);
// BF_EINVAL if the result's status word says a series held a non-finite
// sample (reads it synchronously: call after the result's work is done)
bf_status result_status(const bf_result* r);
// debug builds: BF_EDEVICE if an output buffer was written past its end
constexpr size_t CANARY_BYTES = 256;
constexpr int CANARY_FILL = 0xA5;
bf_status check_canaries(const bf_result* r);

void serve_shutdown(bf_ctx* ctx);

// template half spectra of the FFT route, computed once per bank
bf_status bank_fft_spectra(bf_ctx* ctx, bf_bank* bank, cudaStream_t st);
// Two-slot rings in which a generated bank is synthesised chunk by chunk on
// the context's auxiliary stream while the main stream correlates the chunk
// before; events order the reuse of a slot after the launches that read it.
// The *_prepare calls allocate (into the result's scratch, which outlives the
// launches) and create the events, the launch calls only enqueue work, so a
// plan can capture them.  The events go with the ring.
struct RingEvents {
    cudaEvent_t start = nullptr, made[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    cudaError_t create();
    RingEvents() = default;
    RingEvents(const RingEvents&) = delete;
    RingEvents& operator=(const RingEvents&) = delete;
    ~RingEvents();
};
// direct routes: template tiles in the correlation kernels' layout (api.cu)
struct GenRing {
    void* slot[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    size_t chunk_tiles = 0, n_chunks = 0, t_begin = 0, t_end = 0;
    RingEvents ev;
};
// FFT route: template spectra (corr_fft.cu)
struct FftRing {
    float* scratch = nullptr;               // synthesised rows
    float2* slot[2] = {nullptr, nullptr};   // spectra
    size_t chunk = 0, synth_rows = 0, n_chunks = 0;
    RingEvents ev;
};
// bank rows [k0, k1) of a generated bank (k0 a multiple of 128) synthesised
// into the layout `precision` reads: FP32 rows at slot0, or the tensor-core
// tiles of the hi and lo parts at slot0 and slot1 (gen_slot_bytes each)
cudaError_t gen_synth_rows(const bf_bank* bank, int precision, size_t k0, size_t k1, void* slot0, void* slot1,
                           cudaStream_t s);
size_t gen_slot_bytes(const bf_bank* bank, int precision, size_t rows);
// a segment reading the rows synthesised from k0 into slot0 / slot1
void gen_point_segment(Seg& g, int precision, size_t k0, const void* slot0, const void* slot1);
// template spectra of the FFT route for bank rows [row0, row0 + nrows) (corr_fft.cu)
cudaError_t fft_template_spectra(const bf_bank* bank, size_t row0, size_t nrows, float* scratch,
                                 size_t scratch_rows, const float2* tw, float2* out, int n_sm, cudaStream_t st);
bf_status gen_prepare(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o, bf_result* r, GenRing* g);
cudaError_t gen_launch(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o, const std::vector<Seg>& segs,
                       bf_result* r, cudaStream_t strm, int lt, GenRing& g);
// the tile shape for a generated bank: the first chunk synthesised (on strm,
// synchronously) and the autotuner run on it; call before any capture
int gen_autotune(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o, const std::vector<Seg>& segs,
                 cudaStream_t strm, GenRing& g);
bf_status fft_ring_prepare(bf_ctx* ctx, const bf_bank* bank, uint32_t row_begin, uint32_t row_end,
                           std::vector<void*>& keep, FftRing* ring);

// one call of the FFT route: per batch of series, the segment-spectra job and
// the correlation record, and for a generated bank the spectra ring (api.cu)
struct FftCall {
    std::vector<FftSeriesBatch> series;
    std::vector<uint32_t> totals;
    std::vector<FftParams> batches;
    FftRing ring;
};
bf_status fft_prepare(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o,
                      const std::vector<PreparedSeries>& prep, bf_result* r, cudaStream_t st, FftCall* c);
cudaError_t fft_launch(bf_ctx* ctx, const bf_bank* bank, FftCall& c, bf_result* r, cudaStream_t st);
// the context's twiddle tables of the FFT route (built on first use)
cudaError_t fft_tables(bf_ctx* ctx, cudaStream_t st, const float2** out);
// Parseval predictor of the noise level of rho (predict.cu): predict_prepare
// allocates (into `scratch`, owned by the result) and makes the twiddle
// tables; predict_launch enqueues kernels only, so a plan can capture it.
// sigma of series s, output j goes to out[s * out_stride + j].
struct SigmaBatch;
struct PredictCall {
    const float2* tw = nullptr;
    uint32_t row_begin = 0, row_end = 0, n_out = 0, n_series = 0, chunk = 0;
    float* rows = nullptr;                  // synthesised template rows [chunk][FFT_POINTS]
    float* D = nullptr;                     // power dot products [n_series][rows]
    float* P = nullptr;                     // averaged periodograms [n_series][PRED_BINS]
    std::vector<WelchBatch> welch;
    std::vector<SigmaBatch*> sigma;
    PredictCall() = default;
    PredictCall(const PredictCall&) = delete;
    PredictCall& operator=(const PredictCall&) = delete;
    ~PredictCall();
};
bf_status predict_prepare(bf_ctx* ctx, const bf_bank* bank, const std::vector<const PreparedSeries*>& ps,
                          size_t k_begin, size_t k_end, float* out, size_t out_stride,
                          std::vector<void*>& scratch, cudaStream_t st, PredictCall* c);
cudaError_t predict_launch(bf_ctx* ctx, const bf_bank* bank, const PredictCall& c, cudaStream_t st);

}  // namespace bfi
