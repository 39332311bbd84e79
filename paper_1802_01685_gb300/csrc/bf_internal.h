// Internal declarations of the butterfly-filtering library (not part of the
// C ABI).  Geometry of the kernels, the launch record passed by value to the
// correlation kernels, and the host-side objects behind the opaque handles.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bf.h"

namespace bfi {

// ---------------------------------------------------------------- geometry
// Tensor-core path: one CTA tile is 128 templates (MMA M) x 512 lags (two MMAs
// with N = 256) and runs over the template length in stages of 64 samples.
constexpr int TC_TILE_T = 128;
constexpr int TC_TILE_L = 512;
constexpr int TC_BK = 64;
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 320;           // producer, MMA, 8 epilogue warps
// SIMT FP32 path: one block tile is 64 templates x 256 lags, 32-sample chunks.
constexpr int SIMT_TILE_T = 64;
constexpr int SIMT_TILE_L = 256;
constexpr int SIMT_BK = 32;
constexpr int SIMT_THREADS = 256;

constexpr int M_ALIGN = 64;               // template length padded to this
constexpr int K_ALIGN = 128;              // bank size padded to this
constexpr int MAX_SEG = 64;               // series (segments) per launch
constexpr uint32_t TILE_BYTES_A = TC_TILE_T * TC_BK * 2;   // 16 KiB per k-block

// device error codes written to the context's status word
enum : int { DEV_OK = 0, DEV_TIMEOUT_FULL = 1, DEV_TIMEOUT_EMPTY = 2,
             DEV_TIMEOUT_TMEM = 3, DEV_TMEM_ALLOC = 4, DEV_BOUNDS = 5 };

// Debug builds (-DBF_DEBUG_BOUNDS, built as libbf_debug.so): the kernels
// check the indices their outputs, staging buffers and tables rely on --
// invariants that the launch set-up guarantees, so a release build does not
// test them.  A failed check records DEV_BOUNDS in the context's status word
// (the first code recorded stays) and skips the access; the call then
// returns BF_EDEVICE.  Nothing traps.  In release builds BF_BOUNDS is `true`.
#ifdef BF_DEBUG_BOUNDS
__device__ __forceinline__ bool bounds_ok(int* err, bool ok)
{
    if (!ok && err) atomicCAS(err, DEV_OK, DEV_BOUNDS);
    return ok;
}
#define BF_BOUNDS(err, cond) (::bfi::bounds_ok((err), (cond)))
#else
#define BF_BOUNDS(err, cond) true
#endif

struct Candidate {
    uint32_t series;
    uint32_t k;        // absolute bank index
    uint32_t tau;
    float rho;
};

// One series searched against a contiguous range of template tiles.
struct Seg {
    const float* x;                 // FP32 samples, zero padded (SIMT path)
    const uint4* yhi;               // row w = bf16 hi parts of x[w .. w+7]
    const uint4* ylo;               // row w = bf16 lo parts of x[w .. w+7]
    const float* inv_norm;          // [L] 1 / |window|, 0 for empty windows
    const float* bank_f32;          // [K_pad][M_pad]
    const uint8_t* bank_hi;         // core-matrix tiles, see bank.cu
    const uint8_t* bank_lo;
    unsigned long long* vmax;       // packed max per template, index k - k_begin
    double* sumsq;                  // sum of rho^2 per template
    float* rho;                     // optional dense output [k - k_begin][tau]
    const float* sigma_pred;        // optional predicted sigma per template
                                    // (index k - k_begin): tails are then
                                    // |rho| >= kappa * sigma_pred[k]
    const uint32_t* xmax;           // split-FP16 only: float bits of max |x|, from
                                    // which the operand scales are derived
    const uint32_t* tile_kb;        // per 128-row template tile (absolute index):
                                    // kb_lo | kb_hi << 16, the 64-sample blocks
                                    // [kb_lo, kb_hi) outside which every row of
                                    // the tile is zero; the K loops skip the rest
    float kappa;
    float pad2;
    uint32_t bank_k0;               // template row held at the bank pointers
                                    // (0 for a stored bank, the chunk start
                                    // for a generated one)
    uint32_t quad;                  // rows 2c, 2c+1 are the quadrature pair of
                                    // chirp c: one output sqrt(rho_c^2 + rho_s^2)
    uint64_t tile_begin;            // first global tile index of this segment
    uint32_t L;                     // lags
    uint32_t n_lag_tiles;
    uint32_t tt0, n_tt;             // template tiles [tt0, tt0 + n_tt)
    uint32_t k_begin, k_end;        // template rows whose outputs are kept
    uint32_t M_pad;
    uint32_t series_id;
};

struct CorrParams {
    int n_seg;
    uint32_t idesc;                 // tcgen05 instruction descriptor (operand type)
    uint64_t total_tiles;
    float thr;                      // candidate threshold on |rho|
    unsigned int cand_cap;
    Candidate* cand;
    unsigned int* cand_count;
    int* err;                       // device status word
    uint32_t kchunk_log2;           // split routes: K blocks per accumulator chunk, log2
    uint32_t pad3;
    Seg seg[MAX_SEG];
};

// The FFT route (corr_fft.cu): complex transforms of FFT_POINTS points;
// overlap-save over segments of 2 FFT_POINTS samples (real route, plain banks:
// one template per transform) or FFT_POINTS samples (pair route, quadrature
// banks: a template and its partner per transform).
constexpr int FFT_POINTS = 8192;
constexpr int MAX_FFT_SER = 64;           // series per FFT launch
// A lag goes to the direct fixup when its window holds less than 1/16384 of
// the energy of its FFT segment (|x_seg| / |x_window| > 128): the transform's
// rounding error scales with the segment (measured: at most 3.5e-8 |x_seg| /
// |x_window| in rho), so beyond that ratio it could exceed a quarter of the
// bound on rho.
constexpr double FFT_FIX_RATIO2 = 16384.0;

struct ChirpDev;

struct FftSeries {
    const float2* spec;             // [nseg][fft_spec_bins] segment half spectra
    const float* inv;               // inverse window norms times the inverse
                                    // transform's scale, per segment
                                    // [nseg][Vp]; 0 at the lags left to the
                                    // direct fixup
    unsigned long long* vmax;       // packed max per template, index k - k_begin
    double* sumsq;
    float* rho;                     // optional dense output [k - k_begin][tau]
    const float* sigma_pred;        // optional per-template predicted sigma
    const float* x;                 // FP32 samples (for the direct fixup)
    const uint32_t* fix;            // lags left to the direct fixup, as pairs
                                    // (lag, float bits of its inverse norm) ...
    const uint32_t* n_fix;          // ... and how many
    float kappa;
    uint32_t L, nseg, series_id;
};

struct FftParams {
    const float2* hspec;            // template half spectra [.][fft_spec_bins]; row hrow0 first
    const float2* tw;               // twiddle tables (corr_fft.cu)
    uint32_t k_begin, k_end;        // template rows of the call (outputs count from k_begin)
    uint32_t k_lo, k_hi;            // template rows of this launch, within [k_begin, k_end)
    uint32_t hrow0;                 // template row held at hspec[0]
    int quad;                       // rows (2c, 2c+1) are a quadrature pair (pair route)
    uint32_t V;                     // valid lags per segment, fft_lags_per_seg
    uint32_t Vp;                    // row stride of the per-segment norms
    int n_ser;
    float thr;
    unsigned int cand_cap;
    Candidate* cand;
    unsigned int* cand_count;
    const ChirpDev* chirps;         // bank parameters (the fixup synthesises its rows)
    uint32_t M;                     // template length (at most FFT_POINTS / 2)
    double fs;
    int* err;                       // device status word (debug-build bounds checks)
    FftSeries ser[MAX_FFT_SER];
};

struct FftSeriesBatch {
    int n;
    int quad;                       // pair route (quadrature bank), else real route
    uint32_t F;                     // samples per segment, fft_seg_len(quad)
    uint32_t V;
    const float2* tw;
    const float* x[MAX_FFT_SER];
    uint64_t N[MAX_FFT_SER];
    float2* spec[MAX_FFT_SER];
    uint32_t seg_begin[MAX_FFT_SER];
    // lags for the direct fixup: found from the FP64 prefix of x^2 and the
    // inverse norms (zeroed there), listed in fix[i] as (lag, norm) pairs
    // (2 L words), counted in n_fix[i]
    const double* S[MAX_FFT_SER];
    float* inv[MAX_FFT_SER];
    float* inv_seg[MAX_FFT_SER];    // per-segment norms [nseg][Vp], times scale
    uint32_t Vp;
    float scale;
    uint32_t L[MAX_FFT_SER];
    uint32_t* fix[MAX_FFT_SER];
    uint32_t* n_fix;                // [n] counters, zeroed by launch_fft_series
    int* err;                       // device status word (debug-build bounds checks)
};

// The Parseval predictor (predict.cu, kernels in corr_fft.cu): periodograms
// averaged over Welch segments of PRED_F samples at hop PRED_F / 2, and
// template power spectra, both on the FFT route's real 16384-point transform.
constexpr int PRED_F = 2 * FFT_POINTS;
constexpr int PRED_BINS = FFT_POINTS + 1;     // one-sided bins 0 .. PRED_F / 2
struct WelchBatch {
    int n;
    const float2* tw;
    const float* x[MAX_FFT_SER];
    uint64_t N[MAX_FFT_SER];
    uint32_t seg_begin[MAX_FFT_SER + 1];      // series s: rows [seg_begin[s], seg_begin[s+1])
    float* pseg;                              // [total segments][PRED_BINS]
    float* P;                                 // [n][PRED_BINS] averaged periodograms
};

// A named range on the calling thread for profilers (NVTX: the ranges cost a
// few instructions when no profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- launchers
// Process-wide count of kernel launches made by this library.
extern std::atomic<uint64_t> g_launches;
bf_status cuda_fail(cudaError_t e, const char* what);
inline void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t launch_corr_simt(const CorrParams& p, cudaStream_t s);
cudaError_t launch_wait_selftest(int* err, int signal, uint64_t limit_ns, unsigned long long* waited,
                                 cudaStream_t st);
cudaError_t launch_corr_tc(const CorrParams& p, int nprod, int lt, int n_sm, cudaStream_t s);
// the instruction descriptor of a tensor-core precision (BF16 or FP16 operands)
uint32_t tc_idesc(int precision);
// sets the tensor-core kernels' shared-memory attribute (outside graph capture)
cudaError_t corr_tc_set_attributes();

struct ChirpDev {                   // device copy of a template's parameters
    int32_t track, sense;
    double f_lo, f_hi, D;
    double tc;                      // power-law t_c (0 for linear)
    int32_t MD;                     // support length M_D
    int32_t first;                  // m_s, first support sample of the
                                    // ascending template
};

// rows row0 .. row0 + K_pad - 1 of the bank into the output arrays (rows past
// row0 + K - 1 are zero); quad: row r is chirp r / 2, sine phase when r is odd
cudaError_t launch_bank_synth(const ChirpDev* params, uint32_t row0, int quad, uint32_t K, uint32_t K_pad,
                              uint32_t M, uint32_t M_pad, double fs, float* f32,
                              uint8_t* hi, uint8_t* lo, cudaStream_t s,
                              uint8_t* hi16 = nullptr, uint8_t* lo16 = nullptr);
// templates in the split-FP16 layout are scaled by this power of two
constexpr float TEMPLATE_F16_SCALE = 256.f;

// Series preparation, batched: one launch per kernel for up to MAX_PREP series
// (blockIdx.y is the series).  For each series: zero its padding x[N, xcap),
// the FP64 prefix of x^2 and of the nonzero count, the inverse window norms,
// and (mode 1) split-BF16 rows or (mode 2) split-FP16 rows of x 2^s, s from
// max |x| (written to *xmax as float bits).  status[i] (may be NULL): bit 0 set
// when the FP64 total of x^2 is not finite, i.e. when a sample is NaN or
// infinite.
constexpr int MAX_PREP = 64;
struct PrepBatch {
    int n;
    int mode;                       // 0: norms only, 1: + split-BF16 rows, 2: + split-FP16 rows
    uint32_t M;
    float* x[MAX_PREP];             // samples [0, N), padding [N, xcap)
    uint64_t N[MAX_PREP];
    uint64_t xcap[MAX_PREP];
    uint64_t nb[MAX_PREP];          // FP64 scan blocks of the series
    double* bsum[MAX_PREP];         // their sums: 2 nb doubles (energies, counts)
    double* S[MAX_PREP];            // prefix of x^2 [N + 1], then the uint32 counts [N + 1]
    float* inv[MAX_PREP];           // [N - M + 1]
    unsigned int* status[MAX_PREP];
    uint64_t rows[MAX_PREP];        // split rows
    uint4* yhi[MAX_PREP];
    uint4* ylo[MAX_PREP];
    uint32_t* xmax[MAX_PREP];
};
cudaError_t launch_prep(const PrepBatch& b, cudaStream_t s);
// scan blocks of a series of N samples, and the capacity of its block-sum scratch
uint64_t prep_scan_blocks(uint64_t N);

// The power-of-two exponent s that puts the largest |x| (float bits, >= 0) of a
// series in [2^13, 2^14) for its FP16 split; 0 for an all-zero series.  s is
// held to at most 118 so that 2^s and the epilogue's 2^-(s+8) stay normal
// floats (series whose largest |x| is below 2^-105 are scaled less).
__host__ __device__ inline int f16_series_shift(uint32_t max_bits)
{
    if (max_bits == 0) return 0;
    const int e = (int)(max_bits >> 23) - 127;         // floor(log2 max) for normal floats
    const int s = 13 - e;                              // >= 13 - 127 = -114
    return s > 118 ? 118 : s;
}
uint64_t inv_norm_scratch_blocks(uint64_t N);
// bytes of the prefix scratch: FP64 energies S[0..N], then uint32 counts C[0..N]
size_t prefix_bytes(uint64_t N);

struct FinalizeSeries {
    const unsigned long long* packed;
    const double* sumsq;
    float* vmax;
    int32_t* argmax;
    float* sigma;
    uint32_t* hist;
    float* map;
    uint32_t L;
    uint32_t nt;
};
constexpr int MAX_FIN = 128;        // series per finalize / paint launch
struct FinalizeParams {
    uint32_t s0, n;                 // series [s0, s0 + n) of the result
    uint32_t n_chirps;              // chirps of the bank (painted templates index them)
    int* err;                       // device status word (debug-build bounds checks)
    FinalizeSeries ser[MAX_FIN];
};
cudaError_t launch_finalize(const FinalizeParams& p, uint32_t K, uint32_t nbins, cudaStream_t s);
uint32_t welch_segments(uint64_t N);         // Welch segments of a series of N samples
cudaError_t launch_welch(const WelchBatch& b, int n_sm, cudaStream_t st);
cudaError_t launch_template_power_dot(const float* rows, uint32_t n_rows, const float2* tw, const float* P,
                                      uint32_t n_ser, float* D, uint32_t d_stride, uint32_t row0, int n_sm,
                                      cudaStream_t st);
uint32_t fft_seg_len(bool quad);            // samples per segment
uint32_t fft_spec_bins(bool quad);          // complex bins per segment or template spectrum
uint32_t fft_lags_per_seg(uint32_t M, bool quad);          // V = fft_seg_len - M + 1
uint32_t fft_norm_stride(uint32_t M, bool quad);           // Vp: V rounded up to a multiple of 4
float fft_inverse_scale(bool quad);
// a series' FFT-route scratch: its segment spectra [nseg][fft_spec_bins],
// then its window norms per segment [nseg][fft_norm_stride] (fft_seg_norms)
size_t fft_series_bytes(uint32_t L, uint32_t M, bool quad);
inline float* fft_seg_norms(float2* spec, uint32_t nseg, bool quad)
{
    return reinterpret_cast<float*>(spec + (size_t)nseg * fft_spec_bins(quad));
}
uint32_t fft_segments(uint32_t L, uint32_t M, bool quad);
cudaError_t launch_fft_series(const FftSeriesBatch& b, uint32_t total_segments, int n_sm, cudaStream_t st);
cudaError_t launch_corr_fft(const FftParams& p, int n_sm, cudaStream_t st);
// FFT route: template spectra in chunks, for banks whose spectra are not kept (corr_fft.cu)
struct FftRing;
cudaError_t fft_correlate_chunked(bf_ctx* ctx, const bf_bank* bank, std::vector<FftParams>& batches,
                                  uint32_t row_begin, uint32_t row_end, const FftRing& ring,
                                  cudaStream_t st);
// the nonzero cells of a map of n_cells floats, in increasing index: cell[i],
// value[i] for i < min(*total, cap), *total = their number; counts: scratch of
// map_cell_blocks(n_cells) words
uint64_t map_cell_blocks(uint64_t n_cells);
cudaError_t launch_map_cells(const float* map, uint64_t n_cells, uint32_t* counts, uint32_t* cell, float* value,
                             uint64_t cap, uint32_t* total, cudaStream_t s);
cudaError_t launch_coincidence(const float* A, const float* B, uint32_t nt, uint32_t nf, uint32_t w,
                               uint32_t dt, unsigned int* out, int n_sm, cudaStream_t s);
cudaError_t launch_skewnorm_fit(const float* v, uint64_t n, double* acc, double* out, int n_sm,
                                cudaStream_t s);
cudaError_t launch_mean_max(const float* vmax, uint32_t n_series, uint32_t K, float* mean,
                            cudaStream_t s);
cudaError_t launch_paint(const Candidate* cand, const unsigned int* count,
                         unsigned int cap, const ChirpDev* params,
                         const FinalizeParams& p, uint32_t M, double fs, double dt,
                         double df, uint32_t nf, unsigned int n_sm, cudaStream_t s);

// control randomisation
size_t permute_scratch_bytes(uint64_t n);
cudaError_t launch_permute(const float* in, uint64_t n, uint64_t seed, float* out,
                           void* scratch, cudaStream_t s);
// loads the permutation kernels' code on the current device (permute.cu)
cudaError_t preload_permute();
// set-up of the allocation-free control on `device` (noalloc.cu): loads the
// array of its scratch and the permutation kernels, and caches the array's
// device address (to *addr, if not NULL); called by bf_init for its device
bf_status static_control_setup(int device, void** addr = nullptr);

// ---------------------------------------------------------------- host side
void set_error(const char* fmt, ...);

struct Allocator {
    explicit Allocator(size_t budget) : budget_(budget) {}
    ~Allocator();
    void* alloc(size_t bytes);          // nullptr when over budget / OOM
    void release(void* p);
    void trim();
    size_t in_use() const;
    size_t budget() const { return budget_; }
    bool fits(size_t bytes) const;

  private:
    size_t budget_;
    size_t held_ = 0;                   // bytes obtained from cudaMalloc
    size_t live_ = 0;                   // bytes handed out
    std::multimap<size_t, void*> cache_;
    std::unordered_map<void*, size_t> size_of_;
    mutable std::mutex mu_;
};

struct ServeState;

}  // namespace bfi

struct bf_ctx {
    int device = 0;
    int n_sm = 0;
    bf_config cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;         // template synthesis of generated banks
    std::unique_ptr<bfi::Allocator> mem;
    int* d_err = nullptr;               // kernel status word
    std::mutex launch_mu;               // serialises use of d_err / stream
    bfi::ServeState* serve = nullptr;   // owned; freed by serve_shutdown
    std::map<std::pair<int, uint32_t>, int> tuned;   // (precision, M_pad) -> lags per tile
    float2* fft_tw = nullptr;           // twiddle tables of the FFT route (lazy, cudaMalloc)
    std::mutex tune_mu;
};

struct bf_bank {
    bf_ctx* ctx = nullptr;
    bool generated = false;             // parameters only; synthesised per call
    size_t K = 0, K_pad = 0;            // chirps; rows rounded up to the tile
    size_t rows = 0;                    // template rows: K, or 2K for quadrature pairs
    bool quad = false;
    uint32_t M = 0, M_pad = 0;
    double fs = 0, T = 0;
    unsigned storage = 0;
    std::vector<bf_chirp> params;
    bfi::ChirpDev* d_params = nullptr;
    float* f32 = nullptr;
    uint8_t* hi = nullptr;
    uint8_t* lo = nullptr;
    uint8_t* hi16 = nullptr;            // split-FP16 layout (2^8 h)
    uint8_t* lo16 = nullptr;
    uint32_t* tile_kb = nullptr;        // nonzero 64-sample block range per 128-row tile
    float2* fspec = nullptr;            // template half spectra for the FFT route (lazy)
};

struct bf_result {
    bf_ctx* ctx = nullptr;
    bool plan_owned = false;            // a plan's result: bf_result_destroy leaves it alone
    size_t n_series = 0, K = 0, k_begin = 0;
    uint32_t M = 0, nbins = 0;
    double fs = 0, dt = 0, df = 0;
    bool want_map = false, want_hist = false, want_tails = false, parseval = false;
    float kappa = 5.f;
    float* sigma_pred = nullptr;            // [S][K] predicted sigma (Parseval)
    std::vector<size_t> lengths;
    std::vector<uint32_t> map_nt;
    uint32_t map_nf = 0;
    // device buffers (owned)
    unsigned long long* packed = nullptr;   // [S][K]
    double* sumsq = nullptr;                // [S][K]
    float* vmax = nullptr;                  // [S][K]
    int32_t* argmax = nullptr;              // [S][K]
    float* sigma = nullptr;                 // [S][K]
    uint32_t* hist = nullptr;               // [S][nbins]
    float* map = nullptr;                   // concatenated per-series maps
    std::vector<size_t> map_off;            // element offsets into map
    size_t map_total = 0;
    uint32_t* cell_counts = nullptr;        // per-block scratch of bf_result_copy_map_cells_async
    std::vector<size_t> cell_off;           // each series' first block in it
    float* mean_max = nullptr;              // [K]
    bfi::Candidate* cand = nullptr;
    unsigned int* cand_count = nullptr;
    // device word after cand_count, zeroed with it: bit 0 is set by the series
    // preparation when a series holds a non-finite sample
    unsigned int* status = nullptr;
    unsigned int cand_cap = 0;
    uint64_t n_candidates = 0;
    float thr = 0;
    int tile_lags = 0;
    double correlations = 0;
    double kernel_ms = 0;
    std::vector<void*> scratch;             // released at destroy
    // debug builds: the canary past the end of each output buffer
    std::vector<unsigned char*> canaries;
};
