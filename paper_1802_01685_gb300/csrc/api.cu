// C ABI of the butterfly-filtering library: context, caching device allocator,
// template banks, the batched correlation call, results and the control.
// The serving loop lives in serve.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "bf_internal.h"
#include "runtime.h"

namespace bfi {

std::atomic<uint64_t> g_launches{0};

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

void set_error(const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

bf_status cuda_fail(cudaError_t e, const char* what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return BF_ECUDA;
}

// ---------------------------------------------------------------- allocator
static size_t round_alloc(size_t b)
{
    const size_t small = 512, big = 2u << 20;
    if (b <= big) return (b + small - 1) / small * small;
    return (b + big - 1) / big * big;
}

Allocator::~Allocator()
{
    trim();
    for (auto& kv : size_of_) cudaFree(kv.first);
}

void* Allocator::alloc(size_t bytes)
{
    if (bytes == 0) bytes = 1;
    const size_t b = round_alloc(bytes);
    std::lock_guard<std::mutex> g(mu_);
    auto it = cache_.lower_bound(b);
    if (it != cache_.end() && it->first <= b + b / 4 + 4096) {
        void* p = it->second;
        cache_.erase(it);
        live_ += size_of_[p];
        return p;
    }
    if (held_ + b > budget_) {
        for (auto& kv : cache_) {                      // give back cached blocks
            cudaFree(kv.second);
            held_ -= size_of_[kv.second];
            size_of_.erase(kv.second);
        }
        cache_.clear();
        if (held_ + b > budget_) return nullptr;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, b) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    held_ += b;
    live_ += b;
    size_of_[p] = b;
    return p;
}

void Allocator::release(void* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> g(mu_);
    auto it = size_of_.find(p);
    if (it == size_of_.end()) return;
    live_ -= it->second;
    cache_.emplace(it->second, p);
}

void Allocator::trim()
{
    std::lock_guard<std::mutex> g(mu_);
    for (auto& kv : cache_) {
        cudaFree(kv.second);
        held_ -= size_of_[kv.second];
        size_of_.erase(kv.second);
    }
    cache_.clear();
}

size_t Allocator::in_use() const
{
    std::lock_guard<std::mutex> g(mu_);
    return live_;
}

bool Allocator::fits(size_t bytes) const
{
    std::lock_guard<std::mutex> g(mu_);
    return live_ + round_alloc(bytes) <= budget_;
}

// ---------------------------------------------------------------- helpers
bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

uint32_t template_len(double T, double fs) { return (uint32_t)std::floor(T * fs + 0.5); }

static bool chirp_ok(const bf_chirp& c, double fs, uint32_t M, char* why, size_t n)
{
    if (c.track != BF_LINEAR && c.track != BF_POWERLAW) { snprintf(why, n, "bad track %d", c.track); return false; }
    if (c.sense != BF_ASC && c.sense != BF_DESC && c.sense != BF_BOTH) {
        snprintf(why, n, "bad sense %d", c.sense);
        return false;
    }
    if (!(c.f_lo > 0.0) || !(c.f_hi > c.f_lo) || !(c.f_hi < 0.5 * fs)) {
        snprintf(why, n, "need 0 < f_lo < f_hi < fs/2 (f_lo=%g f_hi=%g fs=%g)", c.f_lo, c.f_hi, fs);
        return false;
    }
    if (!(c.sweep_s > 0.0)) { snprintf(why, n, "sweep time must be positive"); return false; }
    const long MD = (long)std::floor(c.sweep_s * fs + 0.5);
    if (MD < 2 || MD > (long)M) { snprintf(why, n, "sweep of %ld samples outside [2, M=%u]", MD, M); return false; }
    return true;
}

// The samples [lo, hi) of the template row outside which it is zero: the
// ascending support [m_s, m_s + M_D), its mirror [M - m_s - M_D, M - m_s) for a
// descending chirp, and their union for both senses.  The quadrature partner
// has the same support.
static void row_support(const ChirpDev& d, uint32_t M, uint32_t& lo, uint32_t& hi)
{
    const uint32_t a0 = (uint32_t)d.first, a1 = a0 + (uint32_t)d.MD;
    const uint32_t d0 = M - a1, d1 = M - a0;
    if (d.sense == BF_ASC) { lo = a0; hi = a1; }
    else if (d.sense == BF_DESC) { lo = d0; hi = d1; }
    else { lo = std::min(a0, d0); hi = std::max(a1, d1); }
}

static ChirpDev to_dev(const bf_chirp& c, double fs, uint32_t M)
{
    ChirpDev d{};
    d.track = c.track;
    d.sense = c.sense;
    d.f_lo = c.f_lo;
    d.f_hi = c.f_hi;
    d.D = c.sweep_s;
    d.tc = c.track == BF_POWERLAW ? c.sweep_s / (1.0 - std::pow(c.f_lo / c.f_hi, 8.0 / 3.0)) : 0.0;
    d.MD = (int32_t)std::floor(c.sweep_s * fs + 0.5);
    d.first = (int32_t)((M - (uint32_t)d.MD) / 2);
    return d;
}

// ---------------------------------------------------------------- series prep
void PreparedSeries::release(Allocator& mem)
{
    for (void* p : owned) mem.release(p);
    owned.clear();
}

bf_status prepare_series_alloc(bf_ctx* ctx, size_t N, uint32_t M, uint32_t M_pad, int precision,
                               PreparedSeries* out)
{
    PreparedSeries& ps = *out;
    ps.N = N;
    ps.L = (uint32_t)(N - M + 1);
    Allocator& mem = *ctx->mem;
    auto grab = [&](size_t bytes) -> void* {
        void* p = mem.alloc(bytes);
        if (p) ps.owned.push_back(p);
        return p;
    };
    ps.xcap = ceil_div(ps.L, SIMT_TILE_L) * SIMT_TILE_L + M_pad + 1024;
    ps.x = static_cast<float*>(grab(ps.xcap * sizeof(float)));
    ps.inv = static_cast<float*>(grab((size_t)ps.L * sizeof(float)));
    ps.nb = inv_norm_scratch_blocks(N);
    ps.prefix = static_cast<double*>(grab(prefix_bytes(N)));
    ps.bsum = static_cast<double*>(grab(ps.nb * sizeof(double)));
    bool ok = ps.x && ps.inv && ps.prefix && ps.bsum;
    if (ok && uses_split_rows(precision)) {
        ps.rows = ceil_div(ps.L, TC_TILE_L) * TC_TILE_L + M_pad + 64;
        ps.yhi = static_cast<uint4*>(grab(ps.rows * 16));
        ps.ylo = static_cast<uint4*>(grab(ps.rows * 16));
        ok = ps.yhi && ps.ylo;
        if (ok && precision == BF_SPLIT_FP16) {
            ps.xmax = static_cast<uint32_t*>(grab(sizeof(uint32_t)));
            ok = ps.xmax != nullptr;
        }
    }
    if (!ok) {
        ps.release(mem);
        set_error("out of device memory preparing a series of %zu samples", N);
        return BF_ENOMEM;
    }
    return BF_OK;
}

cudaError_t prepare_series_batch(const std::vector<const PreparedSeries*>& ps, uint32_t M, int precision,
                                 cudaStream_t st)
{
    const int mode = precision == BF_SPLIT_FP16 ? 2 : uses_split_rows(precision) ? 1 : 0;
    for (size_t i0 = 0; i0 < ps.size(); i0 += MAX_PREP) {
        PrepBatch b{};
        b.n = (int)std::min<size_t>(MAX_PREP, ps.size() - i0);
        b.mode = mode;
        b.M = M;
        for (int i = 0; i < b.n; ++i) {
            const PreparedSeries& p = *ps[i0 + i];
            b.x[i] = p.x;
            b.N[i] = p.N;
            b.xcap[i] = p.xcap;
            b.nb[i] = prep_scan_blocks(p.N);
            if (2 * b.nb[i] > p.nb) return cudaErrorInvalidValue;      // the block-sum scratch
            b.bsum[i] = p.bsum;
            b.S[i] = p.prefix;
            b.inv[i] = p.inv;
            b.status[i] = p.status;
            b.rows[i] = p.rows;
            b.yhi[i] = p.yhi;
            b.ylo[i] = p.ylo;
            b.xmax[i] = p.xmax;
        }
        const cudaError_t e = launch_prep(b, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t prepare_series_kernels(const PreparedSeries& ps, uint32_t M, int precision,
                                   cudaStream_t st)
{
    return prepare_series_batch({&ps}, M, precision, st);
}

bf_status prepare_series_copy(bf_ctx* ctx, const float* src, size_t N, uint32_t M, uint32_t M_pad,
                              int precision, cudaStream_t st, PreparedSeries* out, unsigned int* status)
{
    bf_status s = prepare_series_alloc(ctx, N, M, M_pad, precision, out);
    if (s) return s;
    out->status = status;
    const cudaError_t e = cudaMemcpyAsync(out->x, src, N * sizeof(float), cudaMemcpyDefault, st);
    if (e != cudaSuccess) {
        out->release(*ctx->mem);
        return cuda_fail(e, "series copy");
    }
    return BF_OK;
}

bf_status prepare_series(bf_ctx* ctx, const float* src, size_t N, uint32_t M, uint32_t M_pad,
                         int precision, cudaStream_t st, PreparedSeries* out, unsigned int* status)
{
    bf_status s = prepare_series_copy(ctx, src, N, M, M_pad, precision, st, out, status);
    if (s) return s;
    const cudaError_t e = prepare_series_kernels(*out, M, precision, st);
    if (e != cudaSuccess) {
        out->release(*ctx->mem);
        return cuda_fail(e, "series preparation");
    }
    return BF_OK;
}

size_t prepared_series_bytes(size_t N, uint32_t M, uint32_t M_pad, int precision)
{
    const uint64_t L = N - M + 1;
    size_t b = (ceil_div(L, SIMT_TILE_L) * SIMT_TILE_L + M_pad + 1024) * 4 + L * 4 + prefix_bytes(N) +
               inv_norm_scratch_blocks(N) * 8;
    if (uses_split_rows(precision)) b += 2 * (ceil_div(L, TC_TILE_L) * TC_TILE_L + M_pad + 64) * 16;
    if (precision == BF_FFT_FP32) {                             // segment spectra (either route), fixup list
        b += std::max(fft_series_bytes((uint32_t)L, M, true), fft_series_bytes((uint32_t)L, M, false)) +
             (2 * L + 1) * 4;
    }
    if (precision == BF_SPLIT_FP16) b += 4096;                  // max |x|
    return b + 8 * 4096;
}

Seg make_segment(const PreparedSeries& ps, uint32_t series_id, const bf_bank* bank, size_t k_begin,
                 size_t k_end, uint32_t tt_first, uint32_t tt_count, int precision,
                 unsigned long long* packed_s, double* sumsq_s, float* rho)
{
    Seg g{};
    g.rho = rho;
    g.x = ps.x;
    g.yhi = ps.yhi;
    g.ylo = ps.ylo;
    g.inv_norm = ps.inv;
    g.bank_f32 = bank->f32;
    g.bank_hi = bank->hi;
    g.bank_lo = bank->lo;
    g.tile_kb = bank->tile_kb;
    g.vmax = packed_s;
    g.sumsq = sumsq_s;
    g.L = ps.L;
    g.n_lag_tiles = (uint32_t)ceil_div(ps.L, tile_lags(precision));
    g.tt0 = tt_first;
    g.n_tt = tt_count;
    if (precision == BF_SPLIT_FP16) {
        g.bank_hi = bank->hi16;
        g.bank_lo = bank->lo16;
        g.xmax = ps.xmax;
    }
    g.k_begin = (uint32_t)bank_row(bank, k_begin);
    g.k_end = (uint32_t)bank_row(bank, k_end);
    g.quad = bank->quad ? 1u : 0u;
    g.M_pad = bank->M_pad;
    g.series_id = series_id;
    return g;
}

// One segment per series over the whole template range.
void build_segments(const std::vector<PreparedSeries*>& ser, const std::vector<uint32_t>& ids,
                           const bf_bank* bank, size_t k_begin, size_t k_end, int precision,
                           unsigned long long* packed, double* sumsq, size_t K,
                           std::vector<Seg>& segs)
{
    const uint32_t tile_t = tile_templates(precision);
    const uint32_t tt0 = (uint32_t)(bank_row(bank, k_begin) / tile_t);
    const uint32_t ntt = (uint32_t)(ceil_div(bank_row(bank, k_end), tile_t) - tt0);
    for (size_t i = 0; i < ser.size(); ++i)
        segs.push_back(make_segment(*ser[i], ids[i], bank, k_begin, k_end, tt0, ntt, precision,
                                    packed + (size_t)ids[i] * K, sumsq + (size_t)ids[i] * K));
}

// Times both tile shapes of the tensor-core kernel on a zero series (its cost
// does not depend on the data) against up to 4 of the segment's template
// tiles, two waves of tiles each, and keeps the faster one per context.
int choose_lag_tile(bf_ctx* ctx, const Seg& g, int precision, cudaStream_t st)
{
    if (precision != BF_BF16) return TC_TILE_L / 2;      // the split routes have one shape
    const std::pair<int, uint32_t> key(precision, g.M_pad);
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) return it->second;
    }
    const uint32_t ntt = std::min<uint32_t>(g.n_tt, 4);
    const uint64_t L = (uint64_t)ctx->n_sm * TC_TILE_L * 2 / ntt + 1;
    const uint64_t rows = ceil_div(L, TC_TILE_L) * TC_TILE_L + g.M_pad + 64;
    Allocator& mem = *ctx->mem;
    void* yh = mem.alloc(rows * 16);
    void* yl = mem.alloc(rows * 16);
    void* inv = mem.alloc(L * 4);
    int best = TC_TILE_L;
    if (yh && yl && inv) {
        Seg t = g;
        t.yhi = static_cast<const uint4*>(yh);
        t.ylo = static_cast<const uint4*>(yl);
        t.inv_norm = static_cast<const float*>(inv);
        t.L = (uint32_t)L;
        t.n_tt = ntt;
        t.k_begin = t.k_end = 0;                  // no output is kept
        t.rho = nullptr;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaError_t e = cudaMemsetAsync(yh, 0, rows * 16, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(yl, 0, rows * 16, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(inv, 0, L * 4, st);
        float ms_best = 0.f;
        for (int lt : {TC_TILE_L, TC_TILE_L / 2}) {
            std::vector<Seg> one{t};
            float ms_min = 1e30f;
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                cudaEventRecord(e0, st);
                e = launch_segments(ctx, one, precision, INFINITY, nullptr, nullptr, 0, st, nullptr, lt);
                cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) ms_min = std::min(ms_min, ms);      // first run warms up
            }
            if (e == cudaSuccess && (lt == TC_TILE_L || ms_min < ms_best)) {
                if (lt != TC_TILE_L) best = lt;
                ms_best = ms_min;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) cudaGetLastError();
        if (ctx->cfg.log_level > 0)
            fprintf(stderr, "bf: autotune precision %d M_pad %u -> %d lags per tile\n", precision,
                    g.M_pad, best);
    }
    mem.release(yh);
    mem.release(yl);
    mem.release(inv);
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tuned[key] = best;
    return best;
}

cudaError_t launch_segments(bf_ctx* ctx, const std::vector<Seg>& segs, int precision, float thr,
                            Candidate* cand, unsigned int* cand_count, unsigned int cand_cap,
                            cudaStream_t st, uint64_t* tiles_out, int lt)
{
    if (precision != BF_FP32 && lt == 0 && !segs.empty()) lt = choose_lag_tile(ctx, segs[0], precision, st);
    if (precision == BF_FP32) lt = SIMT_TILE_L;
    uint64_t tiles = 0;
    for (size_t b = 0; b < segs.size(); b += MAX_SEG) {
        CorrParams p{};
        p.n_seg = (int)std::min(segs.size() - b, (size_t)MAX_SEG);
        uint64_t t = 0;
        for (int i = 0; i < p.n_seg; ++i) {
            p.seg[i] = segs[b + i];
            p.seg[i].n_lag_tiles = (uint32_t)ceil_div(p.seg[i].L, (uint64_t)lt);
            p.seg[i].tile_begin = t;
            t += (uint64_t)p.seg[i].n_lag_tiles * p.seg[i].n_tt;
        }
        p.total_tiles = t;
        p.thr = thr;
        p.cand = cand;
        p.cand_count = cand_count;
        p.cand_cap = cand_cap;
        p.err = ctx->d_err;
        p.idesc = tc_idesc(precision);
        // accumulator chunks of 2048 samples (split-BF16) or 1024 (split-FP16)
        p.kchunk_log2 = precision == BF_SPLIT_FP16 ? 4u : 5u;
        cudaError_t e = precision == BF_FP32 ? launch_corr_simt(p, st)
                                             : launch_corr_tc(p, precision == BF_BF16 ? 1 : 3,
                                                              lt, ctx->n_sm, st);
        if (e != cudaSuccess) return e;
        tiles += t;
    }
    if (tiles_out) *tiles_out = tiles;
    return cudaSuccess;
}

static void free_result_buffers(bf_result* r)
{
    Allocator& mem = *r->ctx->mem;
    for (void* p : {(void*)r->packed, (void*)r->sumsq, (void*)r->vmax, (void*)r->argmax,
                    (void*)r->sigma, (void*)r->hist, (void*)r->map, (void*)r->mean_max,
                    (void*)r->cand, (void*)r->cand_count, (void*)r->sigma_pred})
        mem.release(p);
    r->sigma_pred = nullptr;
    r->canaries.clear();
    for (void* p : r->scratch) mem.release(p);
    r->scratch.clear();
    r->packed = nullptr;
    r->sumsq = nullptr;
    r->vmax = nullptr;
    r->argmax = nullptr;
    r->sigma = nullptr;
    r->hist = nullptr;
    r->map = nullptr;
    r->mean_max = nullptr;
    r->cand = nullptr;
    r->cand_count = nullptr;
    r->status = nullptr;
}

void map_shape(size_t N, double fs, double dt, double df, uint32_t* nt, uint32_t* nf)
{
    *nt = (uint32_t)std::ceil((double)N / (fs * dt));
    *nf = (uint32_t)std::ceil((fs / 2.0) / df);
}

bf_status resolve_opts(const bf_bank* bank, const bf_opts* in, bf_opts* o)
{
    if (in) *o = *in;
    else bf_opts_default(o);
    if (o->bank_end == 0) o->bank_end = bank->K;
    if (o->bank_begin >= o->bank_end || o->bank_end > bank->K) {
        set_error("bank range [%zu, %zu) outside [0, %zu)", o->bank_begin, o->bank_end, bank->K);
        return BF_EINVAL;
    }
    if (o->precision != BF_FP32 && o->precision != BF_BF16 && o->precision != BF_SPLIT_BF16 &&
        o->precision != BF_FFT_FP32 && o->precision != BF_SPLIT_FP16) {
        set_error("unknown precision %d", o->precision);
        return BF_EINVAL;
    }
    if (o->precision == BF_FFT_FP32) {
        // spectra are synthesised from the parameters, whatever the bank stores
        if (bank->M > FFT_POINTS / 2) {
            set_error("the FFT route takes templates of at most %d samples (this bank: %u)",
                      FFT_POINTS / 2, bank->M);
            return BF_ENOTSUP;
        }
    } else if (bank->generated) {
        // synthesised per call in whichever layout the precision needs
    } else if (o->precision == BF_FP32 && !bank->f32) {
        set_error("bank keeps no FP32 layout (create it with BF_BANK_FP32)");
        return BF_EINVAL;
    }
    if (!bank->generated && o->precision == BF_SPLIT_FP16 && !bank->hi16) {
        set_error("bank keeps no split-FP16 layout (create it with BF_BANK_SPLIT_FP16)");
        return BF_EINVAL;
    }
    if (!bank->generated && (o->precision == BF_BF16 || o->precision == BF_SPLIT_BF16) && !bank->hi) {
        set_error("bank keeps no split-BF16 layout (create it with BF_BANK_SPLIT_BF16)");
        return BF_EINVAL;
    }
    if (o->tail_sigma != BF_SIGMA_WHITE && o->tail_sigma != BF_SIGMA_PARSEVAL) {
        set_error("unknown tail_sigma %d", o->tail_sigma);
        return BF_EINVAL;
    }
    if (o->tile_lags == TC_TILE_L && (o->precision == BF_SPLIT_BF16 || o->precision == BF_SPLIT_FP16)) {
        set_error("tile_lags 512 holds one accumulator and serves BF_BF16 only; the split "
                  "precisions accumulate K in chunks across two accumulators (use 0 or 256)");
        return BF_EINVAL;
    }
    if (o->tile_lags != 0 && o->tile_lags != TC_TILE_L && o->tile_lags != TC_TILE_L / 2) {
        set_error("tile_lags %d: use 0 (autotuned), 256 or 512", o->tile_lags);
        return BF_EINVAL;
    }
    if (!(o->kappa > 0.0)) o->kappa = 5.0;
    if (!(o->map_dt_s > 0.0)) o->map_dt_s = 1e-3;
    if (!(o->map_df_hz > 0.0)) o->map_df_hz = 4.0;
    if (o->hist_bins == 0) o->hist_bins = 1024;
    return BF_OK;
}

// Allocates and zeroes the outputs of a result for series of the given lengths.
bf_status alloc_result(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o,
                       const std::vector<size_t>& lengths, double fs, cudaStream_t st,
                       bf_result** out)
{
    std::unique_ptr<bf_result> r(new bf_result());
    r->ctx = ctx;
    r->n_series = lengths.size();
    r->K = o.bank_end - o.bank_begin;
    r->k_begin = o.bank_begin;
    r->M = bank->M;
    r->fs = fs;
    r->dt = o.map_dt_s;
    r->df = o.map_df_hz;
    r->nbins = o.hist_bins;
    r->want_map = o.want_map != 0;
    r->want_hist = o.want_hist != 0;
    r->want_tails = o.want_tails != 0;
    r->parseval = o.tail_sigma == BF_SIGMA_PARSEVAL;
    r->kappa = (float)o.kappa;
    r->lengths = lengths;
    // the white-noise rms of the output: 1/sqrt(M), or sqrt(2/M) for quadrature pairs
    r->thr = (float)(o.kappa * std::sqrt((bank->quad ? 2.0 : 1.0) / (double)bank->M));
    Allocator& mem = *ctx->mem;
    const size_t S = r->n_series, K = r->K;
    bf_result* rr = r.get();
    // an output buffer; debug builds pad it with a canary (checked after the
    // search by check_canaries)
    auto out_alloc = [&mem, rr](size_t bytes) -> void* {
#ifdef BF_DEBUG_BOUNDS
        unsigned char* p = static_cast<unsigned char*>(mem.alloc(bytes + CANARY_BYTES));
        if (p) rr->canaries.push_back(p + bytes);
        return p;
#else
        (void)rr;
        return mem.alloc(bytes);
#endif
    };
    r->packed = static_cast<unsigned long long*>(out_alloc(S * K * 8));
    r->sumsq = static_cast<double*>(out_alloc(S * K * 8));
    r->vmax = static_cast<float*>(out_alloc(S * K * 4));
    r->argmax = static_cast<int32_t*>(out_alloc(S * K * 4));
    r->sigma = static_cast<float*>(out_alloc(S * K * 4));
    r->mean_max = static_cast<float*>(out_alloc(K * 4));
    r->cand_cap = (unsigned int)std::min<size_t>(ctx->cfg.max_candidates, 0xFFFFFFF0u);
    if (!r->want_map && !r->want_tails) r->cand_cap = 0;
    r->cand = static_cast<Candidate*>(out_alloc(std::max<size_t>(r->cand_cap, 1) * sizeof(Candidate)));
    if (r->parseval) r->sigma_pred = static_cast<float*>(out_alloc(S * K * 4));
    r->cand_count = static_cast<unsigned int*>(mem.alloc(2 * sizeof(unsigned int)));
    r->status = r->cand_count ? r->cand_count + 1 : nullptr;
    bool ok = r->packed && r->sumsq && r->vmax && r->argmax && r->sigma && r->mean_max && r->cand &&
              r->cand_count && (!r->parseval || r->sigma_pred);
    if (ok && r->want_hist) {
        r->hist = static_cast<uint32_t*>(out_alloc(S * r->nbins * 4));
        ok = r->hist != nullptr;
    }
    size_t map_total = 0;
    r->map_nt.resize(S);
    for (size_t s = 0; s < S; ++s) {
        uint32_t nt, nf;
        map_shape(lengths[s], fs, r->dt, r->df, &nt, &nf);
        r->map_nt[s] = nt;
        r->map_nf = nf;
        r->map_off.push_back(map_total);
        map_total += (size_t)nt * nf;
    }
    if (ok && r->want_map) {
        r->map = static_cast<float*>(out_alloc(map_total * 4));
        size_t blocks = 0;
        for (size_t s = 0; s < S; ++s) {
            r->cell_off.push_back(blocks);
            blocks += map_cell_blocks((uint64_t)r->map_nt[s] * r->map_nf);
        }
        r->cell_counts = static_cast<uint32_t*>(mem.alloc(std::max<size_t>(blocks, 1) * sizeof(uint32_t)));
        if (r->cell_counts) r->scratch.push_back(r->cell_counts);
        ok = r->map != nullptr && r->cell_counts != nullptr;
    }
    if (!ok) {
        free_result_buffers(r.get());
        set_error("out of device memory for the result buffers");
        return BF_ENOMEM;
    }
    r->map_total = map_total;
    cudaError_t e = cudaSuccess;
    for (unsigned char* c : r->canaries)
        if (e == cudaSuccess) e = cudaMemsetAsync(c, CANARY_FILL, CANARY_BYTES, st);
    if (e == cudaSuccess) e = clear_result(r.get(), st);
    if (e != cudaSuccess) {
        free_result_buffers(r.get());
        return cuda_fail(e, "clearing result buffers");
    }
    *out = r.release();
    return BF_OK;
}

size_t result_bytes(const bf_bank* bank, const bf_opts& o, size_t N, double fs, size_t max_cand)
{
    const size_t K = o.bank_end - o.bank_begin;
    size_t b = K * (8 + 8 + 4 + 4 + 4 + 4) + 16 * 512;
    if (o.want_hist) b += (size_t)o.hist_bins * 4;
    if (o.want_map) {
        uint32_t nt, nf;
        map_shape(N, fs, o.map_dt_s, o.map_df_hz, &nt, &nf);
        b += (size_t)nt * nf * 4 + map_cell_blocks((uint64_t)nt * nf) * sizeof(uint32_t);
    }
    if (o.want_map || o.want_tails) b += max_cand * sizeof(Candidate);
    (void)bank;
    return b;
}

// Zeroes what the kernels accumulate into.
cudaError_t clear_result(bf_result* r, cudaStream_t st)
{
    const size_t S = r->n_series, K = r->K;
    cudaError_t e = cudaMemsetAsync(r->packed, 0, S * K * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->sumsq, 0, S * K * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->cand_count, 0, 2 * sizeof(unsigned int), st);
    if (e == cudaSuccess && r->hist) e = cudaMemsetAsync(r->hist, 0, S * r->nbins * 4, st);
    if (e == cudaSuccess && r->map) e = cudaMemsetAsync(r->map, 0, r->map_total * 4, st);
    return e;
}

// Finalize kernels for a result whose correlation launches are enqueued.
bf_status finalize_result(bf_ctx* ctx, const bf_bank* bank, bf_result* r, cudaStream_t st)
{
    const size_t S = r->n_series, K = r->K;
    cudaError_t e = cudaSuccess;
    for (size_t s0 = 0; s0 < S && e == cudaSuccess; s0 += MAX_FIN) {
        FinalizeParams fp{};
        fp.s0 = (uint32_t)s0;
        fp.n_chirps = (uint32_t)bank->K;
        fp.err = ctx->d_err;
        fp.n = (uint32_t)std::min(S - s0, (size_t)MAX_FIN);
        for (uint32_t i = 0; i < fp.n; ++i) {
            const size_t s = s0 + i;
            FinalizeSeries& f = fp.ser[i];
            f.packed = r->packed + s * K;
            f.sumsq = r->sumsq + s * K;
            f.vmax = r->vmax + s * K;
            f.argmax = r->argmax + s * K;
            f.sigma = r->sigma + s * K;
            f.hist = r->hist ? r->hist + s * r->nbins : nullptr;
            f.map = r->map ? r->map + r->map_off[s] : nullptr;
            f.L = (uint32_t)(r->lengths[s] - bank->M + 1);
            f.nt = r->map_nt[s];
        }
        e = launch_finalize(fp, (uint32_t)K, r->nbins, st);
        if (e == cudaSuccess && r->map)
            e = launch_paint(r->cand, r->cand_count, r->cand_cap, bank->d_params, fp, bank->M,
                             r->fs, r->dt, r->df, r->map_nf, (unsigned)ctx->n_sm, st);
    }
    if (e == cudaSuccess) e = launch_mean_max(r->vmax, (uint32_t)S, (uint32_t)K, r->mean_max, st);
    if (e != cudaSuccess) return cuda_fail(e, "finalize");
    return BF_OK;
}

// Generated bank: templates are synthesised in chunks of template tiles into a
// two-slot ring (~24 MiB per slot, so the ring stays in L2) on the auxiliary
// stream, and each chunk is correlated on the main stream as soon as it is
// ready; chunk c+1 is synthesised while chunk c is correlated.  Events order
// the reuse of a slot after the correlation that read it.  The segments in
// `segs` describe the whole call; each chunk restricts them to its tiles.
constexpr size_t GEN_SLOT_BYTES = 24u << 20;

cudaError_t RingEvents::create()
{
    cudaError_t e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&made[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&used[i], cudaEventDisableTiming);
    }
    return e;
}

// events may be destroyed while pending work still references them
RingEvents::~RingEvents()
{
    if (start) cudaEventDestroy(start);
    for (int i = 0; i < 2; ++i) {
        if (made[i]) cudaEventDestroy(made[i]);
        if (used[i]) cudaEventDestroy(used[i]);
    }
}

bf_status gen_prepare(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o, bf_result* r, GenRing* g)
{
    const bool tc = o.precision != BF_FP32;
    const size_t tile_bytes = (size_t)TC_TILE_T * bank->M_pad * 4;     // hi+lo, or FP32
    g->chunk_tiles = std::max<size_t>(1, GEN_SLOT_BYTES / tile_bytes);
    g->t_begin = bank_row(bank, o.bank_begin) / TC_TILE_T;
    g->t_end = ceil_div(bank_row(bank, o.bank_end), TC_TILE_T);
    g->n_chunks = ceil_div(g->t_end - g->t_begin, g->chunk_tiles);
    const size_t slot_bytes = gen_slot_bytes(bank, o.precision,
                                             std::min(g->chunk_tiles, g->t_end - g->t_begin) * TC_TILE_T);
    Allocator& mem = *ctx->mem;
    for (int i = 0; i < 2 && i < (int)g->n_chunks; ++i)
        for (int j = 0; j < (tc ? 2 : 1); ++j) {
            g->slot[i][j] = mem.alloc(slot_bytes);
            if (!g->slot[i][j]) {
                set_error("out of device memory for the synthesis ring");
                return BF_ENOMEM;
            }
            r->scratch.push_back(g->slot[i][j]);
        }
    cudaError_t e = g->ev.create();
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "ring events");
}

cudaError_t gen_synth_rows(const bf_bank* bank, int precision, size_t k0, size_t k1, void* slot0, void* slot1,
                           cudaStream_t s)
{
    const bool tc = precision != BF_FP32;
    const bool f16 = precision == BF_SPLIT_FP16;
    const size_t kc = std::min(k1, bank->rows) - k0;
    return launch_bank_synth(bank->d_params, (uint32_t)k0, bank->quad, (uint32_t)kc, (uint32_t)(k1 - k0),
                             bank->M, bank->M_pad, bank->fs,
                             tc ? nullptr : static_cast<float*>(slot0),
                             tc && !f16 ? static_cast<uint8_t*>(slot0) : nullptr,
                             tc && !f16 ? static_cast<uint8_t*>(slot1) : nullptr, s,
                             f16 ? static_cast<uint8_t*>(slot0) : nullptr,
                             f16 ? static_cast<uint8_t*>(slot1) : nullptr);
}

void gen_point_segment(Seg& g, int precision, size_t k0, const void* slot0, const void* slot1)
{
    const bool tc = precision != BF_FP32;
    g.bank_k0 = (uint32_t)k0;
    g.bank_f32 = tc ? nullptr : static_cast<const float*>(slot0);
    g.bank_hi = tc ? static_cast<const uint8_t*>(slot0) : nullptr;
    g.bank_lo = tc ? static_cast<const uint8_t*>(slot1) : nullptr;
}

size_t gen_slot_bytes(const bf_bank* bank, int precision, size_t rows)
{
    return rows * bank->M_pad * (precision != BF_FP32 ? 2 : 4);    // per plane (hi, lo) or FP32
}

// synthesis of chunk c of a generated bank into slot sl, on stream s
static cudaError_t gen_synth(const bf_bank* bank, const bf_opts& o, const GenRing& g, size_t c, int sl,
                             cudaStream_t s)
{
    const size_t t0 = g.t_begin + c * g.chunk_tiles;
    const size_t t1 = std::min(t0 + g.chunk_tiles, g.t_end);
    return gen_synth_rows(bank, o.precision, t0 * TC_TILE_T, t1 * TC_TILE_T, g.slot[sl][0], g.slot[sl][1], s);
}

// the call's segments restricted to chunk c's template tiles, reading slot sl
static std::vector<Seg> gen_chunk_segments(const bf_bank* bank, const bf_opts& o, const std::vector<Seg>& segs,
                                           const GenRing& g, size_t c, int sl)
{
    const size_t t0 = g.t_begin + c * g.chunk_tiles;
    const size_t t1 = std::min(t0 + g.chunk_tiles, g.t_end);
    const size_t k0 = t0 * TC_TILE_T;
    const uint32_t tile_t = tile_templates(o.precision);
    const size_t q0 = std::max(k0, bank_row(bank, o.bank_begin)) / tile_t;
    const size_t q1 = ceil_div(std::min(t1 * TC_TILE_T, bank_row(bank, o.bank_end)), tile_t);
    std::vector<Seg> cs = segs;
    for (Seg& s : cs) {
        s.tt0 = (uint32_t)q0;
        s.n_tt = (uint32_t)(q1 - q0);
        gen_point_segment(s, o.precision, k0, g.slot[sl][0], g.slot[sl][1]);
    }
    return cs;
}

int gen_autotune(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o, const std::vector<Seg>& segs,
                 cudaStream_t strm, GenRing& g)
{
    if (gen_synth(bank, o, g, 0, 0, strm) != cudaSuccess) return TC_TILE_L / 2;
    return choose_lag_tile(ctx, gen_chunk_segments(bank, o, segs, g, 0, 0)[0], o.precision, strm);
}

cudaError_t gen_launch(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o, const std::vector<Seg>& segs,
                       bf_result* r, cudaStream_t strm, int lt, GenRing& g)
{
    const RingEvents& ev = g.ev;
    // the synthesis stream starts after everything already queued on the main one
    cudaError_t e = cudaEventRecord(ev.start, strm);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux, ev.start, 0);
    for (size_t c = 0; c < g.n_chunks && e == cudaSuccess; ++c) {
        const int sl = (int)(c & 1);
        if (c >= 2) e = cudaStreamWaitEvent(ctx->aux, ev.used[sl], 0);
        if (e == cudaSuccess) e = gen_synth(bank, o, g, c, sl, ctx->aux);
        if (e == cudaSuccess) e = cudaEventRecord(ev.made[sl], ctx->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(strm, ev.made[sl], 0);
        if (e != cudaSuccess) break;
        std::vector<Seg> cs = gen_chunk_segments(bank, o, segs, g, c, sl);
        if (lt == 0) {
            lt = choose_lag_tile(ctx, cs[0], o.precision, strm);
            r->tile_lags = lt;
        }
        e = launch_segments(ctx, cs, o.precision, r->thr, r->cand, r->cand_count, r->cand_cap, strm,
                            nullptr, lt);
        if (e == cudaSuccess) e = cudaEventRecord(ev.used[sl], strm);
    }
    return e;
}

bf_status check_canaries(const bf_result* r)
{
    for (size_t i = 0; i < r->canaries.size(); ++i) {
        unsigned char h[CANARY_BYTES];
        cudaError_t e = cudaMemcpy(h, r->canaries[i], CANARY_BYTES, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "reading an output canary");
        for (size_t b = 0; b < CANARY_BYTES; ++b)
            if (h[b] != CANARY_FILL) {
                set_error("output buffer %zu was written past its end (canary byte %zu)", i, b);
                return BF_EDEVICE;
            }
    }
    return BF_OK;
}

bf_status result_status(const bf_result* r)
{
    unsigned int w = 0;
    cudaError_t e = cudaMemcpy(&w, r->status, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the result status");
    if (w & 1u) {
        set_error("a series holds a non-finite sample (NaN or infinity)");
        return BF_EINVAL;
    }
    return BF_OK;
}

bf_status check_device_status(bf_ctx* ctx)
{
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading kernel status");
    if (h != DEV_OK) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (h == DEV_BOUNDS) set_error("a kernel's bounds check failed (debug build)");
        else set_error("kernel reported internal timeout (code %d)", h);
        return BF_EDEVICE;
    }
    return BF_OK;
}

// The FFT route, in two halves so that a plan can capture the second:
// fft_prepare makes the twiddle tables and allocates each batch's segment
// spectra (kept in the result's scratch until it is destroyed) and fills the
// launch records; fft_launch enqueues kernels only: the segment spectra of
// every batch of up to MAX_FFT_SER series, then the correlation over all
// template pairs of the bank range (spectra kept with a stored bank, made
// chunk by chunk for a generated one).
bf_status fft_prepare(bf_ctx* ctx, const bf_bank* bank, const bf_opts& o,
                      const std::vector<PreparedSeries>& prep, bf_result* r, cudaStream_t st, FftCall* c)
{
    const size_t S = prep.size(), K = r->K;
    const bool quad = bank->quad;
    const uint32_t V = fft_lags_per_seg(bank->M, quad);
    const float2* tw = nullptr;
    cudaError_t e = fft_tables(ctx, st, &tw);
    if (e != cudaSuccess) return cuda_fail(e, "FFT tables");
    for (size_t s0 = 0; s0 < S; s0 += MAX_FFT_SER) {
        const int n = (int)std::min<size_t>(MAX_FFT_SER, S - s0);
        FftSeriesBatch b{};
        FftParams p{};
        uint32_t total = 0;
        b.n_fix = static_cast<uint32_t*>(ctx->mem->alloc((size_t)n * sizeof(uint32_t)));
        if (!b.n_fix) {
            set_error("out of device memory for the fixup lists");
            return BF_ENOMEM;
        }
        r->scratch.push_back(b.n_fix);
        for (int i = 0; i < n; ++i) {
            const size_t s = s0 + i;
            const uint32_t nseg = fft_segments(prep[s].L, bank->M, quad);
            float2* spec = static_cast<float2*>(ctx->mem->alloc(fft_series_bytes(prep[s].L, bank->M, quad)));
            uint32_t* fix = static_cast<uint32_t*>(ctx->mem->alloc((size_t)prep[s].L * 2 * sizeof(uint32_t)));
            if (spec) r->scratch.push_back(spec);
            if (fix) r->scratch.push_back(fix);
            if (!spec || !fix) {
                set_error("out of device memory for the segment spectra");
                return BF_ENOMEM;
            }
            b.x[i] = prep[s].x;
            b.N[i] = prep[s].N;
            b.spec[i] = spec;
            b.seg_begin[i] = total;
            b.S[i] = prep[s].prefix;
            b.inv[i] = prep[s].inv;
            b.inv_seg[i] = fft_seg_norms(spec, nseg, quad);
            b.L[i] = (uint32_t)prep[s].L;
            b.fix[i] = fix;
            total += nseg;
            FftSeries& f = p.ser[i];
            f.spec = spec;
            f.inv = b.inv_seg[i];
            f.x = prep[s].x;
            f.fix = fix;
            f.n_fix = b.n_fix + i;
            f.vmax = r->packed + s * K;
            f.sumsq = r->sumsq + s * K;
            f.rho = s == 0 ? o.rho_out : nullptr;
            f.sigma_pred = r->sigma_pred ? r->sigma_pred + s * K : nullptr;
            f.kappa = r->kappa;
            f.L = prep[s].L;
            f.nseg = nseg;
            f.series_id = (uint32_t)s;
        }
        b.n = n;
        b.err = ctx->d_err;
        p.err = ctx->d_err;
        b.quad = quad ? 1 : 0;
        b.F = fft_seg_len(quad);
        b.V = V;
        b.Vp = fft_norm_stride(bank->M, quad);
        b.scale = fft_inverse_scale(quad);
        b.tw = tw;
        p.tw = tw;
        p.k_begin = (uint32_t)bank_row(bank, o.bank_begin);
        p.k_end = (uint32_t)bank_row(bank, o.bank_end);
        p.quad = bank->quad ? 1 : 0;
        p.V = V;
        p.Vp = b.Vp;
        p.n_ser = n;
        p.thr = r->thr;
        p.cand_cap = r->cand_cap;
        p.cand = r->cand;
        p.cand_count = r->cand_count;
        p.chirps = bank->d_params;
        p.M = bank->M;
        p.fs = bank->fs;
        c->series.push_back(b);
        c->totals.push_back(total);
        c->batches.push_back(p);
    }
    if (bank->generated && !c->batches.empty())
        return fft_ring_prepare(ctx, bank, c->batches[0].k_begin, c->batches[0].k_end, r->scratch, &c->ring);
    return BF_OK;
}

cudaError_t fft_launch(bf_ctx* ctx, const bf_bank* bank, FftCall& c, bf_result* r, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < c.series.size() && e == cudaSuccess; ++i)
        e = launch_fft_series(c.series[i], c.totals[i], ctx->n_sm, st);
    if (e != cudaSuccess || c.batches.empty()) return e;
    const uint32_t r0 = c.batches[0].k_begin, r1 = c.batches[0].k_end;
    if (bank->generated) return fft_correlate_chunked(ctx, bank, c.batches, r0, r1, c.ring, st);
    // spectra kept with the bank
    for (FftParams& p : c.batches) {
        p.hspec = bank->fspec;
        p.hrow0 = 0;
        p.k_lo = r0;
        p.k_hi = r1;
        e = launch_corr_fft(p, ctx->n_sm, st);
        if (e != cudaSuccess) break;
    }
    return e;
}

}  // namespace bfi

using namespace bfi;

// =================================================================== C ABI
extern "C" {

const char* bf_last_error(void) { return g_err.c_str(); }
int bf_abi_version(void) { return BF_ABI_VERSION; }

bf_status bf_selftest_wait(bf_ctx* ctx, int signal, uint32_t limit_us, double* waited_us)
{
    if (!ctx) { set_error("NULL context"); return BF_EINVAL; }
    if (limit_us == 0 || limit_us > 1000000u) { set_error("limit_us must be in [1, 1e6]"); return BF_EINVAL; }
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    unsigned long long* w = static_cast<unsigned long long*>(ctx->mem->alloc(sizeof(unsigned long long)));
    if (!w) { set_error("out of device memory"); return BF_ENOMEM; }
    cudaError_t e = launch_wait_selftest(ctx->d_err, signal, (uint64_t)limit_us * 1000ull, w, ctx->stream);
    unsigned long long ns = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, w, sizeof ns, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->mem->release(w);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    if (waited_us) *waited_us = (double)ns / 1e3;
    return check_device_status(ctx);
}
uint64_t bf_kernel_launches(void) { return g_launches.load(); }

const char* bf_status_string(bf_status s)
{
    switch (s) {
    case BF_OK: return "ok";
    case BF_EINVAL: return "invalid argument";
    case BF_ENOMEM: return "out of memory";
    case BF_ECUDA: return "CUDA error";
    case BF_ETIMEDOUT: return "timed out";
    case BF_EPENDING: return "pending";
    case BF_EAGAIN: return "queue full";
    case BF_ECANCELED: return "cancelled";
    case BF_EDEVICE: return "device-side error";
    case BF_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

void bf_config_default(bf_config* c)
{
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->device = 0;
    c->hbm_budget = 0;
    c->max_candidates = 1u << 22;
    c->serve_slots = 8;
    c->serve_queue = 1024;
    c->log_level = 0;
    c->serve_policy = BF_SERVE_FAIR;
}

void bf_opts_default(bf_opts* o)
{
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = BF_SPLIT_BF16;
    o->kappa = 5.0;
    o->map_dt_s = 1e-3;
    o->map_df_hz = 4.0;
    o->want_hist = 1;
    o->hist_bins = 1024;
}

bf_status bf_init(const bf_config* cfg, bf_ctx** out)
{
    if (!out) { set_error("out is NULL"); return BF_EINVAL; }
    *out = nullptr;
    bf_config c;
    if (cfg) c = *cfg;
    else bf_config_default(&c);
    if (c.max_candidates == 0) c.max_candidates = 1u << 22;
    if (c.serve_slots <= 0) c.serve_slots = 8;
    if (c.serve_queue <= 0) c.serve_queue = 1024;
    if (c.serve_policy != BF_SERVE_FAIR && c.serve_policy != BF_SERVE_SHORTEST) {
        set_error("serve_policy %d is not a bf_serve_policy", c.serve_policy);
        return BF_EINVAL;
    }
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (c.device < 0 || c.device >= n) { set_error("device %d of %d", c.device, n); return BF_EINVAL; }
    e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaDeviceProp prop{};
    e = cudaGetDeviceProperties(&prop, c.device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3)) {
        set_error("device %d is sm_%d%d; this library is built for sm_103a", c.device, prop.major,
                  prop.minor);
        return BF_ENOTSUP;
    }
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    if (c.hbm_budget == 0) c.hbm_budget = (size_t)(0.9 * (double)fr);
    std::unique_ptr<bf_ctx> ctx(new bf_ctx());
    ctx->device = c.device;
    ctx->n_sm = prop.multiProcessorCount;
    ctx->cfg = c;
    ctx->mem.reset(new Allocator(c.hbm_budget));
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaStreamDestroy(ctx->stream);
        return cuda_fail(e, "status word");
    }
    // the allocation-free control's set-up on this device, so that a caller
    // holding a context never has it happen at its first control
    bf_status st = static_control_setup(c.device);
    if (st) {
        cudaFree(ctx->d_err);
        cudaStreamDestroy(ctx->stream);
        cudaStreamDestroy(ctx->aux);
        return st;
    }
    *out = ctx.release();
    return BF_OK;
}

void bf_destroy(bf_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    cudaStreamSynchronize(ctx->stream);
    ctx->mem.reset();
    cudaFree(ctx->d_err);
    if (ctx->fft_tw) cudaFree(ctx->fft_tw);
    cudaStreamDestroy(ctx->stream);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    delete ctx;
}

bf_status bf_bank_create(bf_ctx* ctx, const bf_chirp* params, size_t K, double fs, double T,
                         unsigned storage, bf_bank** out)
{
    NvtxRange range("bf_bank_create");
    if (!ctx || !params || !out) { set_error("NULL argument"); return BF_EINVAL; }
    *out = nullptr;
    if (K == 0 || K > 0x7FFFFF00u) { set_error("bank size %zu outside [1, 2^31)", K); return BF_EINVAL; }
    if (!(fs > 0.0) || !(T > 0.0)) { set_error("need fs > 0 and T > 0"); return BF_EINVAL; }
    const bool quad = (storage & BF_BANK_QUADRATURE) != 0;
    const unsigned layout = storage & ~(unsigned)BF_BANK_QUADRATURE;
    const bool generated = layout == BF_BANK_GENERATED;
    const unsigned stored = BF_BANK_FP32 | BF_BANK_SPLIT_BF16 | BF_BANK_SPLIT_FP16;
    if (!generated && ((layout & stored) == 0 || (layout & ~stored))) {
        set_error("storage mask %u must be BF_BANK_GENERATED alone, or select any of BF_BANK_FP32, "
                  "BF_BANK_SPLIT_BF16 and BF_BANK_SPLIT_FP16 (either way optionally with "
                  "BF_BANK_QUADRATURE)", storage);
        return BF_EINVAL;
    }
    const uint32_t M = template_len(T, fs);
    if (M < 2 || M > BF_MAX_TEMPLATE_LEN) {
        set_error("template length %u outside [2, %d]", M, BF_MAX_TEMPLATE_LEN);
        return BF_EINVAL;
    }
    char why[256];
    for (size_t k = 0; k < K; ++k)
        if (!chirp_ok(params[k], fs, M, why, sizeof why)) {
            set_error("template %zu: %s", k, why);
            return BF_EINVAL;
        }
    cudaSetDevice(ctx->device);
    std::unique_ptr<bf_bank> b(new bf_bank());
    b->ctx = ctx;
    b->K = K;
    b->quad = quad;
    b->rows = quad ? 2 * K : K;
    b->K_pad = ceil_div(b->rows, K_ALIGN) * K_ALIGN;
    b->M = M;
    b->M_pad = (uint32_t)(ceil_div(M, M_ALIGN) * M_ALIGN);
    b->fs = fs;
    b->T = T;
    b->storage = storage;
    b->generated = generated;
    b->params.assign(params, params + K);
    std::vector<ChirpDev> dev(K);
    for (size_t k = 0; k < K; ++k) dev[k] = to_dev(params[k], fs, M);
    // per 128-row tile, the 64-sample blocks that hold any nonzero sample
    const size_t n_tiles = b->K_pad / TC_TILE_T;
    std::vector<uint32_t> tkb(n_tiles);
    for (size_t t = 0; t < n_tiles; ++t) {
        uint32_t lo = UINT32_MAX, hi = 0;
        for (size_t r = t * TC_TILE_T; r < std::min((t + 1) * TC_TILE_T, b->rows); ++r) {
            uint32_t a, z;
            row_support(dev[quad ? r / 2 : r], M, a, z);
            lo = std::min(lo, a);
            hi = std::max(hi, z);
        }
        const uint32_t kb_lo = lo < hi ? lo / TC_BK : 0;
        const uint32_t kb_hi = lo < hi ? (uint32_t)ceil_div(hi, TC_BK) : 1;
        tkb[t] = kb_lo | (kb_hi << 16);
    }
    Allocator& mem = *ctx->mem;
    b->d_params = static_cast<ChirpDev*>(mem.alloc(K * sizeof(ChirpDev)));
    b->tile_kb = static_cast<uint32_t*>(mem.alloc(n_tiles * sizeof(uint32_t)));
    const size_t elems = b->K_pad * (size_t)b->M_pad;
    if (storage & BF_BANK_FP32) b->f32 = static_cast<float*>(mem.alloc(elems * 4));
    if (storage & BF_BANK_SPLIT_BF16) {
        b->hi = static_cast<uint8_t*>(mem.alloc(elems * 2));
        b->lo = static_cast<uint8_t*>(mem.alloc(elems * 2));
    }
    if (storage & BF_BANK_SPLIT_FP16) {
        b->hi16 = static_cast<uint8_t*>(mem.alloc(elems * 2));
        b->lo16 = static_cast<uint8_t*>(mem.alloc(elems * 2));
    }
    if (!b->d_params || !b->tile_kb || ((storage & BF_BANK_FP32) && !b->f32) ||
        ((storage & BF_BANK_SPLIT_BF16) && (!b->hi || !b->lo)) ||
        ((storage & BF_BANK_SPLIT_FP16) && (!b->hi16 || !b->lo16))) {
        bf_bank_destroy(b.release());
        set_error("bank of %zu x %u samples exceeds the device memory budget", K, M);
        return BF_ENOMEM;
    }
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(b->d_params, dev.data(), K * sizeof(ChirpDev),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tile_kb, tkb.data(), n_tiles * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !generated)
        e = launch_bank_synth(b->d_params, 0, quad, (uint32_t)b->rows, (uint32_t)b->K_pad, M, b->M_pad, fs,
                              b->f32, b->hi, b->lo, st, b->hi16, b->lo16);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        bf_bank_destroy(b.release());
        return cuda_fail(e, "bank synthesis");
    }
    *out = b.release();
    return BF_OK;
}

bf_status bf_bank_create_grid(bf_ctx* ctx, const bf_chirp_grid* g, double fs, double T,
                              unsigned storage, bf_bank** out)
{
    if (!g || !g->tracks || !g->senses || !g->durations) { set_error("NULL grid"); return BF_EINVAL; }
    const size_t K = g->n_tracks * g->n_senses * g->n_durations * g->I * g->J;
    if (K == 0) { set_error("empty grid"); return BF_EINVAL; }
    if (!(g->f_max > g->f_min)) { set_error("need f_min < f_max"); return BF_EINVAL; }
    std::vector<bf_chirp> p;
    p.reserve(K);
    for (size_t a = 0; a < g->n_tracks; ++a)
        for (size_t s = 0; s < g->n_senses; ++s)
            for (size_t d = 0; d < g->n_durations; ++d)
                for (size_t i = 0; i < g->I; ++i) {
                    const double lo = g->f_min + (g->f_max - g->f_min) * (double)i / (double)g->I;
                    for (size_t j = 0; j < g->J; ++j) {
                        bf_chirp c;
                        c.track = g->tracks[a];
                        c.sense = g->senses[s];
                        c.f_lo = lo;
                        c.f_hi = lo + (g->f_max - lo) * (double)(j + 1) / (double)g->J;
                        c.sweep_s = g->durations[d];
                        p.push_back(c);
                    }
                }
    return bf_bank_create(ctx, p.data(), K, fs, T, storage, out);
}

void bf_bank_destroy(bf_bank* b)
{
    if (!b) return;
    Allocator& mem = *b->ctx->mem;
    cudaStreamSynchronize(b->ctx->stream);
    mem.release(b->fspec);
    mem.release(b->d_params);
    mem.release(b->f32);
    mem.release(b->hi);
    mem.release(b->lo);
    mem.release(b->hi16);
    mem.release(b->lo16);
    mem.release(b->tile_kb);
    delete b;
}

size_t bf_bank_size(const bf_bank* b) { return b ? b->K : 0; }
size_t bf_bank_rows(const bf_bank* b) { return b ? b->rows : 0; }
size_t bf_bank_template_len(const bf_bank* b) { return b ? b->M : 0; }

bf_status bf_bank_params(const bf_bank* b, size_t k0, size_t n, bf_chirp* out)
{
    if (!b || !out || k0 + n > b->K) { set_error("bad bank range"); return BF_EINVAL; }
    memcpy(out, b->params.data() + k0, n * sizeof(bf_chirp));
    return BF_OK;
}

bf_status bf_bank_read(const bf_bank* b, size_t c0, size_t nc, float* out)
{
    if (!b || !out || c0 + nc > b->K) { set_error("bad bank range"); return BF_EINVAL; }
    cudaSetDevice(b->ctx->device);
    const size_t k0 = bank_row(b, c0), n = bank_row(b, c0 + nc) - k0;     // rows
    if (b->generated) {
        // synthesise the range into a scratch FP32 block and copy it out
        const size_t n_pad = ceil_div(n, K_ALIGN) * K_ALIGN;
        float* tmp = static_cast<float*>(b->ctx->mem->alloc(n_pad * b->M_pad * sizeof(float)));
        if (!tmp) { set_error("out of device memory reading a generated bank"); return BF_ENOMEM; }
        std::lock_guard<std::mutex> g(b->ctx->launch_mu);
        cudaError_t e = launch_bank_synth(b->d_params, (uint32_t)k0, b->quad, (uint32_t)n, (uint32_t)n_pad,
                                          b->M, b->M_pad, b->fs, tmp, nullptr, nullptr, b->ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(out, b->M * sizeof(float), tmp, b->M_pad * sizeof(float),
                             b->M * sizeof(float), n, cudaMemcpyDeviceToHost);
        b->ctx->mem->release(tmp);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "generated bank read");
    }
    if (b->f32) {
        cudaError_t e = cudaMemcpy2D(out, b->M * sizeof(float), b->f32 + k0 * b->M_pad,
                                     b->M_pad * sizeof(float), b->M * sizeof(float), n,
                                     cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "bank read");
    }
    // split layout: copy whole 128-template tiles and decode hi + lo (BF16, or
    // FP16 of 2^8 h)
    const bool f16 = b->hi == nullptr;
    const uint8_t* dhi = f16 ? b->hi16 : b->hi;
    const uint8_t* dlo = f16 ? b->lo16 : b->lo;
    auto decode = [f16](uint16_t v) -> float {
        if (f16) {
            __half_raw r;
            r.x = v;
            return __half2float(__half(r)) / TEMPLATE_F16_SCALE;
        }
        uint32_t u = (uint32_t)v << 16;
        float f;
        memcpy(&f, &u, 4);
        return f;
    };
    const uint32_t n_kb = b->M_pad / TC_BK;
    const size_t tile_bytes = (size_t)n_kb * TILE_BYTES_A;
    std::vector<uint16_t> hi(tile_bytes / 2), lo(tile_bytes / 2);
    for (size_t tt = k0 / TC_TILE_T; tt * TC_TILE_T < k0 + n; ++tt) {
        cudaError_t e = cudaMemcpy(hi.data(), dhi + tt * tile_bytes, tile_bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(lo.data(), dlo + tt * tile_bytes, tile_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "bank read");
        for (uint32_t r = 0; r < TC_TILE_T; ++r) {
            const size_t k = tt * TC_TILE_T + r;
            if (k < k0 || k >= k0 + n) continue;
            for (uint32_t m = 0; m < b->M; ++m) {
                const uint32_t kb = m / TC_BK, c = m % TC_BK;
                const size_t off = ((size_t)kb * TILE_BYTES_A + (r / 8) * 1024 + (c / 8) * 128 +
                                    (r % 8) * 16 + (c % 8) * 2) / 2;
                out[(k - k0) * b->M + m] = decode(hi[off]) + decode(lo[off]);
            }
        }
    }
    return BF_OK;
}

bf_status bf_correlate(bf_ctx* ctx, const bf_bank* bank, const float* const* series,
                       const size_t* lengths, size_t n_series, double fs, const bf_opts* opts,
                       bf_result** out)
{
    NvtxRange range("bf_correlate");
    if (!ctx || !bank || !series || !lengths || !out || n_series == 0) {
        set_error("NULL argument or no series");
        return BF_EINVAL;
    }
    *out = nullptr;
    if (bank->ctx != ctx) { set_error("bank belongs to another context"); return BF_EINVAL; }
    if (std::fabs(fs - bank->fs) > 1e-9 * bank->fs) {
        set_error("series rate %g differs from the bank's %g", fs, bank->fs);
        return BF_EINVAL;
    }
    bf_opts o;
    bf_status st = resolve_opts(bank, opts, &o);
    if (st) return st;
    if (o.rho_out && n_series != 1) { set_error("rho_out needs exactly one series"); return BF_EINVAL; }
    if (o.rho_out && !is_device_ptr(o.rho_out)) { set_error("rho_out must be device memory"); return BF_EINVAL; }
    for (size_t s = 0; s < n_series; ++s) {
        if (!series[s]) { set_error("series %zu is NULL", s); return BF_EINVAL; }
        if (lengths[s] < bank->M || lengths[s] > 0xFFFFFFF0ull) {
            set_error("series %zu has %zu samples; need M=%u <= N < 2^32", s, lengths[s], bank->M);
            return BF_EINVAL;
        }
    }
    cudaSetDevice(ctx->device);
    const bool sync = o.stream == nullptr;
    cudaStream_t strm = sync ? ctx->stream : static_cast<cudaStream_t>(o.stream);
    std::lock_guard<std::mutex> g(ctx->launch_mu);

    std::vector<size_t> lens(lengths, lengths + n_series);
    bf_result* r = nullptr;
    st = alloc_result(ctx, bank, o, lens, fs, strm, &r);
    if (st) return st;
    std::unique_ptr<bf_result, void (*)(bf_result*)> guard(r, bf_result_destroy);

    std::vector<PreparedSeries> prep(n_series);
    std::vector<PreparedSeries*> pptr;
    std::vector<uint32_t> ids;
    for (size_t s = 0; s < n_series; ++s) {
        st = prepare_series_copy(ctx, series[s], lengths[s], bank->M, bank->M_pad, o.precision, strm,
                                 &prep[s], r->status);
        if (st) {
            for (auto& p : prep) p.release(*ctx->mem);
            return st;
        }
        for (void* p : prep[s].owned) r->scratch.push_back(p);
        prep[s].owned.clear();
        pptr.push_back(&prep[s]);
        ids.push_back((uint32_t)s);
        r->correlations += (double)prep[s].L * (double)r->K * (bank->quad ? 2.0 : 1.0);
    }
    {
        // every series' padding, prefix, norms and split rows: one launch per kernel
        const std::vector<const PreparedSeries*> pp(pptr.begin(), pptr.end());
        const cudaError_t ep = prepare_series_batch(pp, bank->M, o.precision, strm);
        if (ep != cudaSuccess) return cuda_fail(ep, "series preparation");
    }
    const bool fft = o.precision == BF_FFT_FP32;
    std::vector<Seg> segs;
    if (!fft) {
        build_segments(pptr, ids, bank, o.bank_begin, o.bank_end, o.precision, r->packed, r->sumsq, r->K,
                       segs);
        if (o.rho_out) segs[0].rho = o.rho_out;
    }
    if (r->parseval) {
        NvtxRange pr("predictor");
        // the predictor step: sigma_k per series before the search
        std::vector<const PreparedSeries*> pp;
        for (const PreparedSeries& p : prep) pp.push_back(&p);
        PredictCall pc;
        st = predict_prepare(ctx, bank, pp, o.bank_begin, o.bank_end, r->sigma_pred, r->K, r->scratch, strm,
                             &pc);
        if (st) return st;
        cudaError_t ep = predict_launch(ctx, bank, pc, strm);
        if (ep != cudaSuccess) return cuda_fail(ep, "predictor");
        for (size_t s = 0; s < segs.size(); ++s) {
            segs[s].sigma_pred = r->sigma_pred + s * r->K;
            segs[s].kappa = r->kappa;
        }
    }
    if (fft && !bank->generated) {
        // kept with the bank; a generated bank makes them chunk by chunk per call
        st = bank_fft_spectra(ctx, const_cast<bf_bank*>(bank), strm);
        if (st) return st;
    }
    FftCall fc;
    if (fft) {
        st = fft_prepare(ctx, bank, o, prep, r, strm, &fc);
        if (st) return st;
    }
    GenRing ring;
    if (!fft && bank->generated) {
        st = gen_prepare(ctx, bank, o, r, &ring);
        if (st) return st;
    }

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (sync) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, strm);
    }
    // lags per tile: fixed by the caller, else the autotuner's choice (for a
    // generated bank it is made on the first synthesised chunk)
    int lt = o.precision == BF_FP32 ? SIMT_TILE_L : fft ? 0 : o.tile_lags;
    if (lt == 0 && !fft && !bank->generated) lt = choose_lag_tile(ctx, segs[0], o.precision, strm);
    r->tile_lags = lt;
    cudaError_t e = fft ? fft_launch(ctx, bank, fc, r, strm)
                    : bank->generated
                        ? gen_launch(ctx, bank, o, segs, r, strm, lt, ring)
                        : launch_segments(ctx, segs, o.precision, r->thr, r->cand, r->cand_count,
                                          r->cand_cap, strm, nullptr, lt);
    if (sync) cudaEventRecord(e1, strm);
    if (e != cudaSuccess) {
        if (e0) { cudaEventDestroy(e0); cudaEventDestroy(e1); }
        return cuda_fail(e, "correlation launch");
    }
    {
        NvtxRange fr("finalize");
        st = finalize_result(ctx, bank, r, strm);
    }
    if (st) {
        if (e0) { cudaEventDestroy(e0); cudaEventDestroy(e1); }
        return st;
    }
    if (sync) {
        e = cudaStreamSynchronize(strm);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        r->kernel_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return cuda_fail(e, "correlation");
        st = check_device_status(ctx);
        if (st) return st;
        // debug builds: no output written past its end
        st = check_canaries(r);
        if (st) return st;
        // every sample must be finite (the series preparation flags it)
        st = result_status(r);
        for (size_t s = 0; st == BF_EINVAL && s < n_series; ++s) {
            // name the series: the one whose FP64 total of x^2 is not finite
            double total = 0.0;
            if (cudaMemcpy(&total, prep[s].prefix + prep[s].N, sizeof total, cudaMemcpyDeviceToHost) ==
                    cudaSuccess && !std::isfinite(total)) {
                set_error("series %zu holds a non-finite sample (NaN or infinity)", s);
                break;
            }
        }
        if (st) return st;
        unsigned int cnt = 0;
        cudaMemcpy(&cnt, r->cand_count, sizeof cnt, cudaMemcpyDeviceToHost);
        r->n_candidates = cnt;
        for (void* p : r->scratch) ctx->mem->release(p);
        r->scratch.clear();
    }
    *out = guard.release();
    return BF_OK;
}

bf_status bf_result_check(const bf_result* r)
{
    if (!r) { set_error("NULL argument"); return BF_EINVAL; }
    cudaSetDevice(r->ctx->device);
    bf_status st = check_device_status(r->ctx);
    if (st == BF_OK) st = check_canaries(r);
    return st ? st : result_status(r);
}

bf_status bf_result_info_get(const bf_result* r, bf_result_info* info)
{
    if (!r || !info) { set_error("NULL argument"); return BF_EINVAL; }
    memset(info, 0, sizeof *info);
    info->n_series = r->n_series;
    info->n_templates = r->K;
    info->template_len = r->M;
    info->correlations = r->correlations;
    info->useful_flops = 2.0 * r->M * r->correlations;
    uint64_t n = r->n_candidates;
    if (r->cand_count && n == 0) {
        unsigned int c = 0;
        if (cudaMemcpy(&c, r->cand_count, sizeof c, cudaMemcpyDeviceToHost) == cudaSuccess) n = c;
    }
    info->n_candidates = n;
    info->candidates_overflow = n > r->cand_cap ? 1 : 0;
    info->threshold = r->thr;
    info->hist_bins = r->nbins;
    info->kernel_ms = r->kernel_ms;
    info->tile_lags = r->tile_lags;
    return BF_OK;
}

bf_status bf_result_map_shape(const bf_result* r, size_t s, size_t* nt, size_t* nf)
{
    if (!r || s >= r->n_series) { set_error("bad series index"); return BF_EINVAL; }
    if (nt) *nt = r->map_nt[s];
    if (nf) *nf = r->map_nf;
    return BF_OK;
}

bf_status bf_result_get_max(const bf_result* r, size_t s, const float** vmax, const int32_t** argmax,
                            const float** sigma)
{
    if (!r || s >= r->n_series) { set_error("bad series index"); return BF_EINVAL; }
    if (vmax) *vmax = r->vmax + s * r->K;
    if (argmax) *argmax = r->argmax + s * r->K;
    if (sigma) *sigma = r->sigma + s * r->K;
    return BF_OK;
}

bf_status bf_result_get_hist(const bf_result* r, size_t s, const uint32_t** hist)
{
    if (!r || s >= r->n_series || !r->hist) { set_error("no histogram for this series"); return BF_EINVAL; }
    *hist = r->hist + s * r->nbins;
    return BF_OK;
}

bf_status bf_result_get_map(const bf_result* r, size_t s, const float** map)
{
    if (!r || s >= r->n_series || !r->map) { set_error("no map for this series"); return BF_EINVAL; }
    *map = r->map + r->map_off[s];
    return BF_OK;
}

bf_status bf_result_get_mean_max(const bf_result* r, const float** mean_max)
{
    if (!r || !mean_max) { set_error("NULL argument"); return BF_EINVAL; }
    *mean_max = r->mean_max;
    return BF_OK;
}

// The copies of bf_result_copy_to_host(_async): all enqueued on one stream,
// then waited for unless `async`.
static bf_status copy_series(const bf_result* r, size_t s, float* vmax, int32_t* argmax,
                             float* sigma, uint32_t* hist, float* map, cudaStream_t st, bool async)
{
    if (!r || s >= r->n_series) { set_error("bad series index"); return BF_EINVAL; }
    if (hist && !r->hist) { set_error("no histogram was requested"); return BF_EINVAL; }
    if (map && !r->map) { set_error("no map was requested"); return BF_EINVAL; }
    cudaSetDevice(r->ctx->device);
    const size_t K = r->K;
    const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (vmax) e = cudaMemcpyAsync(vmax, r->vmax + s * K, K * 4, d2h, st);
    if (e == cudaSuccess && argmax) e = cudaMemcpyAsync(argmax, r->argmax + s * K, K * 4, d2h, st);
    if (e == cudaSuccess && sigma) e = cudaMemcpyAsync(sigma, r->sigma + s * K, K * 4, d2h, st);
    if (e == cudaSuccess && hist) e = cudaMemcpyAsync(hist, r->hist + s * r->nbins, r->nbins * 4, d2h, st);
    if (e == cudaSuccess && map)
        e = cudaMemcpyAsync(map, r->map + r->map_off[s], (size_t)r->map_nt[s] * r->map_nf * 4, d2h, st);
    if (e == cudaSuccess && !async) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "result copy");
}

bf_status bf_result_copy_to_host(const bf_result* r, size_t s, float* vmax, int32_t* argmax,
                                 float* sigma, uint32_t* hist, float* map)
{
    if (!r) { set_error("NULL result"); return BF_EINVAL; }
    // the legacy default stream, as cudaMemcpy: ordered after work on blocking streams
    return copy_series(r, s, vmax, argmax, sigma, hist, map, cudaStreamLegacy, false);
}

bf_status bf_result_copy_to_host_async(const bf_result* r, size_t s, float* vmax, int32_t* argmax,
                                       float* sigma, uint32_t* hist, float* map, void* stream)
{
    if (!r) { set_error("NULL result"); return BF_EINVAL; }
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
    return copy_series(r, s, vmax, argmax, sigma, hist, map, st, true);
}

// a device address of p (device or managed memory, or page-locked host memory
// mapped into the device's address space), else nullptr
static void* device_view(void* p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

bf_status bf_result_copy_map_cells_async(const bf_result* r, size_t s, uint32_t* cell, float* value,
                                         size_t cap, uint32_t* count, void* stream)
{
    if (!r || !count || (cap && (!cell || !value))) { set_error("NULL argument"); return BF_EINVAL; }
    if (s >= r->n_series) { set_error("bad series index"); return BF_EINVAL; }
    if (!r->map) { set_error("no map was requested"); return BF_EINVAL; }
    const uint64_t n = (uint64_t)r->map_nt[s] * r->map_nf;
    if (n > 0xFFFFFFFFull) { set_error("map of %llu cells: more than 32-bit indices", (unsigned long long)n); return BF_ENOTSUP; }
    cudaSetDevice(r->ctx->device);
    uint32_t* dcount = static_cast<uint32_t*>(device_view(count));
    uint32_t* dcell = cap ? static_cast<uint32_t*>(device_view(cell)) : nullptr;
    float* dvalue = cap ? static_cast<float*>(device_view(value)) : nullptr;
    if (!dcount || (cap && (!dcell || !dvalue))) {
        set_error("the cell arrays and the count must be device memory or mapped page-locked host memory");
        return BF_EINVAL;
    }
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
    const cudaError_t e = launch_map_cells(r->map + r->map_off[s], n, r->cell_counts + r->cell_off[s], dcell,
                                           dvalue, cap, dcount, st);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "map cells");
}

bf_status bf_result_copy_mean_max(const bf_result* r, float* out)
{
    if (!r || !out) { set_error("NULL argument"); return BF_EINVAL; }
    cudaSetDevice(r->ctx->device);
    cudaError_t e = cudaMemcpy(out, r->mean_max, r->K * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "result copy");
}

bf_status bf_result_fit_max(const bf_result* r, size_t s, void* stream, bf_skewnorm* out)
{
    if (!r || !out) { set_error("NULL argument"); return BF_EINVAL; }
    if (s != BF_FIT_MEAN && s >= r->n_series) { set_error("bad series index"); return BF_EINVAL; }
    if (r->K == 0) { set_error("no templates to fit"); return BF_EINVAL; }
    bf_ctx* ctx = r->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    const float* v = s == BF_FIT_MEAN ? r->mean_max : r->vmax + s * r->K;
    double* acc = static_cast<double*>(ctx->mem->alloc(16 * sizeof(double)));
    if (!acc) { set_error("out of device memory (fit)"); return BF_ENOMEM; }
    double host[7];
    cudaError_t e = launch_skewnorm_fit(v, r->K, acc, acc + 8, ctx->n_sm, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, acc + 8, sizeof host, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ctx->mem->release(acc);
    if (e != cudaSuccess) return cuda_fail(e, "skew-normal fit");
    out->n = host[0];
    out->mean = host[1];
    out->sd = host[2];
    out->skewness = host[3];
    out->xi = host[4];
    out->omega = host[5];
    out->alpha = host[6];
    return BF_OK;
}

bf_status bf_result_coincidence(const bf_result* r, size_t a, size_t b, double delta_f_hz,
                                uint32_t dt_cells, void* stream, uint32_t* indep_a, uint32_t* indep_b,
                                uint32_t* coinc_a, uint32_t* coinc_b)
{
    if (!r || a >= r->n_series || b >= r->n_series) { set_error("bad series index"); return BF_EINVAL; }
    if (!r->map) { set_error("no maps (opts.want_map)"); return BF_EINVAL; }
    if (!(delta_f_hz >= 0.0)) { set_error("delta_f_hz must be >= 0"); return BF_EINVAL; }
    bf_ctx* ctx = r->ctx;
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    const uint32_t nf = r->map_nf;
    const uint32_t nt = std::min(r->map_nt[a], r->map_nt[b]);
    const double wc = std::floor(delta_f_hz / r->df + 1e-9);
    const uint32_t w = (uint32_t)std::min<double>(wc, (double)nf);
    const uint32_t dt = std::min(dt_cells, nt);
    unsigned int* d = static_cast<unsigned int*>(ctx->mem->alloc(4 * (size_t)nf * sizeof(unsigned int)));
    if (!d) { set_error("out of device memory (coincidence)"); return BF_ENOMEM; }
    std::vector<unsigned int> h(4 * (size_t)nf);
    cudaError_t e = launch_coincidence(r->map + r->map_off[a], r->map + r->map_off[b], nt, nf, w, dt, d,
                                       ctx->n_sm, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, h.size() * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ctx->mem->release(d);
    if (e != cudaSuccess) return cuda_fail(e, "coincidence");
    uint32_t* outs[4] = {indep_a, indep_b, coinc_a, coinc_b};
    for (int q = 0; q < 4; ++q)
        if (outs[q]) std::copy(h.begin() + (size_t)q * nf, h.begin() + (size_t)(q + 1) * nf, outs[q]);
    return BF_OK;
}

bf_status bf_result_get_sigma_pred(const bf_result* r, size_t s, const float** sigma_pred)
{
    if (!r || s >= r->n_series || !sigma_pred) { set_error("bad argument"); return BF_EINVAL; }
    if (!r->sigma_pred) { set_error("no prediction (opts.tail_sigma = BF_SIGMA_PARSEVAL)"); return BF_EINVAL; }
    *sigma_pred = r->sigma_pred + s * r->K;
    return BF_OK;
}

bf_status bf_result_copy_sigma_pred(const bf_result* r, size_t s, float* host)
{
    const float* dev = nullptr;
    bf_status st = bf_result_get_sigma_pred(r, s, &dev);
    if (st) return st;
    if (!host) { set_error("NULL host array"); return BF_EINVAL; }
    cudaSetDevice(r->ctx->device);
    cudaError_t e = cudaMemcpy(host, dev, r->K * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "sigma copy");
}

static size_t kept_tails(const bf_result* r)
{
    uint64_t n = r->n_candidates;
    if (r->cand_count) {
        unsigned int c = 0;
        if (cudaMemcpy(&c, r->cand_count, sizeof c, cudaMemcpyDeviceToHost) == cudaSuccess) n = c;
    }
    return (size_t)std::min<uint64_t>(n, r->cand_cap);
}

bf_status bf_result_tails(const bf_result* r, const bf_tail** tails, size_t* count)
{
    if (!r || !tails || !count) { set_error("NULL argument"); return BF_EINVAL; }
    if (r->cand_cap == 0) { set_error("tails were not requested (opts.want_tails)"); return BF_EINVAL; }
    static_assert(sizeof(bf_tail) == sizeof(Candidate), "tail record layout");
    cudaSetDevice(r->ctx->device);
    *tails = reinterpret_cast<const bf_tail*>(r->cand);
    *count = kept_tails(r);
    return BF_OK;
}

bf_status bf_result_copy_tails(const bf_result* r, bf_tail* host, size_t cap, size_t* count)
{
    const bf_tail* dev = nullptr;
    size_t n = 0;
    bf_status st = bf_result_tails(r, &dev, &n);
    if (st) return st;
    if (count) *count = n;
    if (!host || cap == 0 || n == 0) return BF_OK;
    cudaError_t e = cudaMemcpy(host, dev, std::min(n, cap) * sizeof(bf_tail), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "tail copy");
}

void bf_result_destroy(bf_result* r)
{
    if (!r) return;
    if (r->plan_owned) {            // bf_plan_destroy frees it
        set_error("bf_result_destroy: the result belongs to a plan (freed by bf_plan_destroy)");
        return;
    }
    free_result_buffers(r);
    delete r;
}

bf_status bf_control_randomize(bf_ctx* ctx, const float* in, size_t n, uint64_t seed, float* out)
{
    NvtxRange range("bf_control_randomize");
    if (!ctx || !in || !out) { set_error("NULL argument"); return BF_EINVAL; }
    if (n == 0) return BF_OK;
    if (n >= 0xFFFFFFFFull) { set_error("series of %zu samples too long", n); return BF_EINVAL; }
    const char* a = reinterpret_cast<const char*>(in);
    const char* b = reinterpret_cast<const char*>(out);
    if (a < b + n * 4 && b < a + n * 4) { set_error("in and out overlap"); return BF_EINVAL; }
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    Allocator& mem = *ctx->mem;
    const bool din = is_device_ptr(in), dout = is_device_ptr(out);
    void* scratch = mem.alloc(permute_scratch_bytes(n));
    float* dx = din ? const_cast<float*>(in) : static_cast<float*>(mem.alloc(n * 4));
    float* dy = dout ? out : static_cast<float*>(mem.alloc(n * 4));
    auto cleanup = [&]() {
        mem.release(scratch);
        if (!din) mem.release(dx);
        if (!dout) mem.release(dy);
    };
    if (!scratch || !dx || !dy) {
        cleanup();
        set_error("out of device memory for the control of %zu samples", n);
        return BF_ENOMEM;
    }
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    if (!din) e = cudaMemcpyAsync(dx, in, n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_permute(dx, n, seed, dy, scratch, st);
    if (e == cudaSuccess && !dout) e = cudaMemcpyAsync(out, dy, n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "control randomisation");
}

}  // extern "C"
