// Serving with continuous batching.
//
// Requests (one series against a slice of a bank) are submitted from any
// thread.  One scheduler thread per context admits queued requests while a
// slot is free and the HBM budget holds their series and result buffers,
// uploads and prepares each admitted series once, and then drives the device
// in iterations: every iteration launches the batched correlation kernel over
// a chunk of template tiles from EVERY admitted request (one segment per
// request), so a request arriving while others run joins the next iteration
// instead of waiting for them to finish.  When a request's last chunk has been
// launched its finalize kernels follow on the same stream; its completion
// event then releases the slot and its memory.  Requests of different
// precisions go to separate launches of the matching kernel.  A request on
// the FFT route makes its segment spectra at admission and then takes a
// chunk of template pairs per iteration, in a launch of its own (the FFT
// kernel walks one template range for all the series it is given).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>

#include "runtime.h"

namespace bfi {

namespace {

using clk = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum RState { R_QUEUED, R_ACTIVE, R_DONE, R_CANCELED, R_FAILED };

struct Request {
    uint64_t ticket = 0;
    std::vector<float> host;        // copy of the series
    double fs = 0;
    const bf_bank* bank = nullptr;
    bf_opts opts{};
    RState state = R_QUEUED;
    bf_status status = BF_OK;
    std::string error;
    // set by bf_serve_cancel (under the serving mutex) and by the scheduler on
    // a failed launch; read by the scheduler without the mutex
    std::atomic<bool> cancel{false};
    bf_result* result = nullptr;
    PreparedSeries prep;
    uint32_t tt_next = 0, tt_end = 0;   // template-tile cursor
    uint32_t n_lag_tiles = 0;
    bool finalized = false;
    cudaEvent_t done = nullptr;
    size_t bytes = 0;
    double t_submit = 0, t_done = 0;
    double correlations = 0;
    // the FFT route
    bool fft = false;
    FftParams fp{};                 // this request's series and outputs
    float2* seg_spec = nullptr;     // its segment spectra
    uint32_t* fix = nullptr;        // lags for the direct fixup [2 L], then their count
    uint32_t k_next = 0, k_stop = 0;   // template-row cursor
    // a generated bank: this request's synthesis slot, refilled every
    // iteration (before that iteration's launch, on the same stream) with the
    // template tiles it correlates -- or, on the FFT route, their spectra
    // (gslot[0]) made through the synthesised rows in gscratch
    void* gslot[2] = {nullptr, nullptr};
    float* gscratch = nullptr;
    uint32_t gcap_rows = 0, gscratch_rows = 0;
    // BF_SERVE_SHORTEST: the request's size (lags x template rows) and its
    // share of the current iteration (work units: tile pairs or transforms)
    double work = 0;
    uint64_t share = 0;
};

// tiles per SM per iteration: large enough to amortise the launch, small
// enough that new arrivals join within a few milliseconds
constexpr uint64_t TILES_PER_SM = 8;
// FFT-route transforms per SM per iteration (about as long as the tiles above)
constexpr uint64_t TRANSFORMS_PER_SM = 100;
// a generated bank's slot per request: template rows of one iteration on the
// direct routes, and 128 MiB of template spectra on the FFT route
constexpr uint32_t GEN_SERVE_ROWS = 3072;
constexpr size_t GEN_SERVE_SPEC_BYTES = size_t(128) << 20;
constexpr uint32_t GEN_SERVE_SYNTH_ROWS = 2048;

uint32_t gen_fft_rows(const bf_bank* bank)
{
    return (uint32_t)(GEN_SERVE_SPEC_BYTES / (fft_spec_bins(bank->quad) * sizeof(float2))) & ~1u;
}

// device bytes of a request's synthesis slot (0 for a stored bank)
size_t gen_serve_bytes(const bf_bank* bank, int precision)
{
    if (!bank->generated) return 0;
    if (precision == BF_FFT_FP32) {
        const size_t rows = gen_fft_rows(bank);
        return (rows + 2) * fft_spec_bins(bank->quad) * sizeof(float2) +
               (size_t)std::min(GEN_SERVE_SYNTH_ROWS, (uint32_t)rows) * FFT_POINTS * sizeof(float);
    }
    return (precision != BF_FP32 ? 2 : 1) * gen_slot_bytes(bank, precision, GEN_SERVE_ROWS);
}

}  // namespace

struct ServeState {
    bf_ctx* ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::unordered_map<uint64_t, Request*> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool started = false;
    cudaStream_t stream = nullptr;
    // statistics
    uint64_t submitted = 0, completed = 0, cancelled = 0, rejected = 0, launches = 0;
    std::vector<double> latency_ms;
    double corr_done = 0, busy_s = 0, busy_since = -1;

    ~ServeState() = default;
};

static void release_request_device(bf_ctx* ctx, Request* r)
{
    r->prep.release(*ctx->mem);
    if (r->fix) {
        ctx->mem->release(r->fix);
        r->fix = nullptr;
    }
    if (r->seg_spec) {
        ctx->mem->release(r->seg_spec);
        r->seg_spec = nullptr;
    }
    for (void*& p : r->gslot) {
        ctx->mem->release(p);
        p = nullptr;
    }
    ctx->mem->release(r->gscratch);
    r->gscratch = nullptr;
    if (r->done) {
        cudaEventDestroy(r->done);
        r->done = nullptr;
    }
}

// Admission: allocate the result, upload and prepare the series.
static bool admit(ServeState* S, Request* r)
{
    bf_ctx* ctx = S->ctx;
    const bf_bank* bank = r->bank;
    std::vector<size_t> len{r->host.size()};
    bf_result* res = nullptr;
    bf_status st = alloc_result(ctx, bank, r->opts, len, r->fs, S->stream, &res);
    if (st == BF_OK) {
        st = prepare_series(ctx, r->host.data(), r->host.size(), bank->M, bank->M_pad,
                            r->opts.precision, S->stream, &r->prep, res->status);
        if (st != BF_OK) bf_result_destroy(res);
    }
    if (st != BF_OK) {
        r->status = st;
        r->error = bf_last_error();
        return false;
    }
    if (res->parseval) {
        std::lock_guard<std::mutex> g(ctx->launch_mu);    // the context's twiddle tables
        PredictCall pc;
        st = predict_prepare(ctx, bank, {&r->prep}, r->opts.bank_begin, r->opts.bank_end, res->sigma_pred,
                             res->K, res->scratch, S->stream, &pc);
        if (st == BF_OK) {
            cudaError_t ep = predict_launch(ctx, bank, pc, S->stream);
            if (ep != cudaSuccess) st = cuda_fail(ep, "predictor");
        }
        if (st != BF_OK) {
            r->status = st;
            r->error = bf_last_error();
            r->prep.release(*ctx->mem);
            bf_result_destroy(res);
            return false;
        }
    }
    if (r->opts.precision == BF_FFT_FP32) {
        // template spectra (kept with the bank), then this series' segment spectra
        std::lock_guard<std::mutex> g(ctx->launch_mu);
        const float2* tw = nullptr;
        cudaError_t e = fft_tables(ctx, S->stream, &tw);
        st = e != cudaSuccess     ? cuda_fail(e, "FFT tables")
             : bank->generated ? BF_OK
                               : bank_fft_spectra(ctx, const_cast<bf_bank*>(bank), S->stream);
        if (st == BF_OK && bank->generated) {
            // the spectra slot and the rows it is made through
            r->gcap_rows = gen_fft_rows(bank);
            r->gscratch_rows = std::min(GEN_SERVE_SYNTH_ROWS, r->gcap_rows);
            r->gslot[0] = ctx->mem->alloc((size_t)(r->gcap_rows + 2) * fft_spec_bins(bank->quad) * sizeof(float2));
            r->gscratch = static_cast<float*>(ctx->mem->alloc((size_t)r->gscratch_rows * FFT_POINTS * sizeof(float)));
            if (!r->gslot[0] || !r->gscratch) {
                set_error("out of device memory for the request's template spectra");
                st = BF_ENOMEM;
            }
        }
        const bool quad = bank->quad;
        const uint32_t nseg = fft_segments(r->prep.L, bank->M, quad);
        if (st == BF_OK) {
            r->seg_spec = static_cast<float2*>(ctx->mem->alloc(fft_series_bytes(r->prep.L, bank->M, quad)));
            r->fix = static_cast<uint32_t*>(ctx->mem->alloc((2 * (size_t)r->prep.L + 1) * sizeof(uint32_t)));
            if (!r->seg_spec || !r->fix) {
                set_error("out of device memory for the segment spectra");
                st = BF_ENOMEM;
            }
        }
        if (st == BF_OK) {
            const uint32_t V = fft_lags_per_seg(bank->M, quad);
            FftSeriesBatch b{};
            b.n = 1;
            b.err = ctx->d_err;
            b.quad = quad ? 1 : 0;
            b.F = fft_seg_len(quad);
            b.V = V;
            b.Vp = fft_norm_stride(bank->M, quad);
            b.scale = fft_inverse_scale(quad);
            b.tw = tw;
            b.x[0] = r->prep.x;
            b.N[0] = r->prep.N;
            b.spec[0] = r->seg_spec;
            b.S[0] = r->prep.prefix;
            b.inv[0] = r->prep.inv;
            b.inv_seg[0] = fft_seg_norms(r->seg_spec, nseg, quad);
            b.L[0] = (uint32_t)r->prep.L;
            b.fix[0] = r->fix;
            b.n_fix = r->fix + 2 * r->prep.L;
            e = launch_fft_series(b, nseg, ctx->n_sm, S->stream);
            if (e != cudaSuccess) st = cuda_fail(e, "segment spectra");
            FftParams& p = r->fp;
            p.hspec = bank->fspec;
            p.tw = tw;
            p.k_begin = (uint32_t)bank_row(bank, r->opts.bank_begin);
            p.k_end = (uint32_t)bank_row(bank, r->opts.bank_end);
            p.hrow0 = 0;
            p.quad = bank->quad ? 1 : 0;
            p.V = V;
            p.Vp = b.Vp;
            p.n_ser = 1;
            p.err = ctx->d_err;
            p.thr = res->thr;
            p.cand_cap = res->cand_cap;
            p.cand = res->cand;
            p.cand_count = res->cand_count;
            p.chirps = bank->d_params;
            p.M = bank->M;
            p.fs = bank->fs;
            FftSeries& f = p.ser[0];
            f.spec = r->seg_spec;
            f.inv = b.inv_seg[0];
            f.x = r->prep.x;
            f.fix = r->fix;
            f.n_fix = r->fix + 2 * r->prep.L;
            f.vmax = res->packed;
            f.sumsq = res->sumsq;
            f.sigma_pred = res->parseval ? res->sigma_pred : nullptr;
            f.kappa = res->kappa;
            f.L = r->prep.L;
            f.nseg = nseg;
            r->fft = true;
            r->k_next = p.k_begin;
            r->k_stop = p.k_end;
        }
        if (st != BF_OK) {
            r->status = st;
            r->error = bf_last_error();
            release_request_device(ctx, r);
            bf_result_destroy(res);
            return false;
        }
    }
    if (bank->generated && !r->fft) {
        // the template-tile slot of the direct routes
        const int planes = r->opts.precision != BF_FP32 ? 2 : 1;
        r->gcap_rows = GEN_SERVE_ROWS;
        for (int i = 0; i < planes; ++i) {
            r->gslot[i] = ctx->mem->alloc(gen_slot_bytes(bank, r->opts.precision, GEN_SERVE_ROWS));
            if (!r->gslot[i]) {
                set_error("out of device memory for the request's synthesis slot");
                r->status = BF_ENOMEM;
                r->error = bf_last_error();
                release_request_device(ctx, r);
                bf_result_destroy(res);
                return false;
            }
        }
    }
    r->result = res;
    const uint32_t tile_t = tile_templates(r->opts.precision);
    r->tt_next = (uint32_t)(bank_row(r->bank, r->opts.bank_begin) / tile_t);
    r->tt_end = r->fft ? r->tt_next : (uint32_t)((bank_row(r->bank, r->opts.bank_end) + tile_t - 1) / tile_t);
    r->n_lag_tiles = (r->prep.L + tile_lags(r->opts.precision) - 1) / tile_lags(r->opts.precision);
    r->correlations = (double)r->prep.L * (double)(r->opts.bank_end - r->opts.bank_begin) *
                      (r->bank->quad ? 2.0 : 1.0);
    res->correlations = r->correlations;
    cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
    r->state = R_ACTIVE;
    return true;
}

static void scheduler(ServeState* S)
{
    bf_ctx* ctx = S->ctx;
    cudaSetDevice(ctx->device);
    cudaEvent_t prev = nullptr, cur = nullptr;
    cudaEventCreateWithFlags(&prev, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&cur, cudaEventDisableTiming);
    bool prev_valid = false;

    for (;;) {
        std::vector<Request*> act;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop) break;
            // admission, in arrival order, while a slot and the budget allow
            const bool shortest = ctx->cfg.serve_policy == BF_SERVE_SHORTEST;
            while (!S->queue.empty() && (int)S->active.size() < ctx->cfg.serve_slots) {
                // arrival order, or the least work first (the earliest among equals)
                auto pick = !shortest ? S->queue.begin()
                                      : std::min_element(S->queue.begin(), S->queue.end(),
                                                         [](const Request* a, const Request* b) {
                                                             return a->work < b->work;
                                                         });
                Request* r = *pick;
                if (r->cancel) {
                    S->queue.erase(pick);
                    r->state = R_CANCELED;
                    ++S->cancelled;
                    S->cv_done.notify_all();
                    continue;
                }
                if (!ctx->mem->fits(r->bytes) && !S->active.empty()) break;
                S->queue.erase(pick);
                lk.unlock();
                const bool ok = admit(S, r);
                lk.lock();
                if (!ok) {
                    r->state = R_FAILED;
                    ++S->rejected;
                    S->cv_done.notify_all();
                    continue;
                }
                if (S->busy_since < 0) S->busy_since = now_s();
                S->active.push_back(r);
            }
            act = S->active;
        }

        // one iteration: a chunk of template tiles of every admitted request
        NvtxRange iter_range("serve iteration");
        std::vector<std::pair<Request*, Seg>> segs[5];          // by precision (the FFT route has none)
        std::vector<Request*> finishing;
        uint64_t n_work = 0;
        for (Request* r : act)
            if (!r->cancel && (r->tt_next < r->tt_end || r->k_next < r->k_stop)) ++n_work;
        const uint64_t budget = (uint64_t)ctx->n_sm * TILES_PER_SM;
        const uint64_t t_budget = (uint64_t)ctx->n_sm * TRANSFORMS_PER_SM;
        const bool shortest = ctx->cfg.serve_policy == BF_SERVE_SHORTEST;
        if (shortest) {
            // each budget to the requests with the least remaining work first,
            // every request still getting one template tile / template per SM
            std::vector<std::pair<uint64_t, Request*>> tiles, ffts;
            for (Request* r : act) {
                if (r->cancel) continue;
                if (r->fft && r->k_next < r->k_stop)
                    ffts.emplace_back((uint64_t)(r->k_stop - r->k_next) / (r->fp.quad ? 2 : 1) *
                                          std::max<uint32_t>(1, r->fp.ser[0].nseg), r);
                else if (!r->fft && r->tt_next < r->tt_end)
                    tiles.emplace_back((uint64_t)(r->tt_end - r->tt_next) * std::max<uint32_t>(1, r->n_lag_tiles), r);
            }
            auto by_rest = [](const std::pair<uint64_t, Request*>& a, const std::pair<uint64_t, Request*>& b) {
                return a.first < b.first;
            };
            std::stable_sort(tiles.begin(), tiles.end(), by_rest);
            std::stable_sort(ffts.begin(), ffts.end(), by_rest);
            uint64_t left = budget;
            for (auto& w : tiles) {
                const uint64_t g = std::max<uint64_t>(std::min(w.first, left), w.second->n_lag_tiles);
                left -= std::min(left, g);
                w.second->share = g;
            }
            left = t_budget;
            for (auto& w : ffts) {
                const uint64_t nseg = std::max<uint32_t>(1, w.second->fp.ser[0].nseg);
                const uint64_t g = std::max<uint64_t>(std::min(w.first, left), (uint64_t)ctx->n_sm * nseg);
                left -= std::min(left, g);
                w.second->share = g;
            }
        }
        for (Request* r : act) {
            if (r->cancel || r->tt_next >= r->tt_end) continue;
            uint64_t per = shortest ? r->share : std::max<uint64_t>(1, budget / std::max<uint64_t>(1, n_work));
            uint64_t ntt = std::max<uint64_t>(1, per / std::max<uint32_t>(1, r->n_lag_tiles));
            ntt = std::min<uint64_t>(ntt, r->tt_end - r->tt_next);
            const uint32_t tile_t = tile_templates(r->opts.precision);
            if (r->bank->generated)     // the rows synthesised (from a multiple of 128) fit the slot
                ntt = std::min<uint64_t>(ntt, (r->gcap_rows - (tile_t < TC_TILE_T ? TC_TILE_T : 0)) / tile_t);
            bf_result* res = r->result;
            Seg g = make_segment(r->prep, 0, r->bank, r->opts.bank_begin, r->opts.bank_end,
                                 r->tt_next, (uint32_t)ntt, r->opts.precision, res->packed,
                                 res->sumsq);
            if (r->bank->generated) {
                const size_t k0 = (size_t)r->tt_next * tile_t / TC_TILE_T * TC_TILE_T;
                const size_t k1 = ceil_div((size_t)(r->tt_next + ntt) * tile_t, (size_t)TC_TILE_T) * TC_TILE_T;
                cudaError_t e = gen_synth_rows(r->bank, r->opts.precision, k0, k1, r->gslot[0], r->gslot[1],
                                               S->stream);
                if (e != cudaSuccess) { r->status = cuda_fail(e, "serve synthesis"); r->cancel = true; }
                gen_point_segment(g, r->opts.precision, k0, r->gslot[0], r->gslot[1]);
            }
            if (res->parseval) {
                g.sigma_pred = res->sigma_pred;
                g.kappa = res->kappa;
            }
            segs[r->opts.precision].emplace_back(r, g);
            r->tt_next += (uint32_t)ntt;
            if (r->tt_next >= r->tt_end) finishing.push_back(r);
        }
        // Requests that keep no tails share one launch per precision (no tail is
        // collected there); a request with a map or a tail list owns the
        // candidate buffer its segment writes, so it gets a launch of its own
        // in the same iteration.
        bool any = false;
        for (int prec = 0; prec < 5; ++prec) {
            if (segs[prec].empty()) continue;
            std::vector<Seg> shared;
            std::vector<Request*> shared_owner;
            for (auto& rs : segs[prec]) {
                Request* r = rs.first;
                if (r->result->cand_cap > 0) {
                    std::vector<Seg> one{rs.second};
                    cudaError_t e = launch_segments(ctx, one, prec, r->result->thr, r->result->cand,
                                                    r->result->cand_count, r->result->cand_cap,
                                                    S->stream, nullptr);
                    if (e != cudaSuccess) { r->status = cuda_fail(e, "serve launch"); r->cancel = true; }
                } else {
                    Seg g = rs.second;
                    g.sigma_pred = nullptr;           // no tails in a shared launch
                    shared.push_back(g);
                    shared_owner.push_back(r);
                }
            }
            if (!shared.empty()) {
                bf_result* r0 = shared_owner[0]->result;
                cudaError_t e = launch_segments(ctx, shared, prec, INFINITY, r0->cand, r0->cand_count,
                                                0, S->stream, nullptr);
                if (e != cudaSuccess)
                    for (Request* r : shared_owner) { r->status = cuda_fail(e, "serve launch"); r->cancel = true; }
            }
            any = true;
        }
        // FFT-route requests: a chunk of templates (real route) or template
        // pairs (pair route) each, one transform per item and segment
        for (Request* r : act) {
            if (!r->fft || r->cancel || r->k_next >= r->k_stop) continue;
            const uint64_t per = shortest ? r->share
                                          : std::max<uint64_t>(1, t_budget / std::max<uint64_t>(1, n_work));
            const uint64_t items = std::max<uint64_t>((uint64_t)ctx->n_sm, per / std::max<uint32_t>(1, r->fp.ser[0].nseg));
            const uint64_t want = r->fp.quad ? 2 * items : items;
            uint32_t rows = (uint32_t)std::min<uint64_t>(want, r->k_stop - r->k_next);
            if (r->bank->generated) rows = std::min(rows, r->gcap_rows);         // even, as k_next
            FftParams p = r->fp;
            p.k_lo = r->k_next;
            p.k_hi = r->k_next + rows;
            cudaError_t e = cudaSuccess;
            if (r->bank->generated) {
                // this iteration's template spectra (a pair route's rows start even)
                e = fft_template_spectra(r->bank, r->k_next, rows, r->gscratch, r->gscratch_rows, p.tw,
                                         static_cast<float2*>(r->gslot[0]), ctx->n_sm, S->stream);
                p.hspec = static_cast<const float2*>(r->gslot[0]);
                p.hrow0 = r->k_next;
            }
            if (e == cudaSuccess) e = launch_corr_fft(p, ctx->n_sm, S->stream);
            if (e != cudaSuccess) { r->status = cuda_fail(e, "serve launch"); r->cancel = true; }
            r->k_next += rows;
            if (r->k_next >= r->k_stop) finishing.push_back(r);
            any = true;
        }
        for (Request* r : finishing) {
            if (r->status == BF_OK && finalize_result(ctx, r->bank, r->result, S->stream) != BF_OK)
                r->status = BF_ECUDA;
            cudaEventRecord(r->done, S->stream);
            r->finalized = true;
        }
        if (any) {
            cudaEventRecord(cur, S->stream);
            std::swap(prev, cur);
            // keep at most two iterations in flight: wait for the one before
            if (prev_valid) cudaEventSynchronize(cur);
            prev_valid = true;
            std::lock_guard<std::mutex> g(S->mu);
            ++S->launches;
        }

        // completions and cancellations
        {
            std::vector<Request*> done_now;
            for (Request* r : act) {
                if (r->finalized && cudaEventQuery(r->done) == cudaSuccess) done_now.push_back(r);
                else if (r->cancel && !r->finalized) {
                    cudaStreamSynchronize(S->stream);
                    done_now.push_back(r);
                }
            }
            if (!any && done_now.empty() && !act.empty()) {
                // nothing launched: wait for outstanding work rather than spin
                cudaStreamSynchronize(S->stream);
                continue;
            }
            if (!done_now.empty()) {
                // a kernel that gave up on a wait marks every request it served
                const bf_status dev = check_device_status(ctx);
                std::lock_guard<std::mutex> g(S->mu);
                const double t = now_s();
                for (Request* r : done_now) {
                    S->active.erase(std::find(S->active.begin(), S->active.end(), r));
                    release_request_device(ctx, r);
                    if (r->cancel && r->status == BF_OK) {
                        bf_result_destroy(r->result);
                        r->result = nullptr;
                        r->state = R_CANCELED;
                        ++S->cancelled;
                        continue;
                    }
                    // the candidate count, then the status word (non-finite samples)
                    unsigned int w[2] = {0, 0};
                    if (r->status == BF_OK && dev == BF_OK &&
                        cudaMemcpy(w, r->result->cand_count, sizeof w, cudaMemcpyDeviceToHost) != cudaSuccess)
                        r->status = BF_ECUDA;
                    if (r->status == BF_OK && dev == BF_OK && (w[1] & 1u)) {
                        r->status = BF_EINVAL;
                        r->error = "the request's series holds a non-finite sample (NaN or infinity)";
                    }
                    if (r->status != BF_OK || dev != BF_OK) {
                        bf_result_destroy(r->result);
                        r->result = nullptr;
                        r->state = R_FAILED;
                    } else {
                        r->result->n_candidates = w[0];
                        r->state = R_DONE;
                        r->t_done = t;
                        ++S->completed;
                        S->latency_ms.push_back(1e3 * (t - r->t_submit));
                        S->corr_done += r->correlations;
                    }
                }
                if (S->active.empty() && S->busy_since >= 0) {
                    S->busy_s += t - S->busy_since;
                    S->busy_since = S->queue.empty() ? -1 : t;
                }
                S->cv_done.notify_all();
            }
        }
    }
    cudaStreamSynchronize(S->stream);
    cudaEventDestroy(prev);
    cudaEventDestroy(cur);
}

static bf_status ensure_started(bf_ctx* ctx)
{
    if (!ctx->serve) {
        ctx->serve = new ServeState();
        ctx->serve->ctx = ctx;
    }
    ServeState* S = ctx->serve;
    if (!S->started) {
        cudaSetDevice(ctx->device);
        cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "serve stream");
        S->th = std::thread(scheduler, S);
        S->started = true;
    }
    return BF_OK;
}

void serve_shutdown(bf_ctx* ctx)
{
    if (!ctx->serve) return;
    ServeState* S = ctx->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto& kv : S->all) {
        Request* r = kv.second;
        release_request_device(ctx, r);
        if (r->result) bf_result_destroy(r->result);
        delete r;
    }
    S->all.clear();
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    ctx->serve = nullptr;
}

}  // namespace bfi

using namespace bfi;

extern "C" {

bf_status bf_serve_submit(bf_ctx* ctx, const bf_request* req, uint64_t* ticket)
{
    if (!ctx || !req || !ticket || !req->series || !req->bank) {
        set_error("NULL argument");
        return BF_EINVAL;
    }
    const bf_bank* bank = req->bank;
    if (bank->ctx != ctx) { set_error("bank belongs to another context"); return BF_EINVAL; }
    if (std::fabs(req->fs - bank->fs) > 1e-9 * bank->fs) {
        set_error("request rate %g differs from the bank's %g", req->fs, bank->fs);
        return BF_EINVAL;
    }
    if (req->n < bank->M || req->n > 0xFFFFFFF0ull) {
        set_error("request series of %zu samples; need M=%u <= N", req->n, bank->M);
        return BF_EINVAL;
    }
    bf_opts o;
    bf_status st = resolve_opts(bank, &req->opts, &o);
    if (st) return st;
    o.stream = nullptr;
    std::unique_ptr<Request> r(new Request());
    r->host.resize(req->n);
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaMemcpy(r->host.data(), req->series, req->n * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "copying the request series");
    r->fs = req->fs;
    r->bank = bank;
    r->opts = o;
    r->work = (double)(req->n - bank->M + 1) * (double)(bank_row(bank, o.bank_end) - bank_row(bank, o.bank_begin));
    r->bytes = prepared_series_bytes(req->n, bank->M, bank->M_pad, o.precision) +
               result_bytes(bank, o, req->n, req->fs, ctx->cfg.max_candidates) +
               gen_serve_bytes(bank, o.precision);
    if (r->bytes > ctx->mem->budget()) {
        set_error("request needs %zu bytes, over the budget of %zu", r->bytes, ctx->mem->budget());
        return BF_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> g(ctx->launch_mu);
        st = ensure_started(ctx);
        if (st) return st;
    }
    ServeState* S = ctx->serve;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if ((int)S->queue.size() >= ctx->cfg.serve_queue) {
            set_error("serving queue full (%d)", ctx->cfg.serve_queue);
            return BF_EAGAIN;
        }
        r->ticket = S->next_ticket++;
        r->t_submit = now_s();
        *ticket = r->ticket;
        S->all[r->ticket] = r.get();
        S->queue.push_back(r.release());
        ++S->submitted;
    }
    S->cv_work.notify_all();
    return BF_OK;
}

bf_status bf_serve_poll(bf_ctx* ctx, uint64_t ticket, int64_t timeout_us, bf_result** out)
{
    if (!ctx || !out) { set_error("NULL argument"); return BF_EINVAL; }
    *out = nullptr;
    if (!ctx->serve) { set_error("unknown ticket %llu", (unsigned long long)ticket); return BF_EINVAL; }
    ServeState* S = ctx->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return BF_EINVAL; }
    Request* r = it->second;
    auto finished = [&] { return r->state == R_DONE || r->state == R_CANCELED || r->state == R_FAILED; };
    if (!finished()) {
        if (timeout_us == 0) return BF_EPENDING;
        if (timeout_us < 0) S->cv_done.wait(lk, finished);
        else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished)) {
            set_error("request %llu still running", (unsigned long long)ticket);
            return BF_ETIMEDOUT;
        }
    }
    S->all.erase(it);
    bf_status st = BF_OK;
    if (r->state == R_DONE) {
        *out = r->result;
    } else if (r->state == R_CANCELED) {
        st = BF_ECANCELED;
        set_error("request %llu was cancelled", (unsigned long long)ticket);
    } else {
        st = r->status != BF_OK ? r->status : BF_ECUDA;
        set_error("%s", r->error.empty() ? "request failed" : r->error.c_str());
    }
    delete r;
    return st;
}

bf_status bf_serve_cancel(bf_ctx* ctx, uint64_t ticket)
{
    if (!ctx || !ctx->serve) { set_error("unknown ticket"); return BF_EINVAL; }
    ServeState* S = ctx->serve;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("unknown ticket"); return BF_EINVAL; }
    Request* r = it->second;
    if (r->state == R_QUEUED || r->state == R_ACTIVE) r->cancel = true;
    S->cv_work.notify_all();
    return BF_OK;
}

bf_status bf_serve_stats_get(bf_ctx* ctx, bf_serve_stats* out)
{
    if (!ctx || !out) { set_error("NULL argument"); return BF_EINVAL; }
    memset(out, 0, sizeof *out);
    out->hbm_in_use = ctx->mem->in_use();
    if (!ctx->serve) return BF_OK;
    ServeState* S = ctx->serve;
    std::lock_guard<std::mutex> g(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->cancelled = S->cancelled;
    out->rejected = S->rejected;
    out->queued = S->queue.size();
    out->active = S->active.size();
    out->launches = S->launches;
    if (!S->latency_ms.empty()) {
        std::vector<double> v = S->latency_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            size_t i = (size_t)std::ceil(q * (double)v.size()) - 1;
            return v[std::min(i, v.size() - 1)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    double busy = S->busy_s + (S->busy_since >= 0 ? now_s() - S->busy_since : 0.0);
    out->correlations_per_s = busy > 0 ? S->corr_done / busy : 0.0;
    return BF_OK;
}

}  // extern "C"
