// Search plans: one search shape captured once as a CUDA graph and replayed.
// Every buffer of the search (result, prepared series, scratch) is allocated
// at creation; a run copies the new series in and launches the graph, so a
// repeated search costs one graph launch instead of one launch per kernel and
// memset (six or more per series plus the correlation and finalize kernels).
#include <cmath>
#include <cstring>

#include "runtime.h"

struct bf_plan {
    bf_ctx* ctx = nullptr;
    const bf_bank* bank = nullptr;
    bf_opts o{};
    std::vector<size_t> lengths;
    double fs = 0;
    bf_result* r = nullptr;
    std::vector<bfi::PreparedSeries> prep;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_run = 0;      // kernel nodes in the graph
};

using namespace bfi;

extern "C" {

void bf_plan_destroy(bf_plan* p)
{
    if (!p) return;
    if (p->ctx) {
        cudaSetDevice(p->ctx->device);
        cudaStreamSynchronize(p->ctx->stream);
    }
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto& ps : p->prep) ps.release(*p->ctx->mem);
    if (p->r) {
        p->r->plan_owned = false;
        bf_result_destroy(p->r);
    }
    delete p;
}

bf_status bf_plan_create(bf_ctx* ctx, const bf_bank* bank, const size_t* lengths, size_t n_series,
                         double fs, const bf_opts* opts, bf_plan** out)
{
    NvtxRange range("bf_plan_create");
    if (!ctx || !bank || !lengths || !out || n_series == 0) {
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
    o.stream = nullptr;
    o.rho_out = nullptr;
    for (size_t s = 0; s < n_series; ++s)
        if (lengths[s] < bank->M || lengths[s] > 0xFFFFFFF0ull) {
            set_error("series %zu has %zu samples; need M=%u <= N < 2^32", s, lengths[s], bank->M);
            return BF_EINVAL;
        }
    cudaSetDevice(ctx->device);
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    std::unique_ptr<bf_plan, void (*)(bf_plan*)> p(new bf_plan(), bf_plan_destroy);
    p->ctx = ctx;
    p->bank = bank;
    p->o = o;
    p->lengths.assign(lengths, lengths + n_series);
    p->fs = fs;
    cudaStream_t strm = ctx->stream;
    st = alloc_result(ctx, bank, o, p->lengths, fs, strm, &p->r);
    if (st) return st;
    p->r->plan_owned = true;
    p->prep.resize(n_series);
    std::vector<PreparedSeries*> pptr;
    std::vector<uint32_t> ids;
    for (size_t s = 0; s < n_series; ++s) {
        st = prepare_series_alloc(ctx, lengths[s], bank->M, bank->M_pad, o.precision, &p->prep[s]);
        if (st) return st;
        p->prep[s].status = p->r->status;           // non-finite samples, per run
        pptr.push_back(&p->prep[s]);
        ids.push_back((uint32_t)s);
        p->r->correlations += (double)p->prep[s].L * (double)p->r->K * (bank->quad ? 2.0 : 1.0);
    }
    const bool fft = o.precision == BF_FFT_FP32;
    std::vector<Seg> segs;
    FftCall fc;
    GenRing ring;
    PredictCall pc;
    int lt = 0;
    if (p->r->parseval) {
        // the predictor's buffers and the twiddle tables before the capture
        std::vector<const PreparedSeries*> pp(pptr.begin(), pptr.end());
        st = predict_prepare(ctx, bank, pp, o.bank_begin, o.bank_end, p->r->sigma_pred, p->r->K,
                             p->r->scratch, strm, &pc);
        if (st) return st;
    }
    if (fft) {
        // everything that allocates or synchronises happens before the capture:
        // the bank's spectra (a generated bank: the spectra ring), the twiddle
        // tables, the segment-spectra buffers
        if (!bank->generated) st = bank_fft_spectra(ctx, const_cast<bf_bank*>(bank), strm);
        if (st == BF_OK) st = fft_prepare(ctx, bank, o, p->prep, p->r, strm, &fc);
        if (st) return st;
        cudaError_t es = cudaStreamSynchronize(strm);
        if (es != cudaSuccess) return cuda_fail(es, "plan set-up");
    } else {
        build_segments(pptr, ids, bank, o.bank_begin, o.bank_end, o.precision, p->r->packed,
                       p->r->sumsq, p->r->K, segs);
        if (p->r->parseval)
            for (size_t s = 0; s < segs.size(); ++s) {
                segs[s].sigma_pred = p->r->sigma_pred + s * p->r->K;
                segs[s].kappa = p->r->kappa;
            }
        if (bank->generated) {
            // the synthesis ring, before the capture
            st = gen_prepare(ctx, bank, o, p->r, &ring);
            if (st) return st;
        }
        cudaError_t es = cudaStreamSynchronize(strm);
        if (es == cudaSuccess) es = corr_tc_set_attributes();
        if (es != cudaSuccess) return cuda_fail(es, "plan set-up");
        // the tile shape is fixed before capture (the autotuner times launches;
        // for a generated bank on its first synthesised chunk)
        lt = o.precision == BF_FP32 ? SIMT_TILE_L
             : o.tile_lags          ? o.tile_lags
             : bank->generated      ? gen_autotune(ctx, bank, o, segs, strm, ring)
                                    : choose_lag_tile(ctx, segs[0], o.precision, strm);
        es = cudaStreamSynchronize(strm);
        if (es != cudaSuccess) return cuda_fail(es, "plan set-up");
    }
    p->r->tile_lags = lt;

    // capture one search
    const uint64_t l0 = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(strm, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t ec = clear_result(p->r, strm);
    if (ec == cudaSuccess) {
        const std::vector<const PreparedSeries*> pp(pptr.begin(), pptr.end());
        ec = prepare_series_batch(pp, bank->M, o.precision, strm);
    }
    if (ec == cudaSuccess && p->r->parseval) ec = predict_launch(ctx, bank, pc, strm);
    if (ec == cudaSuccess)
        ec = fft              ? fft_launch(ctx, bank, fc, p->r, strm)
             : bank->generated ? gen_launch(ctx, bank, o, segs, p->r, strm, lt, ring)
                               : launch_segments(ctx, segs, o.precision, p->r->thr, p->r->cand,
                                                 p->r->cand_count, p->r->cand_cap, strm, nullptr, lt);
    bf_status fst = BF_OK;
    if (ec == cudaSuccess) fst = finalize_result(ctx, bank, p->r, strm);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(strm, &graph);
    if (ec != cudaSuccess || fst != BF_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ec != cudaSuccess ? cuda_fail(ec, "plan capture")
                                 : (fst != BF_OK ? fst : cuda_fail(e, "cudaStreamEndCapture"));
    }
    p->graph = graph;
    p->launches_per_run = g_launches.load() - l0;
    g_launches.fetch_sub(p->launches_per_run);      // counted when the graph runs
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    *out = p.release();
    return BF_OK;
}

bf_status bf_plan_run(bf_plan* p, const float* const* series, void* stream, const bf_result** out)
{
    NvtxRange range("bf_plan_run");
    if (!p || !series || !out) { set_error("NULL argument"); return BF_EINVAL; }
    *out = nullptr;
    for (size_t s = 0; s < p->lengths.size(); ++s)
        if (!series[s]) { set_error("series %zu is NULL", s); return BF_EINVAL; }
    bf_ctx* ctx = p->ctx;
    cudaSetDevice(ctx->device);
    const bool sync = stream == nullptr;
    cudaStream_t strm = sync ? ctx->stream : static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    cudaError_t e = cudaSuccess;
    for (size_t s = 0; s < p->lengths.size() && e == cudaSuccess; ++s)
        e = cudaMemcpyAsync(p->prep[s].x, series[s], p->lengths[s] * sizeof(float), cudaMemcpyDefault,
                            strm);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (sync) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, strm);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, strm);
    if (e == cudaSuccess) count_launches(p->launches_per_run);
    if (sync) cudaEventRecord(e1, strm);
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(strm);
    if (sync) {
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        p->r->kernel_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (e != cudaSuccess) return cuda_fail(e, "plan run");
    p->r->n_candidates = 0;
    if (sync) {
        bf_status st = check_device_status(ctx);
        if (st) return st;
        unsigned int c = 0;
        cudaMemcpy(&c, p->r->cand_count, sizeof c, cudaMemcpyDeviceToHost);
        p->r->n_candidates = c;
        st = check_canaries(p->r);              // debug builds
        if (st == BF_OK) st = result_status(p->r);      // non-finite samples
        if (st) return st;
    }
    *out = p->r;
    return BF_OK;
}

}  // extern "C"
