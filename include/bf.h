/*
 * bf.h -- C ABI of the GB300 (sm_103a) butterfly-filtering library.
 *
 * Butterfly filtering (van Putten, arXiv:1802.01685, Sect. 2.1) is matched
 * filtering of a time series -- a gravitational-wave strain channel or a
 * binned gamma-ray light curve -- against a large bank of ~1 s ascending and
 * descending chirp templates at every time offset.  Sect. 2.2 adds the
 * time-randomised control and the reduction of the filter output rho to its
 * tails rho > kappa * sigma.  This library computes, on one GPU:
 *
 *   rho_k(tau) = sum_m x[tau+m] h_k[m] / sqrt(sum_m x[tau+m]^2),
 *                tau = 0 .. N-M,  rho := 0 where the window is all zero,
 *
 * for every template k of a bank and every lag tau, without materialising
 * rho, and reduces it to per-template max |rho|, its first argmax and
 * sigma_k = sqrt(mean_tau rho^2), a histogram of the per-template maxima and
 * a time-frequency scatter-max map painted by the tracks f(t) of all (k, tau)
 * with |rho| >= kappa / sqrt(M).
 *
 * Conventions for every call:
 *   - Every call returns a bf_status; none aborts the process.  On failure
 *     bf_last_error() gives a message (thread-local, valid until the next call
 *     on the same thread).
 *   - "device pointer" means memory of the context's CUDA device (cudaMalloc,
 *     torch CUDA tensors, ...); "host pointer" means ordinary or pinned host
 *     memory.  Where a call accepts either, it detects which with
 *     cudaPointerGetAttributes.
 *   - Objects returned through an out-parameter are owned by the library until
 *     the matching *_destroy call.  Input arrays are copied; the caller keeps
 *     ownership and may free them when the call returns.
 *   - Series are float32, finite, uniformly sampled at the rate fs given.
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden symbol visibility; the declarations below
 * are its only exports. */
#if defined(BF_BUILDING_LIBRARY) && defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#define BF_ABI_VERSION 2

typedef enum {
    BF_OK = 0,
    BF_EINVAL = 1,      /* invalid argument                                   */
    BF_ENOMEM = 2,      /* device memory or HBM budget exhausted              */
    BF_ECUDA = 3,       /* a CUDA runtime call failed                          */
    BF_ETIMEDOUT = 4,   /* a wait ran out of time                              */
    BF_EPENDING = 5,    /* serving: the request is still in progress           */
    BF_EAGAIN = 6,      /* serving: the queue is full, retry later             */
    BF_ECANCELED = 7,   /* serving: the request was cancelled                  */
    BF_EDEVICE = 8,     /* a kernel reported an error through its status word  */
    BF_ENOTSUP = 9      /* the requested mode is not available on this device */
} bf_status;

/* chirp track and sense (Sect. 2.1: ascending and descending chirps) */
typedef enum { BF_LINEAR = 0, BF_POWERLAW = 1 } bf_track;
typedef enum {
    BF_ASC = 0,
    BF_DESC = 1,
    BF_BOTH = 2     /* superposition of the ascending chirp and its time reverse
                       (the "butterfly": both tracks at once), unit norm       */
} bf_sense;

/* threshold of the tails rho > kappa sigma (Sect. 2.2) */
typedef enum { BF_SIGMA_WHITE = 0, BF_SIGMA_PARSEVAL = 1 } bf_tail_sigma;

/* arithmetic of the correlation (FP32 accumulate in every mode) */
typedef enum {
    BF_FP32 = 0,        /* FP32 operands, FP32 FMA (SIMT)                      */
    BF_BF16 = 1,        /* BF16 operands on tcgen05 tensor cores               */
    BF_SPLIT_BF16 = 2,  /* x = hi + lo, h = hi + lo in BF16; three tcgen05 MMAs
                           hi*hi + hi*lo + lo*hi into FP32 accumulators, K in
                           chunks of 2048 samples added with rounding to
                           nearest (the tensor core's own accumulation
                           truncates)                                        */
    BF_FFT_FP32 = 3,    /* the paper's route (Sect. 2.2, Fig. 5): FP32 FFTs,
                           overlap-save.  Plain banks: real segments of
                           16384 samples (16385 - M lags each), one template
                           per 8192-point complex transform; quadrature
                           banks: segments of 8192 samples (8193 - M lags),
                           template and partner in one transform.  Template
                           spectra are made from the chirp parameters,
                           whatever the bank stores: a stored bank keeps
                           them (64 KiB per template, 32 KiB per
                           quadrature row; made on first use); a generated
                           bank makes them per call, 512 MiB at a time,
                           overlapped with the correlation, so any bank size
                           works.  Templates of at most 4096 samples, else
                           BF_ENOTSUP.  tile_lags is ignored.  Lags
                           whose window holds less than 1/16384 of its
                           segment's energy (quiet or gated stretches next
                           to loud data), where the transform's rounding
                           would swamp rho, are computed directly.          */
    BF_SPLIT_FP16 = 4   /* as BF_SPLIT_BF16 with FP16 hi and lo parts (K
                           chunks of 1024 samples): the split holds x and h
                           to 2^-22 instead of 2^-17, at the same tensor-core
                           rate; the accumulation bounds both splits alike.  FP16's range is kept
                           by exact power-of-two scaling on the device (each
                           series so that its largest |x| lies in
                           [2^13, 2^14), templates by 2^8), undone in the
                           epilogue.  Needs BF_BANK_SPLIT_FP16 or a
                           generated bank.                                   */
} bf_precision;

/* which sample layouts a bank keeps in device memory (bit flags) */
enum {
    BF_BANK_FP32 = 1,          /* needed by BF_FP32                            */
    BF_BANK_SPLIT_BF16 = 2,    /* needed by BF_BF16 and BF_SPLIT_BF16          */
    BF_BANK_GENERATED = 4,     /* keep only the chirp parameters: every
                                  bf_correlate synthesises the templates it
                                  needs on the fly, chunk by chunk, into a
                                  small ring that stays in L2 while the
                                  correlation consumes it.  Exclusive of the
                                  other layout flags; serves every precision. */
    BF_BANK_SPLIT_FP16 = 16,   /* needed by BF_SPLIT_FP16: the tensor-core
                                  layout with FP16 hi and lo parts of 2^8 h    */
    BF_BANK_QUADRATURE = 8     /* with any of the above: every chirp also gets
                                  its quadrature partner, the Hilbert
                                  transform of the template (sin(2 pi c(t))
                                  in place of the cosine, time-reversed parts
                                  negated: descending -g_s[M-1-m], both
                                  senses g_s[m] - g_s[M-1-m]), at unit norm.
                                  The output of chirp k is then the phase-blind
                                  sqrt(rho_cos^2 + rho_sin^2) >= 0 (max, argmax,
                                  sigma = its rms, tails, maps), the white-
                                  noise tail threshold kappa sqrt(2/M), and a
                                  Parseval sigma the root of the pair's summed
                                  squares.  Every precision.  A quadrature
                                  output counts as two correlations.           */
};

/*
 * One chirp template (Sect. 2.1).  The template is T seconds long
 * (M = round(T * fs) samples); the sweep occupies D = sweep_s seconds
 * (M_D = round(D * fs) samples, 0 < M_D <= M) centred in the window, starting
 * at m_s = floor((M - M_D) / 2), with local time t = (m - m_s) / fs:
 *   linear:    f(t) = f_lo + (f_hi - f_lo) t / D
 *   power law: f(t) = f_lo (1 - t/t_c)^(-3/8), t_c = D / (1 - (f_lo/f_hi)^(8/3))
 *   g[m] = sin^2(pi (m - m_s + 1/2) / M_D) cos(2 pi integral_0^t f),
 *   descending templates are the time reverse g[M-1-m] of the ascending one,
 *   BF_BOTH templates are g[m] + g[M-1-m],
 *   h = g / |g|_2.
 * Requires 0 < f_lo < f_hi < fs / 2.
 */
typedef struct {
    int32_t track;      /* bf_track  */
    int32_t sense;      /* bf_sense  */
    double f_lo;        /* Hz */
    double f_hi;        /* Hz */
    double sweep_s;     /* D, seconds, 0 < D <= T */
} bf_chirp;

/*
 * Rectangular grid of chirps (bank sizes of Sect. 2.1-2.2: 0.5 M to 8.64 M):
 *   f_lo_i  = f_min + (f_max - f_min) i / I,          i = 0..I-1
 *   f_hi_ij = f_lo_i + (f_max - f_lo_i) (j + 1) / J,  j = 0..J-1
 * template index k = ((((a * n_senses + b) * n_durations + d) * I + i) * J + j)
 * for tracks[a], senses[b], durations[d].
 */
typedef struct {
    const int32_t* tracks;   size_t n_tracks;
    const int32_t* senses;   size_t n_senses;
    const double* durations; size_t n_durations;
    double f_min, f_max;     /* Hz */
    size_t I, J;
} bf_chirp_grid;

/* Context configuration.  The paper has no counterpart: its platform
 * (Sect. 2.2, twelve GPUs under OpenCL) managed devices in its own runtime;
 * these are this library's per-GPU resource limits. */
typedef struct {
    int32_t device;          /* CUDA device ordinal                             */
    size_t hbm_budget;       /* bytes the context may hold; 0 = 90 % of free    */
    size_t max_candidates;   /* capacity of the tail list per call; 0 = 2^22    */
    int32_t serve_slots;     /* requests served concurrently; 0 = 8             */
    int32_t serve_queue;     /* requests waiting for a slot; 0 = 1024           */
    int32_t log_level;       /* 0 silent .. 3 verbose                           */
    int32_t serve_policy;    /* bf_serve_policy; 0 = BF_SERVE_FAIR              */
} bf_config;

/* How the serving loop shares the GPU (no counterpart in the paper).
 * BF_SERVE_FAIR: requests are admitted in arrival order and every iteration
 * splits its work budget evenly over the active requests (processor
 * sharing).  BF_SERVE_SHORTEST: the queued request with the least work
 * (lags x templates) is admitted first, and every iteration gives its budget
 * to the active requests with the least remaining work first, each active
 * request still getting at least one template tile (FFT route: one template
 * per SM) so that none stalls.  Results do not depend on the policy. */
typedef enum { BF_SERVE_FAIR = 0, BF_SERVE_SHORTEST = 1 } bf_serve_policy;

typedef struct bf_ctx bf_ctx;
typedef struct bf_bank bf_bank;
typedef struct bf_result bf_result;

/* Fills *cfg with the defaults above. */
void bf_config_default(bf_config* cfg);

/* Creates a context on cfg->device (cfg may be NULL for defaults).  The
 * paper has no counterpart: a context is this library's handle on one GPU.
 * It owns two streams, a caching device allocator bounded by hbm_budget, a
 * device status word through which kernels report timed-out waits and, once
 * serving is used, a scheduler thread.  It also does the set-up of
 * bf_control_randomize_static on its device.  *out receives the context.
 * BF_EINVAL for a device ordinal out of range; BF_ENOTSUP if the device is not
 * compute capability 10.3; BF_ECUDA if CUDA fails. */
bf_status bf_init(const bf_config* cfg, bf_ctx** out);
/* Waits for the context's work, stops its serving thread (pending requests
 * are dropped) and frees everything it owns.  Banks, results and plans made
 * in the context must be destroyed first.  NULL is ignored. */
void bf_destroy(bf_ctx* ctx);

/*
 * Template bank (Sect. 2.1).  Synthesises K templates of T seconds at rate fs
 * on the device: phase in FP64 cycles reduced mod 1, cosine in FP32, taper,
 * FP64 unit norm.  `storage` is a mask of BF_BANK_* layouts to keep.
 * params: host array of K chirps, copied.  BF_EINVAL on a chirp violating the
 * rules of bf_chirp or K == 0; BF_ENOMEM when the layouts exceed the budget.
 */
#define BF_MAX_TEMPLATE_LEN 32768   /* M = round(T * fs) samples, at most */
bf_status bf_bank_create(bf_ctx* ctx, const bf_chirp* params, size_t K, double fs,
                         double T, unsigned storage, bf_bank** out);
bf_status bf_bank_create_grid(bf_ctx* ctx, const bf_chirp_grid* grid, double fs,
                              double T, unsigned storage, bf_bank** out);
/* Frees the bank's device memory (after the context's pending work on it);
 * NULL is ignored.  Requests and plans that use the bank must be done. */
void bf_bank_destroy(bf_bank* bank);
/* Shape of the bank (Sect. 2.1: a bank of templates of ~1 s); 0 for NULL. */
size_t bf_bank_size(const bf_bank* bank);           /* K */
size_t bf_bank_template_len(const bf_bank* bank);   /* M */
size_t bf_bank_rows(const bf_bank* bank);   /* template rows: K, or 2K with BF_BANK_QUADRATURE */
/* Copies templates [k0, k0+n) as float32 (row-major [n][M]) to host memory;
 * for a quadrature bank each chirp gives two rows, template then partner
 * ([2n][M]).  Reads the FP32 layout if kept, else hi + lo of the split
 * layout, else synthesises the rows. */
bf_status bf_bank_read(const bf_bank* bank, size_t k0, size_t n, float* host_out);
/* Copies the chirp parameters of templates [k0, k0+n) to host memory. */
bf_status bf_bank_params(const bf_bank* bank, size_t k0, size_t n, bf_chirp* host_out);

typedef struct {
    int32_t precision;       /* bf_precision                                    */
    size_t bank_begin;       /* templates [bank_begin, bank_end); end 0 = all   */
    size_t bank_end;
    double kappa;            /* tails |rho| >= kappa / sqrt(M) paint the map;
                                <= 0 means 5                                    */
    double map_dt_s;         /* map cell: seconds (0 = 1e-3)                    */
    double map_df_hz;        /* map cell: Hz (0 = 4)                            */
    int32_t want_map;        /* paint the time-frequency map                    */
    int32_t want_hist;       /* histogram of per-template maxima                */
    uint32_t hist_bins;      /* 0 = 1024, uniform on [0, 1]                     */
    void* stream;            /* cudaStream_t; NULL = synchronous on the context
                                stream.  Otherwise the call returns once the
                                work is enqueued and the result is valid after
                                the stream has reached that point.             */
    float* rho_out;          /* optional device pointer; with one series, the
                                full filter output rho[k - bank_begin][tau]
                                (n_templates x L floats, row-major) is written
                                here as well.  For inspection of small cases. */
    int32_t want_tails;      /* keep the list of tails (see bf_result_tails)   */
    int32_t tail_sigma;      /* threshold of the tails (map, tail list):
                                BF_SIGMA_WHITE: kappa / sqrt(M), the exact
                                sigma of rho on white noise;
                                BF_SIGMA_PARSEVAL: kappa * sigma_k, with
                                sigma_k predicted per series and template from
                                Parseval's theorem before the search (see
                                bf_result_get_sigma_pred)                      */
    int32_t tile_lags;       /* lags per tensor-core tile: 512 (one TMEM
                                accumulator) or 256 (two, so the epilogue of
                                one tile overlaps the MMAs of the next); 0 =
                                chosen by the library's autotuner, which times
                                both once per precision and template length
                                per context.  Ignored by BF_FP32.            */
} bf_opts;

/* Fills *opts with the defaults: BF_SPLIT_BF16, the whole bank, kappa 5,
 * 1 ms x 4 Hz map cells, 1024 histogram bins, histogram on, no map, no
 * tails, synchronous, white-noise sigma, autotuned tiles. */
void bf_opts_default(bf_opts* opts);

/*
 * Searches n_series series against templates [bank_begin, bank_end) of bank
 * in one batched launch (Sect. 2.1-2.2).  series[s] (host or device pointer)
 * holds lengths[s] >= M samples at rate fs == the bank's rate.  The result
 * holds, per series, per template: max |rho| (float), its first argmax
 * (int32, smallest lag on ties), sigma; the histogram and map when asked;
 * and over all series the per-template mean of the maxima.
 * Samples must be finite.  The window energies come from a running sum of
 * x^2, so one NaN or infinity leaves rho undefined at every later lag of its
 * series, not only in the windows that hold it; mark gaps with zeros (an
 * all-zero window gives rho = 0).  The series preparation flags a series
 * whose FP64 total of x^2 is not finite in the result's status word: a
 * synchronous call (opts->stream NULL) reads it after the search and then
 * returns BF_EINVAL with no result; after a call on a stream, or a plan run
 * on a stream, bf_result_check reads it once the stream has synchronised; a
 * served request fails with BF_EINVAL.
 * BF_EINVAL on a bad length, rate, range, a precision whose layout the bank
 * lacks, or a non-finite sample; BF_EDEVICE if a kernel reported an internal
 * timeout.
 */
bf_status bf_correlate(bf_ctx* ctx, const bf_bank* bank, const float* const* series,
                       const size_t* lengths, size_t n_series, double fs,
                       const bf_opts* opts, bf_result** out);

/* Summary of one search.  correlations counts one template at one lag, the
 * unit of the paper's throughput figure (Sect. 2.2: correlations per second);
 * the rest has no counterpart in the paper. */
typedef struct {
    size_t n_series;
    size_t n_templates;            /* bank_end - bank_begin                     */
    size_t template_len;           /* M                                         */
    double correlations;           /* sum over series of lags x templates       */
    double useful_flops;           /* 2 M x correlations                        */
    uint64_t n_candidates;         /* (k, tau) with |rho| >= threshold          */
    int32_t candidates_overflow;   /* 1 if more than max_candidates: map partial */
    float threshold;               /* kappa / sqrt(M)                           */
    uint32_t hist_bins;
    double kernel_ms;              /* correlation kernel time (synchronous calls) */
    int32_t tile_lags;             /* lags per tile of the kernel that ran      */
} bf_result_info;

/* Status of a result whose work has completed (for calls and plan runs on a
 * caller's stream, after that stream has synchronised; the paper has no
 * counterpart): BF_EINVAL if a series held a NaN or infinite sample (its
 * outputs are then undefined), BF_EDEVICE if a kernel of the context reported
 * a timed-out wait (the context's status word is then cleared), BF_OK
 * otherwise.  Reads device memory synchronously. */
bf_status bf_result_check(const bf_result* r);
/* Copies the summary to *info.  BF_EINVAL for NULL arguments. */
bf_status bf_result_info_get(const bf_result* r, bf_result_info* info);
/* Time-frequency map of series s (Sect. 2.1: chirp-based spectrograms that
 * show trajectories f(t) of finite slope): nt = ceil(N_s / (fs dt)) time
 * cells (rows) by nf = ceil((fs / 2) / df) frequency cells, row-major; cell
 * (b, c) covers times [b dt, (b+1) dt) and frequencies [c df, (c+1) df).
 * BF_EINVAL for a bad series index. */
bf_status bf_result_map_shape(const bf_result* r, size_t s, size_t* nt, size_t* nf);
/* Device pointers into the result for series s, valid until the result is
 * destroyed (a plan's result: until the plan runs again); BF_EINVAL for a bad
 * index or an output the call did not make.
 *   get_max:  per template, max |rho| (float), its first argmax (int32) and
 *             sigma (float) -- the maxima of the butterfly output whose
 *             distributions Fig. 2 compares for data and control;
 *   get_hist: histogram of those maxima (hist_bins uint32 counts on [0, 1],
 *             Fig. 2);
 *   get_map:  the time-frequency map (bf_result_map_shape);
 *   get_mean_max: per template, the mean over the call's series of max |rho|
 *             (Fig. 1: a spectrum averaged over 42 light curves). */
bf_status bf_result_get_max(const bf_result* r, size_t s, const float** vmax,
                            const int32_t** argmax, const float** sigma);
bf_status bf_result_get_hist(const bf_result* r, size_t s, const uint32_t** hist);
bf_status bf_result_get_map(const bf_result* r, size_t s, const float** map);
bf_status bf_result_get_mean_max(const bf_result* r, const float** mean_max);
/* Copies series s's outputs (those of bf_result_get_max, _hist and _map) to
 * host arrays, synchronously; NULL arrays are skipped.  Sizes: n_templates
 * for vmax/argmax/sigma, hist_bins, map_nt * map_nf.  The paper ships only
 * reduced output from the GPU (Sect. 2.2); these are this library's reduced
 * outputs.  BF_EINVAL for a bad index or an array asked for an output the
 * call did not make. */
bf_status bf_result_copy_to_host(const bf_result* r, size_t s, float* vmax,
                                 int32_t* argmax, float* sigma, uint32_t* hist,
                                 float* map);
/* The same copies, enqueued on `stream` (a cudaStream_t; NULL: the legacy
 * default stream) without waiting for them.  They are done when the stream is; until
 * then `r` must not be destroyed (a plan's result: the plan must not run
 * again) and the host arrays must stay allocated.
 * Host arrays should be page-locked (cudaHostAlloc or cudaHostRegister), else
 * the copies may run synchronously.  Errors: as bf_result_copy_to_host, for
 * the enqueueing only; a failed copy shows on the stream. */
bf_status bf_result_copy_to_host_async(const bf_result* r, size_t s, float* vmax,
                                       int32_t* argmax, float* sigma, uint32_t* hist,
                                       float* map, void* stream);
/* The painted (nonzero) cells of series s's time-frequency map (see
 * bf_result_map_shape), in increasing cell index b nf + c, enqueued on
 * `stream` (NULL: the legacy default stream) without waiting: cell[i] and
 * value[i] for i < min(*count, cap), and *count = the number of painted
 * cells, which may exceed cap (then call again with a larger cap).  The map
 * of a search is sparse (Sect. 2.1: the tails rho > kappa sigma painted along
 * the chirps' tracks), so this moves a few kilobytes where the dense map is
 * map_nt * map_nf floats.  cell, value and count must be device memory or
 * page-locked host memory mapped into the device's address space
 * (cudaHostAlloc / cudaMallocHost under unified addressing, or
 * cudaHostRegister with cudaHostRegisterMapped): the kernels write them
 * directly.  The outputs are done when the stream is; until then `r` must not
 * be destroyed (a plan's result: the plan must not run again), and only one
 * such call per series of a result may be in flight.  Errors: BF_EINVAL for
 * NULL arguments (cell and value may be NULL when cap = 0), a bad index, a
 * result without maps, or arrays the device cannot address; BF_ENOTSUP for a
 * map of more than 2^32 cells. */
bf_status bf_result_copy_map_cells_async(const bf_result* r, size_t s, uint32_t* cell, float* value,
                                         size_t cap, uint32_t* count, void* stream);
/* Copies the per-template mean of the maxima (n_templates floats, Fig. 1)
 * to host memory, synchronously. */
bf_status bf_result_copy_mean_max(const bf_result* r, float* host_mean_max);

/* Skew-normal fit of the per-template maxima (Sect. 1, Fig. 2: the
 * distributions of maxima of the filter output, for the data and for the
 * time-randomised control, are left-truncated skewed Gaussians whose
 * difference is the statistic).  The fit is the method of moments of
 * Azzalini (1985) on the population (1/n) moments, computed in FP64 on the
 * device; the skewness is clipped to the skew-normal's range |g| < 0.99527
 * and the truncation is not modelled.  Density of the fit:
 *   f(v) = 2/omega phi((v - xi)/omega) Phi(alpha (v - xi)/omega). */
typedef struct bf_skewnorm {
    double n;                /* number of maxima fitted                          */
    double mean, sd;         /* sample mean and standard deviation (1/n)         */
    double skewness;         /* sample skewness, after clipping                  */
    double xi, omega, alpha; /* location, scale, shape                           */
} bf_skewnorm;

#define BF_FIT_MEAN ((size_t)-1)

/* Fits the maxima of series s, or with s = BF_FIT_MEAN the mean over series
 * (bf_result_get_mean_max).  Runs on `stream` (NULL: the context stream),
 * after whatever the caller enqueued there, and synchronises it before
 * writing *out.  BF_EINVAL for a bad index or a NULL argument. */
bf_status bf_result_fit_max(const bf_result* r, size_t s, void* stream, bf_skewnorm* out);

/* Pseudo-spectra of tails of two detectors (Fig. 6: counts of rho > kappa
 * sigma against frequency, for H1 and L1 independently and simultaneously,
 * with frequency pairs within delta f = 50 Hz).  Series a and b of a result
 * made with want_map are the two detectors over the same time block.  A map
 * cell (t, c) is occupied when a tail of that series painted it (the tail
 * threshold of opts.kappa and opts.tail_sigma).  For each frequency cell
 * c = 0 .. map_nf - 1 (frequencies [c df, (c+1) df)):
 *   indep_a[c] = number of time cells t with (t, c) occupied in a;
 *   coinc_a[c] = number of those with an occupied cell (t', c') of b,
 *                |t' - t| <= dt_cells and |c' - c| <= floor(delta_f_hz / df);
 * and indep_b, coinc_b with a and b exchanged.  The maps are compared over
 * their common time cells.  Averages over blocks are sums over calls divided
 * by their number.  Host arrays of map_nf entries each (NULL to skip); runs
 * on `stream` (NULL: the context stream) and synchronises it.  BF_EINVAL
 * without maps, for a bad index or delta_f_hz < 0. */
bf_status bf_result_coincidence(const bf_result* r, size_t a, size_t b, double delta_f_hz,
                                uint32_t dt_cells, void* stream, uint32_t* indep_a,
                                uint32_t* indep_b, uint32_t* coinc_a, uint32_t* coinc_b);

/*
 * Predicted noise level of rho (Sect. 2.2 and Fig. 5 caption: sigma from
 * Parseval's theorem in a predictor step, before the search), kept when
 * opts.tail_sigma == BF_SIGMA_PARSEVAL:
 *   sigma_k^2 = sum_f P_x(f) |H_k(f)|^2 / (F^2 M sigma_x^2),   F = 16384,
 * the sum over all F bins, P_x the periodogram of the series averaged over
 * rectangular F-sample segments at hop F/2 (a series shorter than F: one
 * zero-padded segment scaled by F/N), H_k the F-point DFT of template k,
 * sigma_x^2 the mean of x^2.  Its expectation on white noise is 1/M.  F is
 * the FFT route's real segment length: the predictor runs on the library's
 * own transforms, in plans and serving too, and takes templates of at most
 * 8192 samples (BF_ENOTSUP otherwise).  n_templates floats per series.
 */
bf_status bf_result_get_sigma_pred(const bf_result* r, size_t s, const float** sigma_pred);
bf_status bf_result_copy_sigma_pred(const bf_result* r, size_t s, float* host);

/*
 * Tails of the filter output (Sect. 2.2: only the tails rho > kappa sigma are
 * handed on from the GPU): every (series, k, tau) with |rho| >= the call's
 * threshold kappa / sqrt(M), with its signed rho.  Kept when opts.want_tails
 * or opts.want_map is set, up to bf_config.max_candidates entries per call
 * (bf_result_info.candidates_overflow tells when more were found); the order
 * is unspecified.  bf_result_tails gives the device array; copy_tails copies
 * at most cap entries to host memory and reports the count kept.
 */
typedef struct {
    uint32_t series;   /* index into the call's series                       */
    uint32_t k;        /* absolute template index in the bank                */
    uint32_t tau;      /* lag                                                */
    float rho;         /* normalised correlation                             */
} bf_tail;
bf_status bf_result_tails(const bf_result* r, const bf_tail** tails, size_t* count);
bf_status bf_result_copy_tails(const bf_result* r, bf_tail* host, size_t cap, size_t* count);
/* Frees a result; NULL is ignored; a plan's result is refused (it belongs to
 * the plan; bf_last_error says so). */
void bf_result_destroy(bf_result* r);

/*
 * Search plans: a fixed search shape replayed as one CUDA graph.  The paper
 * has no counterpart; plans serve its workloads of many series searched
 * against one bank (Sect. 2.1: 42 light curves; Fig. 6: 288 blocks of data),
 * where per-call set-up would otherwise repeat for every block.
 * bf_plan_create fixes the bank, the template range, the number and lengths of
 * the series, the rate and the options (opts.stream and opts.rho_out are
 * ignored), allocates every buffer once and captures the device work of one
 * search -- clearing the outputs, series preparation, the batched correlation,
 * finalize, histogram and map -- into a CUDA graph.  bf_plan_run copies new
 * series (host or device pointers, the lengths given at creation) into the
 * plan and launches the graph on `stream` (NULL: synchronously on the
 * context stream).  *out points at the plan's result: valid until the next run
 * or bf_plan_destroy, read with the bf_result_* calls, never destroyed by the
 * caller (bf_result_destroy on it does nothing but set bf_last_error).
 * A generated bank's synthesis ring (template chunks, or their spectra,
 * made on the context's second stream) is captured in the graph too.  Runs
 * of one plan must
 * not overlap on the GPU, nor a run with asynchronous copies of the previous
 * run's result.
 */
typedef struct bf_plan bf_plan;
bf_status bf_plan_create(bf_ctx* ctx, const bf_bank* bank, const size_t* lengths,
                         size_t n_series, double fs, const bf_opts* opts, bf_plan** out);
bf_status bf_plan_run(bf_plan* plan, const float* const* series, void* stream,
                      const bf_result** out);
void bf_plan_destroy(bf_plan* plan);

/*
 * Time-randomised control (Sect. 2.2 and Fig. 2: maximal-entropy data with
 * the same sample histogram).  out[j] = in[pi(j)] with pi the argsort of the
 * pairs (splitmix64(seed XOR i), i), i = 0..n-1; splitmix64 is the published
 * generator (one step from state z: z += 0x9E3779B97F4A7C15, two
 * xor-shift-multiply rounds, final xor-shift).  `in` and `out` are host or
 * device pointers of n floats and must not overlap.  Deterministic for
 * (n, seed).  Synchronous.
 */
bf_status bf_control_randomize(bf_ctx* ctx, const float* in, size_t n, uint64_t seed,
                               float* out);

/*
 * Time-randomised control that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory where they need the control -- code inside a framework whose
 * allocator owns all device memory, pipelines with a device-memory plan fixed
 * up front (cudaMalloc can also stall them on an implicit synchronisation),
 * callers under a hard memory cap.  It needs no context.
 *   in, out  device pointers (current device) of n floats, not overlapping;
 *   n        1 .. BF_STATIC_CONTROL_MAX (larger n: BF_EINVAL);
 *   stream   cudaStream_t to enqueue on, NULL for the default stream.  The call
 *            returns once the work is enqueued; out is valid when the stream
 *            reaches it.
 * Output equals bf_control_randomize(ctx, in, n, seed, out).  The sort scratch
 * is a fixed array in the library's device code (6 MiB, held on every GPU
 * that loads it until the process exits); it is shared by every call and
 * keeps the last call's contents (nothing in it needs clearing), so calls
 * whose work overlaps on the GPU, e.g. on two streams, race.
 * Set-up: CUDA loads a library's device code lazily by default, so the first
 * call on a device -- or bf_init on that device, which does the same set-up --
 * loads the array and the permutation kernels into device memory and looks up
 * the array's device address (cudaGetSymbolAddress).  That first call may
 * allocate through the CUDA driver: make it (n = 1 is enough), or create a
 * context on the device, before the point where nothing may be allocated, and
 * outside any stream capture.  Later calls allocate nothing.  After a
 * cudaDeviceReset the next call on that device is a first call again.
 */
#define BF_STATIC_CONTROL_MAX 524288
bf_status bf_control_randomize_static(const float* in, size_t n, uint64_t seed, float* out,
                                      void* stream);

/*
 * Serving with continuous batching.  The paper has no counterpart: it runs
 * one campaign at a time (Sect. 2.2); serving lets searches of different
 * lengths and bank slices share one GPU.  submit copies the series and returns a
 * ticket without waiting for GPU work; a scheduler thread admits requests
 * while slots and HBM budget allow, and each launch of the batched kernel
 * mixes template tiles of every admitted request, so a request that arrives
 * while others run joins the next launch.  A request on a generated bank
 * gets a synthesis slot of its own (about 50 MB of template tiles, or 128 MiB
 * of template spectra on the FFT route, counted against the budget), refilled
 * every iteration with what that iteration correlates.  BF_EAGAIN: queue
 * full.  BF_ENOMEM: the request alone exceeds the budget.  BF_EINVAL: bad
 * request.
 */
typedef struct {
    const float* series;     /* host or device, n samples                        */
    size_t n;
    double fs;
    const bf_bank* bank;     /* must stay alive until the request completes      */
    bf_opts opts;            /* opts.stream is ignored                           */
} bf_request;

bf_status bf_serve_submit(bf_ctx* ctx, const bf_request* req, uint64_t* ticket);
/* Waits up to timeout_us (< 0: forever, 0: no wait).  BF_OK hands over the
 * result (caller destroys it); BF_EPENDING / BF_ETIMEDOUT if not done;
 * BF_ECANCELED if cancelled; BF_EINVAL for an unknown ticket. */
bf_status bf_serve_poll(bf_ctx* ctx, uint64_t ticket, int64_t timeout_us,
                        bf_result** out);
/* Asks for the request to stop; its next poll returns BF_ECANCELED (or its
 * result, if it finished first).  BF_EINVAL for an unknown ticket. */
bf_status bf_serve_cancel(bf_ctx* ctx, uint64_t ticket);

/* Counters of the serving loop since the context was made (no counterpart in
 * the paper). */
typedef struct {
    uint64_t submitted, completed, cancelled, rejected;
    uint64_t queued, active;
    double p50_ms, p99_ms;         /* submit -> completion latency              */
    double correlations_per_s;     /* completed lag-correlations / busy time    */
    uint64_t launches;             /* batched kernel launches so far            */
    size_t hbm_in_use;
} bf_serve_stats;

bf_status bf_serve_stats_get(bf_ctx* ctx, bf_serve_stats* out);

/* Diagnostics (no counterpart in the paper): the calling thread's last error
 * message, the text of a status, and BF_ABI_VERSION of the built library. */
const char* bf_last_error(void);
const char* bf_status_string(bf_status s);
int bf_abi_version(void);

/* Self-test of the bounded waits that guard the tensor-core kernel's
 * pipeline (every mbarrier wait gives up after a time limit, records a code
 * in the context's device status word and lets the kernel drain and return,
 * so that no wait can hang the GPU).  Runs the same wait on an mbarrier that
 * receives its one arrival when `signal` is nonzero and never otherwise, with
 * a limit of limit_us microseconds (at most 1,000,000), synchronously on the
 * context stream.  Returns BF_OK when the arrival came, BF_EDEVICE when the
 * wait ran out (the status word is then cleared and the context stays
 * usable), BF_EINVAL for a limit out of range.  *waited_us (if not NULL) gets
 * the time the wait took. */
bf_status bf_selftest_wait(bf_ctx* ctx, int signal, uint32_t limit_us, double* waited_us);
/* Number of kernels this library has launched in the process so far (all
 * contexts); a diagnostic for benchmarks.  The paper has no counterpart. */
uint64_t bf_kernel_launches(void);

/* Measured FMA rates of device `device` (a diagnostic for the rooflines of
 * the ALU-bound kernels; the paper has no counterpart): FP32 and FP64 FMA
 * loops of independent chains filling every SM, timed with CUDA events, best
 * of three launches of about 40 ms each.  Writes TFLOP/s (two flops per FMA)
 * to the non-NULL outputs.  Allocates a small output buffer and a stream for
 * the duration of the call and restores the current device.  BF_EINVAL if
 * both outputs are NULL; BF_ECUDA on a CUDA error. */
bf_status bf_probe_alu_peaks(int device, double* fp32_tflops, double* fp64_tflops);

#if defined(BF_BUILDING_LIBRARY) && defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* BF_H */
