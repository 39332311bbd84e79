/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the butterfly-filtering hot path
 * of van Putten, "GPU-accelerated broadband analysis of multi-messenger light
 * curves of GRBs" (arXiv:1802.01685), Sect. 2.1 "Butterfly filtering" and
 * Sect. 2.2 "GPU acceleration".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load the shared library built from this
 * file.  It shares no code, header, table or constant generator with the CUDA
 * library; the product path never calls it.
 *
 * Every loop below follows the plain definition of the quantity it computes:
 * no blocking, no fusion, no FFT.  OpenMP only distributes independent
 * templates over cores.
 *
 * The paper states the method in words only (matched filtering of a time
 * series against a large bank of ~1 s ascending and descending chirps, Sect.
 * 2.1; time-randomised control, Sect. 2.2 and Fig. 2; tails rho > kappa*sigma,
 * Sect. 2.2 and Fig. 5).  It prints no template formula, normalisation, grid
 * or worked example, so the precise definitions used here are readings of
 * that text; each is stated where it is used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PI 3.14159265358979323846

enum { O_LINEAR = 0, O_POWERLAW = 1 };
enum { O_ASC = 0, O_DESC = 1, O_BOTH = 2 };

/* ------------------------------------------------------------------------ */
/* Chirp tracks (Sect. 2.1: trajectories f(t) of finite slope; ascending and  */
/* descending chirps of about 1 s).                                           */
/*                                                                            */
/* Reading: a template sweeps f_lo -> f_hi over a sweep time D (0 < D <= T)   */
/* along either                                                               */
/*   linear:    f(t) = f_lo + (f_hi - f_lo) t / D                             */
/*   power law: f(t) = f_lo (1 - t/t_c)^(-3/8),                               */
/*              t_c = D / (1 - (f_lo/f_hi)^(8/3)),  so f(D) = f_hi.           */
/* The phase in cycles is the time integral of f from 0.                      */
/* ------------------------------------------------------------------------ */

double oracle_powerlaw_tc(double f_lo, double f_hi, double D)
{
    return D / (1.0 - pow(f_lo / f_hi, 8.0 / 3.0));
}

/* cycles elapsed at local time t since the start of the ascending sweep */
double oracle_cycles(int track, double f_lo, double f_hi, double D, double t)
{
    if (track == O_LINEAR)
        return f_lo * t + (f_hi - f_lo) * t * t / (2.0 * D);
    double tc = oracle_powerlaw_tc(f_lo, f_hi, D);
    return 1.6 * f_lo * tc * (1.0 - pow(1.0 - t / tc, 0.625));
}

/* instantaneous frequency of the ascending track at local time t */
double oracle_freq(int track, double f_lo, double f_hi, double D, double t)
{
    /* the end of the sweep: f(D) = f_hi by the definition of both tracks.
     * Evaluated through the formula it lands within an ulp of f_hi, and
     * where f_hi / df is a whole number the map cell would hang on that ulp. */
    if (t >= D) return f_hi;
    if (track == O_LINEAR)
        return f_lo + (f_hi - f_lo) * t / D;
    double tc = oracle_powerlaw_tc(f_lo, f_hi, D);
    return f_lo * pow(1.0 - t / tc, -0.375);
}

/* support length M_D = round(D * fs) and its start m_s inside the window */
long oracle_support_len(double D, double fs) { return (long)floor(D * fs + 0.5); }
long oracle_support_start(long M, long MD) { return (M - MD) / 2; }

/* first sample of the support of a template with the given sense: the
 * descending template is the time reverse of the ascending one, so its
 * support is mirrored inside the window. */
long oracle_support_first(int sense, long M, long MD)
{
    long ms = oracle_support_start(M, MD);
    return sense == O_ASC ? ms : M - ms - MD;
}

/* Returns 0 when the parameters describe a valid template, else -1. */
int oracle_check_chirp(int track, int sense, double f_lo, double f_hi, double D,
                       double fs, long M)
{
    if (track != O_LINEAR && track != O_POWERLAW) return -1;
    if (sense != O_ASC && sense != O_DESC && sense != O_BOTH) return -1;
    if (!(fs > 0.0) || M <= 0) return -1;
    if (!(f_lo > 0.0) || !(f_hi > f_lo) || !(f_hi < 0.5 * fs)) return -1;
    if (!(D > 0.0)) return -1;
    long MD = oracle_support_len(D, fs);
    if (MD < 2 || MD > M) return -1;
    return 0;
}

/*
 * One template h[0..M-1] (Sect. 2.1, "templates ... superpositions of
 * ascending and descending chirps of intermediate duration").  Reading:
 *   j = m - m_s in [0, M_D), t = j / fs,
 *   g[m] = sin^2(pi (j + 1/2) / M_D) * cos(2 pi c(t)),  zero off the support,
 *   descending: g[M - 1 - m] (the time reverse),
 *   both ("butterfly"): g[m] + g[M - 1 - m], the superposition of the two,
 *   h = the chosen g / sqrt(sum g^2)   (unit L2 norm).
 * The quadrature partner (phase = 1) is the Hilbert transform of the
 * template, for the phase-insensitive output sqrt(rho_cos^2 + rho_sin^2):
 * g_s takes sin(2 pi c(t)) in place of the cosine, and a time-reversed part
 * enters with a minus sign (reversal negates the Hilbert transform), so
 *   ascending g_s[m], descending -g_s[M - 1 - m],
 *   both g_s[m] - g_s[M - 1 - m],
 * each at unit norm.
 */
int oracle_template_phase(int track, int sense, double f_lo, double f_hi, double D,
                          double fs, long M, int phase, double *h)
{
    if (oracle_check_chirp(track, sense, f_lo, f_hi, D, fs, M)) return -1;
    long MD = oracle_support_len(D, fs);
    long ms = oracle_support_start(M, MD);
    for (long m = 0; m < M; ++m) h[m] = 0.0;
    for (long j = 0; j < MD; ++j) {
        double t = (double)j / fs;
        double s = sin(O_PI * ((double)j + 0.5) / (double)MD);
        double c = oracle_cycles(track, f_lo, f_hi, D, t);
        h[ms + j] = s * s * (phase ? sin(2.0 * O_PI * c) : cos(2.0 * O_PI * c));
    }
    if (sense == O_BOTH) {
        for (long a = 0, b = M - 1; a <= b; ++a, --b) {
            if (phase) {
                double d = h[a] - h[b];
                h[a] = d;
                h[b] = -d;
            } else {
                double s = h[a] + h[b];
                h[a] = s;
                h[b] = s;
            }
        }
    }
    double e = 0.0;
    for (long m = 0; m < M; ++m) e += h[m] * h[m];
    double inv = 1.0 / sqrt(e);
    for (long m = 0; m < M; ++m) h[m] *= inv;
    if (sense == O_DESC) {       /* reversal keeps the norm: reverse last */
        for (long a = 0, b = M - 1; a < b; ++a, --b) {
            double tmp = h[a];
            h[a] = h[b];
            h[b] = tmp;
        }
        if (phase)
            for (long m = 0; m < M; ++m) h[m] = -h[m];
    }
    return 0;
}

int oracle_template(int track, int sense, double f_lo, double f_hi, double D,
                    double fs, long M, double *h)
{
    return oracle_template_phase(track, sense, f_lo, f_hi, D, fs, M, 0, h);
}

/*
 * Rectangular bank grid (reading; the paper gives bank sizes only: 8.64 M,
 * 4 M, 8 M and 0.5 M templates, Sect. 2.1-2.2 and Fig. 6).
 *   f_lo_i  = f_min + (f_max - f_min) i / I,            i = 0..I-1
 *   f_hi_ij = f_lo_i + (f_max - f_lo_i) (j + 1) / J,    j = 0..J-1
 *   k = ((((a * n_senses + b) * n_dur + d) * I + i) * J + j)
 * for track list index a, sense list index b and duration index d.
 * Returns the number of templates written.
 */
long oracle_grid(const int *tracks, long n_tracks, const int *senses, long n_senses,
                 const double *durs, long n_dur, double f_min, double f_max,
                 long I, long J, int *track, int *sense, double *f_lo,
                 double *f_hi, double *D)
{
    long k = 0;
    for (long a = 0; a < n_tracks; ++a)
        for (long b = 0; b < n_senses; ++b)
            for (long d = 0; d < n_dur; ++d)
                for (long i = 0; i < I; ++i)
                    for (long j = 0; j < J; ++j) {
                        double lo = f_min + (f_max - f_min) * (double)i / (double)I;
                        double hi = lo + (f_max - lo) * (double)(j + 1) / (double)J;
                        track[k] = tracks[a];
                        sense[k] = senses[b];
                        f_lo[k] = lo;
                        f_hi[k] = hi;
                        D[k] = durs[d];
                        ++k;
                    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Normalised correlation (Sect. 2.1 "matched filtering"; normalisation by   */
/* the local window norm).  Reading:                                          */
/*   num(tau)  = sum_m x[tau+m] h[m]                                          */
/*   E(tau)    = sum_m x[tau+m]^2                                             */
/*   rho(tau)  = num(tau) / sqrt(E(tau)),  rho := 0 where E(tau) == 0,        */
/* for tau = 0 .. N-M.                                                        */
/* ------------------------------------------------------------------------ */

/* numerator and window energy of one template at every lag */
void oracle_correlate_raw(const float *x, long N, const double *h, long M,
                          double *num, double *energy)
{
    long L = N - M + 1;
    for (long tau = 0; tau < L; ++tau) {
        double s = 0.0, e = 0.0;
        for (long m = 0; m < M; ++m) {
            double v = (double)x[tau + m];
            s += v * h[m];
            e += v * v;
        }
        num[tau] = s;
        energy[tau] = e;
    }
}

/*
 * Full search of one series against K templates given by their chirp
 * parameters.  The tail threshold is thr for every template, or thr_k[k]
 * when thr_k is not NULL.  Outputs (any pointer may be NULL):
 *   rho[k*L + tau]   normalised correlation,
 *   vmax[k]          max over tau of |rho|           (Fig. 2: maxima of
 *                                                      butterfly output),
 *   argmax[k]        smallest tau attaining vmax[k],
 *   sigma[k]         sqrt(mean over tau of rho^2)    (standard deviation of
 *                                                      the filter output,
 *                                                      Sect. 2.2),
 *   map[b*nf + f]    time-frequency map: every (k, tau) with |rho| >= thr
 *                    (the tails rho > kappa sigma of Sect. 2.2, here with
 *                    thr = kappa / sqrt(M)) paints the template's track f(t)
 *                    onto cells of dt seconds x df Hz by maximum (chirp-based
 *                    spectrogram, Sect. 2.1).  Must be zeroed by the caller.
 * Returns 0, or -1 for invalid input.
 */
static void paint_one(double *map, long nt, long nf, double dt, double df,
                      int track, int sense, double f_lo, double f_hi, double D,
                      double fs, long M, long tau, double a)
{
    long MD = oracle_support_len(D, fs);
    long first = oracle_support_first(sense, M, MD);
    double t0 = (double)(tau + first) / fs;
    double t1 = (double)(tau + first + MD) / fs;
    long b_lo = (long)floor(t0 / dt - 0.5);
    long b_hi = (long)ceil(t1 / dt);
    if (b_lo < 0) b_lo = 0;
    for (long b = b_lo; b <= b_hi && b < nt; ++b) {
        double tb = ((double)b + 0.5) * dt;
        if (!(tb >= t0 && tb < t1)) continue;
        double t = tb - t0;
        /* descending templates run the ascending track backwards in time;
         * the argument is clamped to the sweep [0, D]. */
        double u = (sense == O_ASC) ? t : D - t;
        if (u < 0.0) u = 0.0;
        if (u > D) u = D;
        double f = oracle_freq(track, f_lo, f_hi, D, u);
        long fb = (long)floor(f / df);
        if (fb < 0 || fb >= nf) continue;
        double *cell = map + b * nf + fb;
        if (a > *cell) *cell = a;
    }
}

/* a superposed ("butterfly") template paints both of its tracks */
static void paint_track(double *map, long nt, long nf, double dt, double df,
                        int track, int sense, double f_lo, double f_hi, double D,
                        double fs, long M, long tau, double a)
{
    if (sense == O_BOTH) {
        paint_one(map, nt, nf, dt, df, track, O_ASC, f_lo, f_hi, D, fs, M, tau, a);
        paint_one(map, nt, nf, dt, df, track, O_DESC, f_lo, f_hi, D, fs, M, tau, a);
    } else {
        paint_one(map, nt, nf, dt, df, track, sense, f_lo, f_hi, D, fs, M, tau, a);
    }
}

int oracle_search(const float *x, long N, double fs, const int *track,
                  const int *sense, const double *f_lo, const double *f_hi,
                  const double *D, long K, long M, int quad, double thr, const double *thr_k,
                  double dt, double df, long nt, long nf, double *rho, double *vmax,
                  long *argmax, double *sigma, double *map)
{
    if (N < M || M <= 0 || K < 0) return -1;
    for (long k = 0; k < K; ++k)
        if (oracle_check_chirp(track[k], sense[k], f_lo[k], f_hi[k], D[k], fs, M))
            return -1;
    long L = N - M + 1;

    /* window energies, shared by all templates (lags are independent) */
    double *energy = (double *)malloc(sizeof(double) * (size_t)L);
    if (!energy) return -1;
#pragma omp parallel for schedule(static)
    for (long tau = 0; tau < L; ++tau) {
        double e = 0.0;
        for (long m = 0; m < M; ++m) e += (double)x[tau + m] * (double)x[tau + m];
        energy[tau] = e;
    }

    int failed = 0;
#pragma omp parallel
    {
        double *h = (double *)malloc(sizeof(double) * (size_t)M);
        double *hs = (double *)malloc(sizeof(double) * (size_t)M);
        if (!h || !hs) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (long k = 0; k < K; ++k) {
            if (!h || !hs) continue;
            oracle_template_phase(track[k], sense[k], f_lo[k], f_hi[k], D[k], fs, M, 0, h);
            if (quad)
                oracle_template_phase(track[k], sense[k], f_lo[k], f_hi[k], D[k], fs, M, 1, hs);
            double best = -1.0, ss = 0.0;
            long best_tau = 0;
            const double thr_here = thr_k ? thr_k[k] : thr;   /* per-template tails */
            for (long tau = 0; tau < L; ++tau) {
                double s = 0.0;
                for (long m = 0; m < M; ++m) s += (double)x[tau + m] * h[m];
                double r = energy[tau] > 0.0 ? s / sqrt(energy[tau]) : 0.0;
                if (quad) {
                    /* quadrature: the magnitude of (rho_cos, rho_sin) */
                    double q = 0.0;
                    for (long m = 0; m < M; ++m) q += (double)x[tau + m] * hs[m];
                    double rs = energy[tau] > 0.0 ? q / sqrt(energy[tau]) : 0.0;
                    r = sqrt(r * r + rs * rs);
                }
                if (rho) rho[k * L + tau] = r;
                double a = fabs(r);
                if (a > best) {   /* strict: the smallest lag wins ties */
                    best = a;
                    best_tau = tau;
                }
                ss += r * r;
                if (map && a >= thr_here) {
#pragma omp critical(oracle_map)
                    paint_track(map, nt, nf, dt, df, track[k], sense[k], f_lo[k],
                                f_hi[k], D[k], fs, M, tau, a);
                }
            }
            if (vmax) vmax[k] = best;
            if (argmax) argmax[k] = best_tau;
            if (sigma) sigma[k] = sqrt(ss / (double)L);
        }
        free(h);
        free(hs);
    }
    free(energy);
    return failed ? -1 : 0;
}

/*
 * Histogram of per-template maxima (Fig. 2: distributions of the maxima of
 * butterfly output for data and control).  Reading: nbins uniform bins on
 * [0, 1]; b = min(floor(nbins * v), nbins - 1).
 */
void oracle_histogram(const double *v, long K, long nbins, uint32_t *counts)
{
    for (long b = 0; b < nbins; ++b) counts[b] = 0;
    for (long k = 0; k < K; ++k) {
        long b = (long)floor((double)nbins * v[k]);
        if (b < 0) b = 0;
        if (b > nbins - 1) b = nbins - 1;
        counts[b] += 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Time-randomised control (Sect. 2.2: time-randomisation gives data of      */
/* maximal entropy and keeps the histogram of samples).  Reading: a seeded   */
/* permutation pi = argsort over i of the pair (splitmix64(seed XOR i), i),   */
/* y[j] = x[pi(j)].  splitmix64 is the published generator of Steele, Lea    */
/* and Flood (OOPSLA 2014), one step from state z.                           */
/* ------------------------------------------------------------------------ */

uint64_t oracle_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    uint64_t key;
    int64_t idx;
} okey;

static int okey_cmp(const void *pa, const void *pb)
{
    const okey *a = (const okey *)pa, *b = (const okey *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

/* writes the permutation pi[0..n-1] */
int oracle_permutation(long n, uint64_t seed, int64_t *pi)
{
    okey *k = (okey *)malloc(sizeof(okey) * (size_t)(n > 0 ? n : 1));
    if (!k) return -1;
    for (long i = 0; i < n; ++i) {
        k[i].key = oracle_splitmix64(seed ^ (uint64_t)i);
        k[i].idx = i;
    }
    qsort(k, (size_t)n, sizeof(okey), okey_cmp);
    for (long j = 0; j < n; ++j) pi[j] = k[j].idx;
    free(k);
    return 0;
}

int oracle_permute(const float *x, long n, uint64_t seed, float *y)
{
    int64_t *pi = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!pi) return -1;
    if (oracle_permutation(n, seed, pi)) {
        free(pi);
        return -1;
    }
    for (long j = 0; j < n; ++j) y[j] = x[pi[j]];
    free(pi);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
