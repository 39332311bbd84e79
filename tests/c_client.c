/*
 * A client of libbf written in plain C against include/bf.h: no Python, host
 * pointers throughout.  It checks closed-form results of the search
 * (Sect. 2.1-2.2 of arXiv:1802.01685):
 *   - a bank template placed, scaled, into an otherwise zero series gives
 *     normalised correlation 1 at its offset (Cauchy-Schwarz equality);
 *   - the time-randomised control is a permutation of the series;
 *   - the asynchronous result copy gives what the synchronous one gives;
 *   - a served request gives what bf_correlate gives.
 * Exit status: 0 all checks passed, 1 a check failed, 2 a call failed,
 * 77 no GPU (bf_init failed).  Test infrastructure.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "bf.h"

#define CALL(x)                                                                  \
    do {                                                                         \
        bf_status st_ = (x);                                                     \
        if (st_ != BF_OK) {                                                      \
            fprintf(stderr, "%s: %s (%s)\n", #x, bf_status_string(st_),          \
                    bf_last_error());                                            \
            return 2;                                                            \
        }                                                                        \
    } while (0)

static int cmp_float(const void* a, const void* b)
{
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

int main(void)
{
    const double fs = 2048.0;
    const size_t N = 9000, n0 = 3333;
    const size_t K = 6, k_inj = 4;
    bf_config cfg;
    bf_config_default(&cfg);
    bf_ctx* ctx = NULL;
    if (bf_init(&cfg, &ctx) != BF_OK) {
        fprintf(stderr, "no GPU: %s\n", bf_last_error());
        return 77;
    }
    const bf_chirp chirps[6] = {
        {BF_LINEAR, BF_ASC, 50.0, 900.0, 1.0},   {BF_LINEAR, BF_DESC, 300.0, 700.0, 0.5},
        {BF_POWERLAW, BF_ASC, 40.0, 400.0, 1.0}, {BF_POWERLAW, BF_DESC, 60.0, 250.0, 0.8},
        {BF_LINEAR, BF_BOTH, 120.0, 800.0, 0.9}, {BF_POWERLAW, BF_ASC, 20.0, 1000.0, 0.3}};
    bf_bank* bank = NULL;
    CALL(bf_bank_create(ctx, chirps, K, fs, 1.0, BF_BANK_SPLIT_BF16, &bank));
    const size_t M = bf_bank_template_len(bank);

    /* the series: zeros with 2.5 h_k placed at n0 */
    float* h = malloc(M * sizeof(float));
    float* x = calloc(N, sizeof(float));
    CALL(bf_bank_read(bank, k_inj, 1, h));
    for (size_t m = 0; m < M; ++m) x[n0 + m] = 2.5f * h[m];

    bf_opts opts;
    bf_opts_default(&opts);
    opts.precision = BF_SPLIT_BF16;
    const float* series[1] = {x};
    const size_t lengths[1] = {N};
    bf_result* res = NULL;
    CALL(bf_correlate(ctx, bank, series, lengths, 1, fs, &opts, &res));
    float vmax[6], sigma[6];
    int32_t argmax[6];
    CALL(bf_result_copy_to_host(res, 0, vmax, argmax, sigma, NULL, NULL));
    int fail = 0;
    printf("injected template %zu: max %.7f at lag %d\n", k_inj, vmax[k_inj], argmax[k_inj]);
    if (fabsf(vmax[k_inj] - 1.0f) > 2e-5f || argmax[k_inj] != (int32_t)n0) fail = 1;
    for (size_t k = 0; k < K; ++k)
        if (!(vmax[k] <= 1.0f + 2e-5f) || !(vmax[k] >= 0.0f)) fail = 1;

    /* the asynchronous copy on the legacy default stream; the synchronous copy
     * after it runs on that stream too and waits for it */
    float amax[6], asig[6], tmp[6];
    int32_t aarg[6];
    CALL(bf_result_copy_to_host_async(res, 0, amax, aarg, asig, NULL, NULL, NULL));
    CALL(bf_result_copy_to_host(res, 0, tmp, NULL, NULL, NULL, NULL));
    const int async_same = memcmp(amax, vmax, sizeof vmax) == 0 &&
                           memcmp(aarg, argmax, sizeof argmax) == 0 &&
                           memcmp(asig, sigma, sizeof sigma) == 0;
    printf("asynchronous copy equals the synchronous one: %s\n", async_same ? "yes" : "no");
    if (!async_same) fail = 1;

    /* time-randomised control: a permutation of the series */
    float* y = malloc(N * sizeof(float));
    CALL(bf_control_randomize(ctx, x, N, 12345u, y));
    float* xs = malloc(N * sizeof(float));
    memcpy(xs, x, N * sizeof(float));
    qsort(xs, N, sizeof(float), cmp_float);
    qsort(y, N, sizeof(float), cmp_float);
    const int perm_ok = memcmp(xs, y, N * sizeof(float)) == 0;
    printf("control is a permutation: %s\n", perm_ok ? "yes" : "no");
    if (!perm_ok) fail = 1;

    /* the same search as a served request */
    bf_request req;
    memset(&req, 0, sizeof req);
    req.series = x;
    req.n = N;
    req.fs = fs;
    req.bank = bank;
    req.opts = opts;
    uint64_t ticket = 0;
    CALL(bf_serve_submit(ctx, &req, &ticket));
    bf_result* served = NULL;
    CALL(bf_serve_poll(ctx, ticket, 60000000, &served));
    float smax[6], ssig[6];
    int32_t sarg[6];
    CALL(bf_result_copy_to_host(served, 0, smax, sarg, ssig, NULL, NULL));
    const int same = memcmp(smax, vmax, sizeof vmax) == 0 && memcmp(sarg, argmax, sizeof argmax) == 0;
    printf("served result equals the direct call: %s\n", same ? "yes" : "no");
    if (!same) fail = 1;

    bf_result_destroy(served);
    bf_result_destroy(res);
    bf_bank_destroy(bank);
    bf_destroy(ctx);
    free(h);
    free(x);
    free(y);
    free(xs);
    printf("%s\n", fail ? "FAILED" : "OK");
    return fail;
}
