// Correlation by FFT: the paper's own route to the filter output (Sect. 2.2
// and Fig. 5: the output of every template against data segments through
// single-precision FFTs on the GPU, with only the tails rho > kappa sigma
// leaving the device).  Overlap-save with transforms of F = 8192 points:
//
//   segment j of a series covers lags tau0 = j V .. tau0 + V - 1, V = F - M + 1,
//   X_j = DFT_F(x[tau0 .. tau0 + F))             (zero past the series end)
//   H_k = DFT_F(h_k zero-padded to F)
//   c_k[tau0 + t] = (1/F) sum_f X_j[f] conj(H_k[f]) e^{+2 pi i f t / F},  t < V,
//
// which is the circular correlation of the segment with the padded template;
// for t < V no product wraps around, so it equals the direct sum
// sum_m h_k[m] x[tau0 + t + m].  The result is normalised by the window norm
// and reduced exactly like the direct kernels (max |rho| with its first
// argmax, sum rho^2, tails).
//
// GB300 layout of the work:
//  * template spectra (two real templates per complex FFT) are half spectra
//    of 4096 complex values per template, bin 0 carrying the DC and Nyquist
//    terms (both real).  A stored bank keeps them in HBM, made once; a
//    generated bank makes them per call, 16,384 rows at a time, in a two-slot
//    ring on the auxiliary stream;
//  * each segment spectrum is computed once per call; all of them stay in L2
//    and reach shared memory by asynchronous copies (cp.async) issued one
//    segment ahead, together with the segment's window norms;
//  * one CTA of 512 threads owns a pair of templates (a, b) at a time and
//    holds their spectra in registers (8 bins per thread).  For every segment
//    it forms Z = X conj(H_a) + i X conj(H_b) over all F bins (Hermitian
//    symmetry fills the upper half; each thread keeps the half that its
//    first FFT pass reads in registers), runs one inverse complex FFT in
//    shared memory and reads c_a = Re z, c_b = Im z -- two real correlations
//    per transform (or, for a quadrature pair, |z|).  The last radix-2 stage
//    of the FFT is fused into the epilogue, so the filter output never
//    reaches HBM.
//  * The FFT is a Stockham autosort FFT with three radix-16 passes (each
//    thread one 16-point DFT per pass, in registers) and a final radix-2
//    stage; the work array holds complex values with index i stored at
//    i + i/16, so that every pass moves a warp's 64-bit values in the
//    minimum two wavefronts, and every thread addresses it at fixed offsets
//    from one base.  The twiddles of each pass sit in their own table, laid out
//    [r][k] so that a warp reads consecutive entries: 15 x 16 and 15 x 256
//    entries for the second and third passes and 4096 for the last stage,
//    rounded from FP64 once per context and copied into shared memory by
//    every CTA.
//  * The transform's rounding error scales with its whole segment, so lags
//    whose window holds almost none of the segment's energy are taken out of
//    the FFT route (k_fft_flags) and computed directly (k_fft_fixup).
#include "corr_common.cuh"
#include "synth.cuh"
#include "runtime.h"

namespace bfi {

namespace {

constexpr int FN = FFT_POINTS;            // 8192
constexpr int FH = FN / 2;                // 4096 half-spectrum bins (+ Nyquist packed in bin 0)
constexpr int FT = 512;                   // threads per FFT block
constexpr int FBINS = FH / FT;            // 8 bins per thread
constexpr int ZPAD = FN + FN / 16;        // padded complex values of the work array
constexpr int ROW = FT + FT / 16;         // padded distance of elements 512 apart (544)
constexpr int UPPER = FH + FH / 16;       // padded distance of elements 4096 apart (4352)
// twiddle tables e^{+2 pi i n / 8192}: pass 2 [15][16], pass 3 [15][256], last stage [4096]
constexpr int TW2 = 0, TW3 = 15 * 16, TWF = TW3 + 15 * 256, TW_N = TWF + FH;   // 8176 entries
constexpr int INV_MAX = FN;               // window norms staged per segment (V <= 8192)
// shared memory: work array, twiddles, then (correlation only) the staged
// segment spectrum and window norms
constexpr size_t FFT_SMEM = (ZPAD + TW_N) * sizeof(float2);
constexpr size_t CORR_SMEM = FFT_SMEM + FH * sizeof(float2) + INV_MAX * sizeof(float);

__global__ void k_fft_tables(float2* __restrict__ tw)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < TW_N; e += gridDim.x * blockDim.x) {
        int n;                                    // exponent in units of 2 pi / 8192
        if (e < TW3) n = ((e - TW2) / 16 + 1) * ((e - TW2) % 16) * 32;
        else if (e < TWF) n = ((e - TW3) / 256 + 1) * ((e - TW3) % 256) * 2;
        else n = e - TWF;
        double sn, cs;
        sincospi((double)n / 4096.0, &sn, &cs);
        tw[e] = make_float2((float)cs, (float)sn);
    }
}

// Work array z (complex, index i stored at i + i/16), twiddle tables, and the
// staging buffers of the correlation kernel.
struct Smem {
    float2* z;
    const float2* tw;
    float2* x;
    float* inv;
};

__device__ __forceinline__ Smem smem_setup(const float2* __restrict__ tw_global)
{
    extern __shared__ __align__(16) float2 fsm[];
    Smem m{fsm, fsm + ZPAD, fsm + ZPAD + TW_N, reinterpret_cast<float*>(fsm + ZPAD + TW_N + FH)};
    float4* dst = reinterpret_cast<float4*>(fsm + ZPAD);
    const float4* src = reinterpret_cast<const float4*>(tw_global);
    for (int i = threadIdx.x; i < TW_N / 2; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    return m;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// waits until at most N of this thread's most recent groups are in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int SIGN>
__device__ __forceinline__ float2 tw_get(const float2* t, int e)
{
    const float2 w = t[e];
    return make_float2(w.x, SIGN > 0 ? w.y : -w.y);
}

__device__ __forceinline__ void rotate(float& r, float& i, float2 w)
{
    const float a = r * w.x - i * w.y;
    i = r * w.y + i * w.x;
    r = a;
}

// 4-point DFT with kernel e^{SIGN 2 pi i n k / 4}, in place
template <int SIGN>
__device__ __forceinline__ void dft4(float& ar, float& ai, float& br, float& bi, float& cr, float& ci,
                                     float& dr, float& di)
{
    const float t0r = ar + cr, t0i = ai + ci;
    const float t1r = ar - cr, t1i = ai - ci;
    const float t2r = br + dr, t2i = bi + di;
    const float t3r = br - dr, t3i = bi - di;
    const float ur = SIGN > 0 ? -t3i : t3i;       // SIGN * i * (b - d)
    const float ui = SIGN > 0 ? t3r : -t3r;
    ar = t0r + t2r;
    ai = t0i + t2i;
    cr = t0r - t2r;
    ci = t0i - t2i;
    br = t1r + ur;
    bi = t1i + ui;
    dr = t1r - ur;
    di = t1i - ui;
}

// 16-point DFT as 4 x 4 (Cooley-Tukey, n = 4 n1 + n2, k = k1 + 4 k2): DFTs
// over n1, twiddles e^{SIGN 2 pi i n2 k1 / 16}, DFTs over n2.  On return
// position 4 k1 + k2 holds output k1 + 4 k2.
template <int SIGN>
__device__ __forceinline__ void dft16(float (&r)[16], float (&i)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2)
        dft4<SIGN>(r[n2], i[n2], r[4 + n2], i[4 + n2], r[8 + n2], i[8 + n2], r[12 + n2], i[12 + n2]);
    constexpr float C1 = 0.923879532511286756f;   // cos(pi/8)
    constexpr float S1 = 0.382683432365089772f;   // sin(pi/8)
    constexpr float R2 = 0.707106781186547524f;   // cos(pi/4)
    constexpr float S = SIGN > 0 ? 1.f : -1.f;
    // position 4 k1 + n2 gets e^{SIGN 2 pi i (n2 k1) / 16}
    rotate(r[5], i[5], make_float2(C1, S * S1));      // n2 k1 = 1
    rotate(r[9], i[9], make_float2(R2, S * R2));      // 2
    rotate(r[13], i[13], make_float2(S1, S * C1));    // 3
    rotate(r[6], i[6], make_float2(R2, S * R2));      // 2
    rotate(r[10], i[10], make_float2(0.f, S));        // 4
    rotate(r[14], i[14], make_float2(-R2, S * R2));   // 6
    rotate(r[7], i[7], make_float2(S1, S * C1));      // 3
    rotate(r[11], i[11], make_float2(-R2, S * R2));   // 6
    rotate(r[15], i[15], make_float2(-C1, -S * S1));  // 9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
        dft4<SIGN>(r[4 * k1], i[4 * k1], r[4 * k1 + 1], i[4 * k1 + 1], r[4 * k1 + 2], i[4 * k1 + 2],
                   r[4 * k1 + 3], i[4 * k1 + 3]);
}

// One radix-16 Stockham pass over 8192 points with stride NS (1, 16, 256):
// thread j reads in[j + 512 r], twiddles by e^{SIGN 2 pi i r (j mod NS) / (16 NS)},
// takes the 16-point DFT and writes out[(j / NS) 16 NS + j mod NS + q NS].
// Padded addresses (i + i/16) are a per-thread base plus constant offsets.
// The second half of a pass, from the 16 inputs already in registers.
template <int SIGN, int NS>
__device__ __forceinline__ void pass16_from(const Smem& m, float (&vr)[16], float (&vi)[16])
{
    const int j = threadIdx.x;
    if (NS > 1) {
        const int k = j % NS;
        const float2* t = m.tw + (NS == 16 ? TW2 : TW3) + k;
#pragma unroll
        for (int r = 1; r < 16; ++r) rotate(vr[r], vi[r], tw_get<SIGN>(t, (r - 1) * NS));
    }
    dft16<SIGN>(vr, vi);
    int wb;                                       // padded address of output q = 0
    if (NS == 1) wb = 17 * j;
    else if (NS == 16) wb = (j / 16) * 272 + (j % 16);
    else wb = (j / 256) * 4352 + (j % 256) + ((j % 256) >> 4);
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const int q = 4 * (p % 4) + p / 4;
        const int off = NS == 1 ? q : NS == 16 ? 17 * q : 272 * q;
        m.z[wb + off] = make_float2(vr[p], vi[p]);
    }
    __syncthreads();
}

template <int SIGN, int NS>
__device__ __forceinline__ void pass16(const Smem& m)
{
    const int j = threadIdx.x;
    const int rd = j + (j >> 4);
    float vr[16], vi[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const float2 v = m.z[rd + ROW * r];
        vr[r] = v.x;
        vi[r] = v.y;
    }
    __syncthreads();
    pass16_from<SIGN, NS>(m, vr, vi);
}

template <int SIGN>
__device__ __forceinline__ void fft_passes(const Smem& m)
{
    pass16<SIGN, 1>(m);
    pass16<SIGN, 16>(m);
    pass16<SIGN, 256>(m);
}

// The final radix-2 stage for output pair (k, k + 4096), k = tid + 512 i.
template <int SIGN>
__device__ __forceinline__ void fft_final(const Smem& m, int i, float2& lo, float2& hi)
{
    const int k = threadIdx.x + FT * i;
    const int a = threadIdx.x + (threadIdx.x >> 4) + ROW * i;
    const float2 v = m.z[a + UPPER];
    float vr = v.x, vi = v.y;
    rotate(vr, vi, tw_get<SIGN>(m.tw + TWF, k));
    const float2 u = m.z[a];
    lo = make_float2(u.x + vr, u.y + vi);
    hi = make_float2(u.x - vr, u.y - vi);
}

// Z[F - k] = the upper output of the final stage at 4096 - k, 1 <= k < 4096
template <int SIGN>
__device__ __forceinline__ float2 fft_final_mirror(const Smem& m, int k)
{
    const int kk = FH - k;
    const int a = kk + (kk >> 4);
    const float2 v = m.z[a + UPPER];
    float vr = v.x, vi = v.y;
    rotate(vr, vi, tw_get<SIGN>(m.tw + TWF, kk));
    const float2 u = m.z[a];
    return make_float2(u.x - vr, u.y - vi);
}

// Spectra of segments of a batch of series: real input, half spectrum out.
__global__ void __launch_bounds__(FT, 1) k_fft_series(const __grid_constant__ FftSeriesBatch p,
                                                      uint32_t total)
{
    const Smem m = smem_setup(p.tw);
    const int tid = threadIdx.x;
    for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
        int s = 0;
        while (s + 1 < p.n && g >= p.seg_begin[s + 1]) ++s;
        const uint32_t j = g - p.seg_begin[s];
        const float* x = p.x[s];
        const uint64_t N = p.N[s], t0 = (uint64_t)j * p.V;
        for (int n = tid; n < FN; n += FT) m.z[n + (n >> 4)] = make_float2(t0 + n < N ? x[t0 + n] : 0.f, 0.f);
        __syncthreads();
        fft_passes<-1>(m);
        float2* out = p.spec[s] + (size_t)j * FH;
#pragma unroll
        for (int i = 0; i < FBINS; ++i) {
            float2 lo, hi;
            fft_final<-1>(m, i, lo, hi);
            out[tid + FT * i] = (tid == 0 && i == 0) ? make_float2(lo.x, hi.x) : lo;
        }
        __syncthreads();
    }
}

// Spectra of templates (2q, 2q + 1) of a chunk of synthesised rows: one
// complex transform of h_a + i h_b, separated by Hermitian symmetry.
__global__ void __launch_bounds__(FT, 1) k_fft_bank(const float* __restrict__ rows, uint32_t n_rows,
                                                    uint32_t n_pairs, const float2* __restrict__ tw,
                                                    float2* __restrict__ spec)
{
    const Smem m = smem_setup(tw);
    const int tid = threadIdx.x;
    for (uint32_t q = blockIdx.x; q < n_pairs; q += gridDim.x) {
        const uint32_t a = 2 * q, b = a + 1;
        const float* ra = rows + (size_t)a * FN;
        const float* rb = rows + (size_t)b * FN;
        for (int n = tid; n < FN; n += FT) m.z[n + (n >> 4)] = make_float2(ra[n], b < n_rows ? rb[n] : 0.f);
        __syncthreads();
        fft_passes<-1>(m);
        float2* sa = spec + (size_t)a * FH;
        float2* sb = spec + (size_t)b * FH;
#pragma unroll
        for (int i = 0; i < FBINS; ++i) {
            const int k = tid + FT * i;
            float2 zk, zn;
            fft_final<-1>(m, i, zk, zn);           // Z[k], Z[k + 4096]
            if (k == 0) {
                // DC and Nyquist of both real templates: real parts of Z[0], Z[4096]
                sa[0] = make_float2(zk.x, zn.x);
                if (b < n_rows) sb[0] = make_float2(zk.y, zn.y);
            } else {
                const float2 zm = fft_final_mirror<-1>(m, k);      // Z[F - k]
                // H_a = (Z[k] + conj Z[F-k]) / 2,  H_b = (Z[k] - conj Z[F-k]) / 2i
                sa[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                if (b < n_rows) sb[k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void push_tail(const FftParams& p, uint32_t series, uint32_t k, uint32_t tau,
                                          float rho)
{
    unsigned int i = atomicAdd(p.cand_count, 1u);
    if (i < p.cand_cap) p.cand[i] = Candidate{series, k, tau, rho};
}

// running max |rho| with its first lag (lags arrive out of order within a thread)
__device__ __forceinline__ void track_max(float a, uint32_t tau, float& best, uint32_t& arg)
{
    if (a > best || (a == best && tau < arg)) {
        best = a;
        arg = tau;
    }
}

// segment spectrum j of a series into shared memory (16-byte asynchronous copies)
__device__ __forceinline__ void stage_spectrum(const Smem& m, const float2* src)
{
    for (int c = threadIdx.x; c < FH / 2; c += FT) cp_async16(m.x + 2 * c, src + 2 * c);
}

// The correlation.  Each CTA walks its items (template pair, series, segment)
// in order; while the FFT of one segment runs, the spectrum of the next one
// and the window norms of this one arrive in shared memory.
// QUAD (a compile-time copy of p.quad, so that each epilogue gets its own
// register allocation): the pair is a template and its quadrature partner.
template <bool QUAD>
__global__ void __launch_bounds__(FT, 1) k_corr_fft(const __grid_constant__ FftParams p)
{
    const Smem m = smem_setup(p.tw);
    const int tid = threadIdx.x, lane = tid & 31;
    const int rd = tid + (tid >> 4);
    const int rv = (FN - tid) + ((FN - tid) >> 4);        // padded address of Z[F - tid]
    const uint32_t n_pairs = (p.k_hi - p.k_lo + 1) / 2;
    const float scale = 1.f / (float)FN;
    uint32_t pair = blockIdx.x;
    if (pair >= n_pairs || p.n_ser == 0) return;
    int s = 0;
    uint32_t j = 0;
    stage_spectrum(m, p.ser[0].spec);
    cp_async_commit();

    float2 ha[FBINS], hb[FBINS];
    uint32_t ka = 0, kb = 0;
    bool has_b = false;
    float thr_a = 0.f, thr_b = 0.f;
    float best_a = -1.f, best_b = -1.f;
    uint32_t arg_a = 0xFFFFFFFFu, arg_b = 0xFFFFFFFFu;
    // per-thread sums of rho^2 over a series (a few thousand terms of similar
    // size: FP32 is ample); the sums over threads are FP64
    float ss_a = 0.f, ss_b = 0.f;
    bool new_pair = true, new_series = true;

    for (;;) {
        const FftSeries& S = p.ser[s];
        if (new_pair) {
            ka = p.k_lo + 2 * pair;
            kb = ka + 1;
            has_b = kb < p.k_hi;
#pragma unroll
            for (int i = 0; i < FBINS; ++i) {
                const int f = tid + FT * i;
                ha[i] = p.hspec[(size_t)(ka - p.hrow0) * FH + f];
                hb[i] = has_b ? p.hspec[(size_t)(kb - p.hrow0) * FH + f] : make_float2(0.f, 0.f);
            }
        }
        // output indices: one per row, or one per quadrature pair (rows ka, kb)
        const uint32_t la = QUAD ? (ka - p.k_begin) >> 1 : ka - p.k_begin, lb = kb - p.k_begin;
        if (new_series) {
            thr_a = S.sigma_pred ? S.kappa * S.sigma_pred[la] : p.thr;
            thr_b = (!has_b || QUAD) ? INFINITY : (S.sigma_pred ? S.kappa * S.sigma_pred[lb] : p.thr);
            best_a = best_b = -1.f;
            arg_a = arg_b = 0xFFFFFFFFu;
            ss_a = ss_b = 0.f;
        }
        const uint32_t t0 = j * p.V;
        const uint32_t nv = min(p.V, S.L - t0);
        for (uint32_t e = tid; e < nv; e += FT) cp_async4(m.inv + e, S.inv + t0 + e);
        cp_async_commit();
        // the item after this one
        uint32_t np = pair, nj = j + 1;
        int ns = s;
        if (nj >= S.nseg) {
            nj = 0;
            if (++ns >= p.n_ser) {
                ns = 0;
                np = pair + gridDim.x;
            }
        }
        cp_async_wait<1>();                         // this segment's spectrum
        __syncthreads();
        // Z = X conj(H_a) + i X conj(H_b).  The first pass of the FFT reads
        // Z[tid + 512 r]: for r < 8 those are this thread's own bins, kept in
        // registers; for r >= 8 they are Z[F - f] of the mirror thread 512 - tid
        // (thread 0: its own bins and the Nyquist term), exchanged through
        // shared memory.
        float vr[16], vi[16];
#pragma unroll
        for (int i = 0; i < FBINS; ++i) {
            const float2 x = m.x[tid + FT * i];
            if (tid == 0 && i == 0) {
                // DC (x.x) and Nyquist (x.y): real products
                vr[0] = x.x * ha[0].x;
                vi[0] = x.x * hb[0].x;
                m.z[UPPER] = make_float2(x.y * ha[0].y, x.y * hb[0].y);
            } else {
                // Y = X conj(H); Z[f] = Ya + i Yb, Z[F - f] = conj(Ya) + i conj(Yb)
                const float yar = x.x * ha[i].x + x.y * ha[i].y;
                const float yai = x.y * ha[i].x - x.x * ha[i].y;
                const float ybr = x.x * hb[i].x + x.y * hb[i].y;
                const float ybi = x.y * hb[i].x - x.x * hb[i].y;
                vr[i] = yar - ybi;
                vi[i] = yai + ybr;
                m.z[rv - ROW * i] = make_float2(yar + ybi, ybr - yai);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = FBINS; r < 16; ++r) {
            const float2 v = m.z[rd + ROW * r];
            vr[r] = v.x;
            vi[r] = v.y;
        }
        if (np < n_pairs) stage_spectrum(m, p.ser[ns].spec + (size_t)nj * FH);
        cp_async_commit();
        __syncthreads();                            // every exchange read before pass 1 writes
        pass16_from<1, 1>(m, vr, vi);
        pass16<1, 16>(m);
        pass16<1, 256>(m);
        cp_async_wait<1>();                         // this segment's window norms
        __syncthreads();
        float pa = 0.f, pb = 0.f;
#pragma unroll 4          // a full unroll pushes the non-quadrature copy past 128 registers
        for (int i = 0; i < FBINS; ++i) {
            float2 z[2];
            fft_final<1>(m, i, z[0], z[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t t = (uint32_t)(tid + FT * i + FH * h);
                if (QUAD && t < nv) {
                    // quadrature pair: |c_cos + i c_sin| / |window|
                    const uint32_t tau = t0 + t;
                    const float r = sqrtf(z[h].x * z[h].x + z[h].y * z[h].y) * (m.inv[t] * scale);
                    track_max(r, tau, best_a, arg_a);
                    pa = fmaf(r, r, pa);
                    if (r >= thr_a) push_tail(p, S.series_id, ka >> 1, tau, r);
                    if (S.rho) S.rho[(size_t)la * S.L + tau] = r;
                } else if (!QUAD && t < nv) {
                    const uint32_t tau = t0 + t;
                    const float inv = m.inv[t] * scale;
                    const float ra = z[h].x * inv, rb = z[h].y * inv;
                    const float aa = fabsf(ra), ab = fabsf(rb);
                    track_max(aa, tau, best_a, arg_a);
                    track_max(ab, tau, best_b, arg_b);
                    pa = fmaf(ra, ra, pa);
                    pb = fmaf(rb, rb, pb);
                    if (aa >= thr_a || ab >= thr_b) {
                        if (aa >= thr_a) push_tail(p, S.series_id, ka, tau, ra);
                        if (ab >= thr_b) push_tail(p, S.series_id, kb, tau, rb);
                    }
                    if (S.rho) {
                        S.rho[(size_t)la * S.L + tau] = ra;
                        if (has_b) S.rho[(size_t)lb * S.L + tau] = rb;
                    }
                }
            }
        }
        ss_a += pa;
        ss_b += pb;
        if (nj == 0) {
            // last segment of this series: reduce and publish
            unsigned long long key_a = best_a >= 0.f ? pack_max(best_a, arg_a) : 0ull;
            unsigned long long key_b = best_b >= 0.f ? pack_max(best_b, arg_b) : 0ull;
            double da = (double)ss_a, db = (double)ss_b;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long oa = __shfl_xor_sync(0xffffffffu, key_a, o);
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, key_b, o);
                key_a = oa > key_a ? oa : key_a;
                key_b = ob > key_b ? ob : key_b;
                da += __shfl_xor_sync(0xffffffffu, da, o);
                db += __shfl_xor_sync(0xffffffffu, db, o);
            }
            if (lane == 0) {
                atomicMax(S.vmax + la, key_a);
                atomicAdd(S.sumsq + la, da);
                if (has_b && !QUAD) {
                    atomicMax(S.vmax + lb, key_b);
                    atomicAdd(S.sumsq + lb, db);
                }
            }
        }
        __syncthreads();
        if (np >= n_pairs) break;
        new_pair = np != pair;
        new_series = nj == 0;
        pair = np;
        s = ns;
        j = nj;
    }
    cp_async_wait<0>();
}

// Lags whose window holds less than 1/FFT_FIX_RATIO2 of the energy of its
// FFT segment (e.g. a quiet stretch or the tapered edge of a loud chirp next to
// silence): the transform's rounding error scales with the segment, so there it
// would swamp rho.  Their inverse norm is set to 0, so the correlation kernel
// gives them rho = 0 (no tail, nothing to the sum of squares, never above the
// true maximum), and they are listed, with the norm, for k_fft_fixup.  The
// energies come from the FP64 prefix of x^2.  One grid row per series.
__global__ void __launch_bounds__(256) k_fft_flags(const __grid_constant__ FftSeriesBatch b)
{
    const int i = blockIdx.y;
    if (i >= b.n) return;
    const uint64_t L = b.L[i], N = b.N[i];
    const double* S = b.S[i];
    float* inv = b.inv[i];
    const uint32_t lane = threadIdx.x & 31;
    // the loop bound is uniform over a warp, so each warp appends its lanes'
    // lags together, in lag order (the fixup reads them as coalesced runs)
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < L; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = base + threadIdx.x;
        bool flag = false;
        float iv = 0.f;
        if (t < L) {
            iv = inv[t];
            if (iv > 0.f) {                             // empty window: rho = 0 exactly
                const uint64_t a = t / b.V * b.V;       // the segment's first sample
                const uint64_t e = min(a + (uint64_t)FN, N);
                const double E = S[e] - S[a];
                flag = E * (double)iv * (double)iv > FFT_FIX_RATIO2;
            }
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, flag);
        if (mask == 0u) continue;
        uint32_t slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(b.n_fix + i, (uint32_t)__popc(mask));   // each lag once: < L entries
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        if (flag) {
            inv[t] = 0.f;
            const uint32_t slot = slot0 + __popc(mask & ((1u << lane) - 1u));
            b.fix[i][2 * slot] = (uint32_t)t;
            b.fix[i][2 * slot + 1] = __float_as_uint(iv);
        }
    }
}

// The direct computation of the listed lags.  Each CTA takes FIX_ROWS template
// rows of the launch's range (FIX_ROWS / 2 quadrature pairs), synthesises them
// in shared memory as the bank does (FP32 rows at unit norm), and gives each
// lane one listed lag: the lane runs the FP32 dot products of its window with
// every row, four samples at a time (four window loads, one 16-byte broadcast
// per row), so one shared-memory wavefront feeds 32 FMAs of the warp rather
// than one.  The products then feed the same max keys, sums of rho^2, tails and
// dense output (written after the correlation kernel's 0 there) as the
// correlation kernel.  Returns at once when no series has a listed lag.
constexpr int FIX_T = 256;
constexpr int FIX_ROWS = 4;
constexpr size_t FIX_SMEM = (size_t)FIX_ROWS * FH * sizeof(float);      // rows of at most FH samples

template <bool QUAD>
__global__ void __launch_bounds__(FIX_T) k_fft_fixup(const __grid_constant__ FftParams p)
{
    constexpr int NOUT = QUAD ? FIX_ROWS / 2 : FIX_ROWS;
    extern __shared__ __align__(16) float fx_rows[];                     // [FIX_ROWS][M_s]
    __shared__ double red[8];
    __shared__ unsigned long long w_key[FIX_T / 32][NOUT];
    __shared__ double w_ss[FIX_T / 32][NOUT];
    uint32_t total = 0;
    for (int i = 0; i < p.n_ser; ++i) total += *p.ser[i].n_fix;
    if (total == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t M = p.M, M_s = (M + 63u) & ~63u;
    const uint32_t n_groups = (p.k_hi - p.k_lo + FIX_ROWS - 1) / FIX_ROWS;   // a pair never splits
    for (uint32_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
        const uint32_t row0 = p.k_lo + grp * FIX_ROWS;
        const uint32_t nr = min((uint32_t)FIX_ROWS, p.k_hi - row0);
        for (uint32_t r = 0; r < (uint32_t)FIX_ROWS; ++r) {
            float* g = fx_rows + (size_t)r * M_s;
            const float nrm = synth_row(p.chirps, row0 + r, p.quad, r < nr, M, M_s, p.fs, g, red);
            for (uint32_t m = threadIdx.x; m < M_s; m += FIX_T) g[m] *= nrm;
        }
        __syncthreads();
        uint32_t o[NOUT], kt[NOUT];
        bool live[NOUT];
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
            const uint32_t row = row0 + (QUAD ? 2 * j : j);
            live[j] = row < p.k_hi;
            o[j] = QUAD ? (row - p.k_begin) >> 1 : row - p.k_begin;      // output index
            kt[j] = QUAD ? row >> 1 : row;                               // tail index
        }
        for (int i = 0; i < p.n_ser; ++i) {
            const FftSeries& S = p.ser[i];
            const uint32_t n = min(*S.n_fix, S.L);
            if (n == 0) continue;                                        // uniform over the CTA
            float thr[NOUT];
#pragma unroll
            for (int j = 0; j < NOUT; ++j)
                thr[j] = !live[j] ? INFINITY : (S.sigma_pred ? S.kappa * S.sigma_pred[o[j]] : p.thr);
            unsigned long long best[NOUT];
            double ss[NOUT];
#pragma unroll
            for (int j = 0; j < NOUT; ++j) {
                best[j] = 0ull;
                ss[j] = 0.0;
            }
            for (uint32_t f0 = warp * 32u; f0 < n; f0 += FIX_T) {
                const uint32_t f = f0 + lane;
                const bool act = f < n;
                const uint32_t tau = act ? S.fix[2 * f] : 0u;
                const float iv = act ? __uint_as_float(S.fix[2 * f + 1]) : 0.f;   // the window's norm
                const float* xw = S.x + tau;    // padded: reads up to tau + M + 2 stay inside
                float c[FIX_ROWS];
#pragma unroll
                for (int r = 0; r < FIX_ROWS; ++r) c[r] = 0.f;
                for (uint32_t m = 0; m < M; m += 4) {           // rows are zero past M
                    const float x0 = xw[m], x1 = xw[m + 1], x2 = xw[m + 2], x3 = xw[m + 3];
#pragma unroll
                    for (int r = 0; r < FIX_ROWS; ++r) {
                        const float4 gv = *reinterpret_cast<const float4*>(fx_rows + (size_t)r * M_s + m);
                        c[r] = fmaf(x0, gv.x, c[r]);
                        c[r] = fmaf(x1, gv.y, c[r]);
                        c[r] = fmaf(x2, gv.z, c[r]);
                        c[r] = fmaf(x3, gv.w, c[r]);
                    }
                }
                if (!act) continue;
#pragma unroll
                for (int j = 0; j < NOUT; ++j) {
                    if (!live[j]) continue;
                    const float rho = QUAD ? sqrtf(c[2 * j] * c[2 * j] + c[2 * j + 1] * c[2 * j + 1]) * iv
                                           : c[j] * iv;
                    const float a = fabsf(rho);
                    const unsigned long long key = pack_max(a, tau);
                    best[j] = key > best[j] ? key : best[j];
                    ss[j] += (double)rho * (double)rho;
                    if (a >= thr[j]) push_tail(p, S.series_id, kt[j], tau, rho);
                    if (S.rho) S.rho[(size_t)o[j] * S.L + tau] = rho;
                }
            }
#pragma unroll
            for (int j = 0; j < NOUT; ++j) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best[j], off);
                    best[j] = ok > best[j] ? ok : best[j];
                    ss[j] += __shfl_xor_sync(0xffffffffu, ss[j], off);
                }
                if (lane == 0) {
                    w_key[warp][j] = best[j];
                    w_ss[warp][j] = ss[j];
                }
            }
            __syncthreads();
            if (threadIdx.x < NOUT && live[threadIdx.x]) {
                const int j = threadIdx.x;
                unsigned long long kmax = 0ull;
                double tot = 0.0;
                for (int w = 0; w < FIX_T / 32; ++w) {
                    kmax = w_key[w][j] > kmax ? w_key[w][j] : kmax;
                    tot += w_ss[w][j];
                }
                if (kmax != 0ull) {
                    atomicMax(S.vmax + o[j], kmax);
                    atomicAdd(S.sumsq + o[j], tot);
                }
            }
            __syncthreads();
        }
    }
}

cudaError_t fft_attributes()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_corr_fft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_corr_fft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_series, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_bank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_fixup<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FIX_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_fixup<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FIX_SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

}  // namespace

// The context's twiddle tables, built on first use.
cudaError_t fft_tables(bf_ctx* ctx, cudaStream_t st, const float2** out)
{
    if (!ctx->fft_tw) {
        float2* t = nullptr;
        cudaError_t e = cudaMalloc(&t, TW_N * sizeof(float2));
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_fft_tables<<<(TW_N + 255) / 256, 256, 0, st>>>(t);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaFree(t);
            return e;
        }
        ctx->fft_tw = t;
    }
    *out = ctx->fft_tw;
    return fft_attributes();
}

// Half spectra of template rows [row0, row0 + nrows) into out[0 ..] (nrows
// rounded up to even; an odd tail pairs with a zero row whose spectrum is not
// written), through `scratch`, room for `scratch_rows` synthesised rows of F
// samples.  Asynchronous on st.
static cudaError_t template_spectra(const bf_bank* bank, size_t row0, size_t nrows, float* scratch,
                                    size_t scratch_rows, const float2* tw, float2* out, int n_sm,
                                    cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < nrows && e == cudaSuccess; k += scratch_rows) {
        const size_t kc = std::min(scratch_rows, nrows - k);     // rows of this sub-chunk
        const size_t nr = kc + (kc & 1);                          // scratch_rows is even
        e = launch_bank_synth(bank->d_params, (uint32_t)(row0 + k), bank->quad, (uint32_t)kc, (uint32_t)nr,
                              bank->M, FN, bank->fs, scratch, nullptr, nullptr, st);
        if (e == cudaSuccess) {
            const uint32_t pairs = (uint32_t)(nr / 2);
            count_launches(1);
            k_fft_bank<<<std::min<uint32_t>(pairs, (uint32_t)n_sm), FT, FFT_SMEM, st>>>(
                scratch, (uint32_t)kc, pairs, tw, out + k * FH);
            e = cudaGetLastError();
        }
    }
    return e;
}

// Half spectra of every template of the bank, [K rounded up to even][4096]
// complex, computed once and kept with the bank.
bf_status bank_fft_spectra(bf_ctx* ctx, bf_bank* bank, cudaStream_t st)
{
    if (bank->fspec) return BF_OK;
    if (bank->M > FFT_POINTS / 2) {
        set_error("the FFT route takes templates of at most %d samples (this bank: %u)", FFT_POINTS / 2,
                  bank->M);
        return BF_ENOTSUP;
    }
    const float2* tw = nullptr;
    cudaError_t e = fft_tables(ctx, st, &tw);
    if (e != cudaSuccess) return cuda_fail(e, "FFT tables");
    const size_t K2 = bank->rows + (bank->rows & 1);
    Allocator& mem = *ctx->mem;
    float2* spec = static_cast<float2*>(mem.alloc(K2 * FH * sizeof(float2)));
    const size_t chunk = std::min<size_t>(4096, K2);
    float* rows = static_cast<float*>(mem.alloc(chunk * FN * sizeof(float)));
    if (!spec || !rows) {
        mem.release(spec);
        mem.release(rows);
        set_error("out of device memory for the template spectra (%zu MB)", (K2 * FH * 8) >> 20);
        return BF_ENOMEM;
    }
    e = template_spectra(bank, 0, bank->rows, rows, chunk, tw, spec, ctx->n_sm, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    mem.release(rows);
    if (e != cudaSuccess) {
        mem.release(spec);
        return cuda_fail(e, "template spectra");
    }
    bank->fspec = spec;
    return BF_OK;
}

uint32_t fft_segments(uint32_t L, uint32_t M)
{
    const uint64_t V = FFT_POINTS - M + 1;
    return (uint32_t)(((uint64_t)L + V - 1) / V);          // L may be close to 2^32
}

cudaError_t launch_fft_series(const FftSeriesBatch& b, uint32_t total_segments, int n_sm, cudaStream_t st)
{
    if (total_segments == 0) return cudaSuccess;
    count_launches(1);
    k_fft_series<<<std::min<uint32_t>(total_segments, (uint32_t)n_sm), FT, FFT_SMEM, st>>>(b, total_segments);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !b.n_fix) return e;
    // the lags for the direct fixup
    e = cudaMemsetAsync(b.n_fix, 0, (size_t)b.n * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    uint32_t L_max = 0;
    for (int i = 0; i < b.n; ++i) L_max = std::max(L_max, b.L[i]);
    const unsigned bx = (unsigned)std::max<uint32_t>(1, std::min<uint32_t>((L_max + 255) / 256, 1024));
    count_launches(1);
    k_fft_flags<<<dim3(bx, (unsigned)b.n), 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_corr_fft(const FftParams& p, int n_sm, cudaStream_t st)
{
    const uint32_t n_pairs = (p.k_hi - p.k_lo + 1) / 2;
    if (n_pairs == 0 || p.n_ser == 0) return cudaSuccess;
    const unsigned grid = std::min<unsigned>(n_pairs, (unsigned)n_sm);
    count_launches(1);
    if (p.quad) k_corr_fft<true><<<grid, FT, CORR_SMEM, st>>>(p);
    else k_corr_fft<false><<<grid, FT, CORR_SMEM, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !p.chirps) return e;
    // the lags left to the direct computation (none: the CTAs return at once)
    const uint32_t n_groups = (p.k_hi - p.k_lo + FIX_ROWS - 1) / FIX_ROWS;
    if (n_groups == 0) return e;
    const unsigned fgrid = std::min<unsigned>(n_groups, (unsigned)n_sm * 3);
    const size_t smem = (size_t)FIX_ROWS * ((p.M + 63u) & ~63u) * sizeof(float);
    count_launches(1);
    if (p.quad) k_fft_fixup<true><<<fgrid, FIX_T, smem, st>>>(p);
    else k_fft_fixup<false><<<fgrid, FIX_T, smem, st>>>(p);
    return cudaGetLastError();
}

// A bank that keeps only its chirp parameters: the template spectra are made
// chunk by chunk (FFT_CHUNK_ROWS rows, 512 MiB of spectra) into a two-slot
// ring on the auxiliary stream, and chunk c is correlated against every
// series batch on the main stream while chunk c+1 is made.  Events order the
// reuse of a slot after the launches that read it.
constexpr size_t FFT_CHUNK_ROWS = 16384;
constexpr size_t FFT_SYNTH_ROWS = 4096;

cudaError_t fft_correlate_chunked(bf_ctx* ctx, const bf_bank* bank, std::vector<FftParams>& batches,
                                  uint32_t row_begin, uint32_t row_end, std::vector<void*>& keep,
                                  cudaStream_t st)
{
    const size_t n_rows = row_end - row_begin;
    const size_t chunk = std::min(FFT_CHUNK_ROWS, n_rows + (n_rows & 1));
    const size_t n_chunks = (n_rows + chunk - 1) / chunk;
    Allocator& mem = *ctx->mem;
    float2* slot[2] = {nullptr, nullptr};
    // the ring outlives this call's launches: the result releases it
    const size_t synth_rows = std::min(FFT_SYNTH_ROWS, chunk);           // both even
    float* scratch = static_cast<float*>(mem.alloc(synth_rows * FN * sizeof(float)));
    keep.push_back(scratch);
    for (int i = 0; i < 2 && i < (int)n_chunks; ++i) {
        slot[i] = static_cast<float2*>(mem.alloc((chunk + 2) * FH * sizeof(float2)));
        keep.push_back(slot[i]);
    }
    if (!scratch || !slot[0] || (n_chunks > 1 && !slot[1])) {
        set_error("out of device memory for the template-spectra ring");
        return cudaErrorMemoryAllocation;
    }
    const float2* tw = batches.empty() ? nullptr : batches[0].tw;
    cudaEvent_t ev_start, made[2], used[2];
    cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
    for (int i = 0; i < 2; ++i) {
        cudaEventCreateWithFlags(&made[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&used[i], cudaEventDisableTiming);
    }
    cudaError_t e = cudaEventRecord(ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux, ev_start, 0);
    for (size_t c = 0; c < n_chunks && e == cudaSuccess; ++c) {
        const int sl = (int)(c & 1);
        const uint32_t c0 = row_begin + (uint32_t)(c * chunk);
        const uint32_t c1 = (uint32_t)std::min<size_t>(c0 + chunk, row_end);
        // the spectra are made for the even-aligned row pairs that a stored bank
        // uses, partner rows outside the slice included: each spectrum carries
        // its partner's rounding, so the outputs equal the stored bank's
        const uint32_t s0 = c0 & ~1u;
        const uint32_t s1 = (uint32_t)std::min<size_t>((c1 + 1) & ~1u, bank->rows);
        if (c >= 2) e = cudaStreamWaitEvent(ctx->aux, used[sl], 0);
        if (e == cudaSuccess)
            e = template_spectra(bank, s0, s1 - s0, scratch, synth_rows, tw, slot[sl], ctx->n_sm, ctx->aux);
        if (e == cudaSuccess) e = cudaEventRecord(made[sl], ctx->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, made[sl], 0);
        for (FftParams& p : batches) {
            if (e != cudaSuccess) break;
            p.hspec = slot[sl];
            p.hrow0 = s0;
            p.k_lo = c0;
            p.k_hi = c1;
            e = launch_corr_fft(p, ctx->n_sm, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(used[sl], st);
    }
    // events may be destroyed while pending work still references them
    cudaEventDestroy(ev_start);
    for (int i = 0; i < 2; ++i) {
        cudaEventDestroy(made[i]);
        cudaEventDestroy(used[i]);
    }
    return e;
}

}  // namespace bfi
