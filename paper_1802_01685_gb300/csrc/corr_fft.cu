// Correlation by FFT: the paper's own route to the filter output (Sect. 2.2
// and Fig. 5: the output of every template against data segments through
// single-precision FFTs on the GPU, with only the tails rho > kappa sigma
// leaving the device).  Overlap-save: with segments of F samples,
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
// Every transform here is a complex FFT of N = 8192 points in one CTA.  Two
// ways of using it:
//  * the real route (plain banks): segments of F = 2N = 16384 samples.  The
//    real input of length F is packed as N complex values (even samples in
//    the real part, odd in the imaginary) and the half spectra of N + 1 bins
//    are separated from the complex transform by the usual even/odd split; the
//    inverse runs the same way backwards: the N complex outputs of one inverse
//    transform are the correlation at 2N consecutive lags of ONE template.
//    At M = 4096 that is 12289 useful lags per transform.
//  * the pair route (quadrature banks): segments of F = N = 8192 samples and
//    a template with its quadrature partner in one complex transform, output
//    |c_cos + i c_sin| at the V = 8193 - M lags of the segment.
//
// GB300 layout of the work:
//  * template spectra are kept by a stored bank in HBM (made once) and made
//    per call for a generated bank, chunk by chunk, in a two-slot ring on the
//    auxiliary stream;
//  * each segment spectrum is computed once per call; all of them stay in L2
//    and reach shared memory by asynchronous copies (cp.async) issued one
//    segment ahead; the segment's window norms are read from L2 straight
//    into registers;
//  * one CTA of 512 threads owns a template (real route) or a pair (pair
//    route) at a time and holds its spectra in registers (16 bins per
//    thread).  For every segment it forms the product spectrum; the first FFT
//    pass reads, per thread, 8 bins it formed itself and 8 that the mirror
//    thread formed (Hermitian symmetry), exchanged through shared memory; it
//    runs one inverse transform in shared memory, alternating between two
//    work arrays, and reduces the output in registers, with a warp-level
//    test before the max/argmax and tail work.  The last radix-2 stage of the
//    FFT is fused into the epilogue, so the filter output never reaches HBM.
//  * The FFT is a Stockham autosort FFT with three radix-16 passes (each
//    thread one 16-point DFT per pass, in registers) and a final radix-2
//    stage; the work array holds complex values with index i stored at
//    i + i/16, so that every pass moves a warp's 64-bit values in the
//    minimum two wavefronts, and every thread addresses it at fixed offsets
//    from one base.  Twiddles: the second pass reads a [15][16] table, the
//    third reads e^{2 pi i r k / 4096} for r = 1, 2, 3, 4, 8, 12 and forms the
//    others as one product of two; the last stage and the real route's
//    even/odd split use per-thread constants e^{i pi tid / 4096} and
//    e^{i pi tid / 8192} (rounded from FP64 once per thread) times exact-
//    to-rounding roots of unity.  The tables are rounded from FP64 once per
//    context and copied into shared memory by every CTA.
//  * The transform's rounding error scales with its whole segment, so lags
//    whose window holds almost none of the segment's energy are taken out of
//    the FFT route (k_fft_flags) and computed directly (k_fft_fixup).
#include "corr_common.cuh"
#include "synth.cuh"
#include "runtime.h"

namespace bfi {

namespace {

constexpr int FN = FFT_POINTS;            // 8192 complex points per transform
constexpr int FH = FN / 2;                // 4096
constexpr int FR = 2 * FN;                // 16384 samples per segment of the real route
constexpr int FT = 512;                   // threads per FFT block
constexpr int FBINS = FH / FT;            // 8 bins per thread (and their 8 mirrors)
constexpr int ZPAD = FN + FN / 16;        // padded complex values of the work array
constexpr int ROW = FT + FT / 16;         // padded distance of elements 512 apart (544)
constexpr int UPPER = FH + FH / 16;       // padded distance of elements 4096 apart (4352)
// twiddle tables e^{+2 pi i n / 8192}: pass 2 [15][16] (r (j mod 16) units of
// 32), pass 3 [6][256] (r (j mod 256) units of 2 for r = 1, 2, 3, 4, 8, 12)
constexpr int TW2 = 0, TW3 = 15 * 16, TW_N = TW3 + 6 * 256;     // 1776 entries
// shared memory: work array, twiddles, then (correlation only) a second work
// array, so that the passes alternate between the two, and the staged segment
// spectrum (FH bins on the pair route, FN on the real route)
constexpr size_t FFT_SMEM = (ZPAD + TW_N) * sizeof(float2);
constexpr size_t CORR_SMEM = FFT_SMEM + ZPAD * sizeof(float2) + FH * sizeof(float2);
constexpr size_t RCORR_SMEM = FFT_SMEM + ZPAD * sizeof(float2) + FN * sizeof(float2);
static_assert(RCORR_SMEM <= 227 * 1024, "real-route correlation fits one SM's shared memory");
static_assert(FFT_SMEM % 16 == 0 && (FFT_SMEM + ZPAD * sizeof(float2)) % 16 == 0, "16-byte staging");

__global__ void k_fft_tables(float2* __restrict__ tw)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < TW_N; e += gridDim.x * blockDim.x) {
        int n;                                    // exponent in units of 2 pi / 8192
        if (e < TW3) {
            n = ((e - TW2) / 16 + 1) * ((e - TW2) % 16) * 32;
        } else {
            const int q = (e - TW3) / 256, k = (e - TW3) % 256;
            const int r = q < 4 ? q + 1 : 4 * (q - 2);           // 1, 2, 3, 4, 8, 12
            n = r * k * 2;
        }
        double sn, cs;
        sincospi((double)n / 4096.0, &sn, &cs);
        tw[e] = make_float2((float)cs, (float)sn);
    }
}

// Work array z (complex, index i stored at i + i/16), twiddle tables, and, in
// the correlation kernels, a second work array z2 and the staged spectrum x.
struct Smem {
    float2* z;
    const float2* tw;
    float2* z2;
    float2* x;
};

template <bool CORR>
__device__ __forceinline__ Smem smem_setup(const float2* __restrict__ tw_global)
{
    extern __shared__ __align__(16) float2 fsm[];
    Smem m{fsm, fsm + ZPAD, CORR ? fsm + ZPAD + TW_N : nullptr, CORR ? fsm + 2 * ZPAD + TW_N : nullptr};
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

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void rotate(float& r, float& i, float2 w)
{
    const float a = r * w.x - i * w.y;
    i = r * w.y + i * w.x;
    r = a;
}

// e^{i pi a / 16} for a compile-time a in [0, 16): cos(pi a/16) for a <= 8 is
// C[a], past 8 it is -C[16 - a]; sin(pi a/16) is C[8 - a], past 8 C[a - 8]
__device__ __forceinline__ float2 root32(int a)
{
    const float C[9] = {1.0f, 0.9807852804032304491262f, 0.9238795325112867561282f,
                        0.8314696123025452370788f, 0.7071067811865475244008f,
                        0.5555702330196022247428f, 0.3826834323650897717285f,
                        0.1950903220161282678483f, 0.0f};
    return a <= 8 ? make_float2(C[a], C[8 - a]) : make_float2(-C[16 - a], C[a - 8]);
}

// e^{i pi tid / den}, rounded from FP64 (a per-thread constant)
__device__ __forceinline__ float2 thread_root(double den)
{
    double sn, cs;
    sincospi((double)threadIdx.x / den, &sn, &cs);
    return make_float2((float)cs, (float)sn);
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
// The second half of a pass, from the 16 inputs already in registers, into
// the work array dst; it ends with a barrier, before which the calling
// thread's pending cp.async groups but WAIT_CP are waited for (WAIT_CP < 0:
// no wait).
template <int SIGN, int NS, int WAIT_CP = -1>
__device__ __forceinline__ void pass16_from(const Smem& m, float2* dst, float (&vr)[16], float (&vi)[16])
{
    const int j = threadIdx.x;
    if (NS == 16) {
        const float2* t = m.tw + TW2 + (j % 16);
#pragma unroll
        for (int r = 1; r < 16; ++r) rotate(vr[r], vi[r], tw_get<SIGN>(t, (r - 1) * 16));
    } else if (NS == 256) {
        // e^{2 pi i r k / 4096}, k = j mod 256, from r = 1, 2, 3, 4, 8, 12
        const float2* t = m.tw + TW3 + (j % 256);
        const float2 w1 = tw_get<SIGN>(t, 0), w2 = tw_get<SIGN>(t, 256), w3 = tw_get<SIGN>(t, 512);
        const float2 w4 = tw_get<SIGN>(t, 768), w8 = tw_get<SIGN>(t, 1024), w12 = tw_get<SIGN>(t, 1280);
        rotate(vr[1], vi[1], w1);
        rotate(vr[2], vi[2], w2);
        rotate(vr[3], vi[3], w3);
        rotate(vr[4], vi[4], w4);
        rotate(vr[5], vi[5], cmul(w4, w1));
        rotate(vr[6], vi[6], cmul(w4, w2));
        rotate(vr[7], vi[7], cmul(w4, w3));
        rotate(vr[8], vi[8], w8);
        rotate(vr[9], vi[9], cmul(w8, w1));
        rotate(vr[10], vi[10], cmul(w8, w2));
        rotate(vr[11], vi[11], cmul(w8, w3));
        rotate(vr[12], vi[12], w12);
        rotate(vr[13], vi[13], cmul(w12, w1));
        rotate(vr[14], vi[14], cmul(w12, w2));
        rotate(vr[15], vi[15], cmul(w12, w3));
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
        dst[wb + off] = make_float2(vr[p], vi[p]);
    }
    if (WAIT_CP >= 0) cp_async_wait<(WAIT_CP >= 0 ? WAIT_CP : 0)>();
    __syncthreads();
}

// A pass from work array src to dst; in place (src == dst) every thread's
// reads complete at a barrier before the first write.
template <int SIGN, int NS, int WAIT_CP = -1, bool IN_PLACE = true>
__device__ __forceinline__ void pass16(const Smem& m, const float2* src, float2* dst)
{
    const int j = threadIdx.x;
    const int rd = j + (j >> 4);
    float vr[16], vi[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const float2 v = src[rd + ROW * r];
        vr[r] = v.x;
        vi[r] = v.y;
    }
    if (IN_PLACE) __syncthreads();
    pass16_from<SIGN, NS, WAIT_CP>(m, dst, vr, vi);
}

template <int SIGN>
__device__ __forceinline__ void fft_passes(const Smem& m)
{
    pass16<SIGN, 1>(m, m.z, m.z);
    pass16<SIGN, 16>(m, m.z, m.z);
    pass16<SIGN, 256>(m, m.z, m.z);
}

// twiddle e^{SIGN i pi k / 4096} of the final radix-2 stage for k = tid + 512 i
// (base_f = e^{i pi tid / 4096})
template <int SIGN>
__device__ __forceinline__ float2 final_tw(float2 base_f, int i)
{
    const float2 w = cmul(base_f, root32(2 * i));
    return make_float2(w.x, SIGN > 0 ? w.y : -w.y);
}

// The final radix-2 stage for output pair (k, k + 4096), k = tid + 512 i, with
// its twiddle w = final_tw<SIGN>(base_f, i), from the work array z.
__device__ __forceinline__ void fft_final(const float2* z, int i, float2 w, float2& lo, float2& hi)
{
    const int a = threadIdx.x + (threadIdx.x >> 4) + ROW * i;
    const float2 v = z[a + UPPER];
    float vr = v.x, vi = v.y;
    rotate(vr, vi, w);
    const float2 u = z[a];
    lo = make_float2(u.x + vr, u.y + vi);
    hi = make_float2(u.x - vr, u.y - vi);
}

// Z[8192 - k] = the upper output of the final stage at 4096 - k, 1 <= k < 4096,
// whose twiddle e^{SIGN i pi (4096 - k) / 4096} is -conj(w), w that of k
__device__ __forceinline__ float2 fft_final_mirror(const float2* z, int k, float2 w)
{
    const int kk = FH - k;
    const int a = kk + (kk >> 4);
    const float2 v = z[a + UPPER];
    float vr = v.x, vi = v.y;
    rotate(vr, vi, make_float2(-w.x, w.y));
    const float2 u = z[a];
    return make_float2(u.x - vr, u.y - vi);
}

// Half spectrum of a real signal s of F = 16384 samples from the complex
// transform U of u[n] = s[2n] + i s[2n+1] (in the work array after
// fft_passes<-1>): with E = (U[k] + conj U[N-k]) / 2 and
// O = (U[k] - conj U[N-k]) / 2i the transforms of the even and odd samples,
//   S[k] = E + e^{-i pi k / N} O,   S[N - k] = conj(E - e^{-i pi k / N} O),
//   S[N/2] = conj(U[N/2]),  S[0] = E_0 + O_0,  S[N] = E_0 - O_0 (real).
// Calls emit(i, slot, k, S[k]) for this thread's bins: slot 0 for
// k = tid + 512 i, slot 1 for N - k (i < 8); thread 0, i = 0 emits slot 0
// with k = 0 and (S[0], S[N]) packed, and slot 2 with k = N/2.  i is a
// compile-time constant in each call.
template <typename Emit>
__device__ __forceinline__ void real_spectrum(const Smem& m, float2 base_f, float2 base_r, Emit emit)
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < FBINS; ++i) {
        const int k = tid + FT * i;
        const float2 w = final_tw<-1>(base_f, i);
        float2 zk, zh;
        fft_final(m.z, i, w, zk, zh);                               // U[k], U[k + 4096]
        if (k == 0) {
            emit(i, 0, 0, make_float2(zk.x + zk.y, zk.x - zk.y));
            emit(i, 2, FH, make_float2(zh.x, -zh.y));
        } else {
            const float2 zm = fft_final_mirror(m.z, k, w);         // U[N - k]
            const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            const float2 wr = cmul(base_r, root32(i));            // e^{i pi k / N}
            const float2 wo = cmul(make_float2(wr.x, -wr.y), o);
            emit(i, 0, k, make_float2(e.x + wo.x, e.y + wo.y));
            emit(i, 1, FN - k, make_float2(e.x - wo.x, wo.y - e.y));
        }
    }
}

// the spectrum as out[0 .. N), out[0] = (S[0], S[N])
__device__ __forceinline__ void real_spectrum_out(const Smem& m, float2 base_f, float2 base_r,
                                                  float2* __restrict__ out)
{
    real_spectrum(m, base_f, base_r, [&](int, int, int k, float2 v) { out[k] = v; });
}

// Spectra of segments of a batch of series.  Pair route (F = 8192): the real
// segment through one complex transform, half spectrum of 4096 bins with bin
// 0 = (DC, Nyquist).  Real route (F = 16384): even/odd packed, 8192 bins with
// bin 0 = (DC, Nyquist).
template <bool REAL>
__global__ void __launch_bounds__(FT, 1) k_fft_series(const __grid_constant__ FftSeriesBatch p,
                                                      uint32_t total)
{
    const Smem m = smem_setup<false>(p.tw);
    const int tid = threadIdx.x;
    const float2 base_f = thread_root(4096.0);
    const float2 base_r = thread_root(8192.0);
    for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
        int s = 0;
        while (s + 1 < p.n && g >= p.seg_begin[s + 1]) ++s;
        const uint32_t j = g - p.seg_begin[s];
        const float* x = p.x[s];
        const uint64_t N = p.N[s], t0 = (uint64_t)j * p.V;
        if (REAL) {
            for (int n = tid; n < FN; n += FT) {
                const uint64_t a = t0 + 2 * (uint64_t)n;
                m.z[n + (n >> 4)] = make_float2(a < N ? x[a] : 0.f, a + 1 < N ? x[a + 1] : 0.f);
            }
        } else {
            for (int n = tid; n < FN; n += FT) m.z[n + (n >> 4)] = make_float2(t0 + n < N ? x[t0 + n] : 0.f, 0.f);
        }
        __syncthreads();
        fft_passes<-1>(m);
        if (REAL) {
            real_spectrum_out(m, base_f, base_r, p.spec[s] + (size_t)j * FN);
        } else {
            float2* out = p.spec[s] + (size_t)j * FH;
#pragma unroll
            for (int i = 0; i < FBINS; ++i) {
                float2 lo, hi;
                fft_final(m.z, i, final_tw<-1>(base_f, i), lo, hi);
                out[tid + FT * i] = (tid == 0 && i == 0) ? make_float2(lo.x, hi.x) : lo;
            }
        }
        __syncthreads();
    }
}

// Template spectra of a chunk of synthesised rows (rows of 8192 samples, zero
// past M), pair route: rows (2q, 2q + 1) through one complex transform of
// h_a + i h_b, separated by Hermitian symmetry into two half spectra of 4096
// bins.
__global__ void __launch_bounds__(FT, 1) k_fft_bank_pair(const float* __restrict__ rows, uint32_t n_rows,
                                                         uint32_t n_items, const float2* __restrict__ tw,
                                                         float2* __restrict__ spec)
{
    const Smem m = smem_setup<false>(tw);
    const int tid = threadIdx.x;
    const float2 base_f = thread_root(4096.0);
    for (uint32_t q = blockIdx.x; q < n_items; q += gridDim.x) {
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
            const float2 w = final_tw<-1>(base_f, i);
            float2 zk, zn;
            fft_final(m.z, i, w, zk, zn);          // Z[k], Z[k + 4096]
            if (k == 0) {
                // DC and Nyquist of both real templates: real parts of Z[0], Z[4096]
                sa[0] = make_float2(zk.x, zn.x);
                if (b < n_rows) sb[0] = make_float2(zk.y, zn.y);
            } else {
                const float2 zm = fft_final_mirror(m.z, k, w);    // Z[F - k]
                // H_a = (Z[k] + conj Z[F-k]) / 2,  H_b = (Z[k] - conj Z[F-k]) / 2i
                sa[k] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                if (b < n_rows) sb[k] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
            }
        }
        __syncthreads();
    }
}

// Template spectra of the real route from synthesised rows (8192 samples each,
// zero past M): one row per transform, even/odd packed into 4096 complex
// values and zero past them (the 16384-sample segment), 8192 bins per row.
// While one row is transformed the next one's first M samples arrive by
// cp.async, and the passes alternate between the two work arrays: four
// barriers per row.  The route takes M <= 4096, so the inputs past the first
// quarter of the transform are zero, and the first pass knows it at compile
// time.
__global__ void __launch_bounds__(FT, 1) k_fft_bank_real(const float* __restrict__ rows, uint32_t n_rows,
                                                         uint32_t M, const float2* __restrict__ tw,
                                                         float2* __restrict__ spec)
{
    const Smem m = smem_setup<true>(tw);
    const int tid = threadIdx.x;
    const float2 base_f = thread_root(4096.0);
    const float2 base_r = thread_root(8192.0);
    const uint32_t n16 = (M + 3) / 4;             // 16-byte pieces holding a row's first M samples
    const uint32_t mh = 2 * n16;                  // complex values staged (M <= FH: mh <= FH / 2)
    uint32_t q = blockIdx.x;
    if (q >= n_rows) return;
    auto stage = [&](uint32_t r) {
        const float* src = rows + (size_t)r * FN;
        for (uint32_t c = tid; c < n16; c += FT) cp_async16(m.x + 2 * c, src + 4 * c);
    };
    stage(q);
    cp_async_commit();
    for (;;) {
        cp_async_wait<0>();
        __syncthreads();                          // the row staged; the previous spectrum read
        float vr[16], vi[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const uint32_t n = (uint32_t)(tid + FT * r);
            const float2 v = r < FBINS / 2 && n < mh ? m.x[n] : make_float2(0.f, 0.f);
            vr[r] = v.x;
            vi[r] = v.y;
        }
        pass16_from<-1, 1>(m, m.z, vr, vi);       // every thread has read its staged values
        const uint32_t qn = q + gridDim.x;
        if (qn < n_rows) stage(qn);
        cp_async_commit();
        pass16<-1, 16, -1, false>(m, m.z, m.z2);
        pass16<-1, 256, -1, false>(m, m.z2, m.z);
        real_spectrum_out(m, base_f, base_r, spec + (size_t)q * FN);
        if (qn >= n_rows) break;
        q = qn;
    }
}

// ---- Parseval predictor of sigma (Sect. 2.2, Fig. 5 caption): periodograms
// and template power spectra on the real route's 16384-point transform.

// |S[k]|^2, k = 0 .. N, of this thread's bins into out (N + 1 floats)
__device__ __forceinline__ void real_power_out(const Smem& m, float2 base_f, float2 base_r,
                                               float* __restrict__ out)
{
    real_spectrum(m, base_f, base_r, [&](int, int, int k, float2 v) {
        if (k == 0) {
            out[0] = v.x * v.x;
            out[FN] = v.y * v.y;
        } else {
            out[k] = v.x * v.x + v.y * v.y;
        }
    });
}

// Periodograms of the Welch segments of a batch of series: segment g of
// series s covers samples [g F/2, g F/2 + F), zero past the end; row
// seg_begin[s] + g of pseg gets |S[k]|^2 for k = 0 .. N.
__global__ void __launch_bounds__(FT, 1) k_welch_segments(const __grid_constant__ WelchBatch p, uint32_t total)
{
    const Smem m = smem_setup<false>(p.tw);
    const int tid = threadIdx.x;
    const float2 base_f = thread_root(4096.0);
    const float2 base_r = thread_root(8192.0);
    for (uint32_t g = blockIdx.x; g < total; g += gridDim.x) {
        int s = 0;
        while (s + 1 < p.n && g >= p.seg_begin[s + 1]) ++s;
        const uint64_t N = p.N[s], a0 = (uint64_t)(g - p.seg_begin[s]) * FN;      // hop F/2 = N
        const float* x = p.x[s];
        for (int n = tid; n < FN; n += FT) {
            const uint64_t a = a0 + 2 * (uint64_t)n;
            m.z[n + (n >> 4)] = make_float2(a < N ? x[a] : 0.f, a + 1 < N ? x[a + 1] : 0.f);
        }
        __syncthreads();
        fft_passes<-1>(m);
        real_power_out(m, base_f, base_r, p.pseg + (size_t)g * PRED_BINS);
        __syncthreads();
    }
}

// P_s(k) = c_s / S_s sum_g pseg[g](k) over the S_s segments of series s, the
// sum in FP64 in segment order; c_s = 1, or F / N_s for a series shorter than
// F (one zero-padded segment).  Grid: (bins, series).
__global__ void k_welch_mean(const __grid_constant__ WelchBatch p)
{
    const int s = blockIdx.y;
    if (s >= p.n) return;
    const uint32_t g0 = p.seg_begin[s], S = p.seg_begin[s + 1] - g0;
    const double c = p.N[s] < (uint64_t)PRED_F ? (double)PRED_F / (double)p.N[s] : 1.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < (uint32_t)PRED_BINS; k += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (uint32_t g = 0; g < S; ++g) acc += (double)p.pseg[(size_t)(g0 + g) * PRED_BINS + k];
        p.P[(size_t)s * PRED_BINS + k] = (float)(acc * c / (double)S);
    }
}

// For template rows q < n_rows of a chunk (8192 samples each, zero past M):
// D[s][row0 + q] = sum over all F bins of P_s(f) |H_q(f)|^2, i.e. the bins
// 0 and N once and the others twice, for each series s < n_ser; the partial
// sums per thread in FP32 (16 terms), across the CTA in FP64.
__global__ void __launch_bounds__(FT, 1) k_template_power_dot(const float* __restrict__ rows, uint32_t n_rows,
                                                              const float2* __restrict__ tw,
                                                              const float* __restrict__ P, uint32_t n_ser,
                                                              float* __restrict__ D, uint32_t d_stride,
                                                              uint32_t row0)
{
    const Smem m = smem_setup<false>(tw);
    __shared__ double red[FT / 32];
    const int tid = threadIdx.x;
    const float2 base_f = thread_root(4096.0);
    const float2 base_r = thread_root(8192.0);
    for (uint32_t q = blockIdx.x; q < n_rows; q += gridDim.x) {
        const float2* r2 = reinterpret_cast<const float2*>(rows + (size_t)q * FN);
        for (int n = tid; n < FN; n += FT) m.z[n + (n >> 4)] = n < FH ? r2[n] : make_float2(0.f, 0.f);
        __syncthreads();
        fft_passes<-1>(m);
        // this thread's weighted powers: pw[i] at k = tid + 512 i, pm[i] at
        // N - k (thread 0, i = 0: S[0] and S[N], each once); thread 0 also
        // holds the middle bin N/2 in mid
        float pw[FBINS], pm[FBINS], mid = 0.f;
        real_spectrum(m, base_f, base_r, [&](int i, int slot, int k, float2 v) {
            const float a = 2.f * (v.x * v.x + v.y * v.y);
            if (slot == 0 && k == 0) {                      // S[0] and S[N], each once
                pw[i] = v.x * v.x;
                pm[i] = v.y * v.y;
            } else if (slot == 0) {
                pw[i] = a;
            } else if (slot == 1) {
                pm[i] = a;
            } else {
                mid = a;
            }
        });
        __syncthreads();                        // work array read: the next row may load
        for (uint32_t s = 0; s < n_ser; ++s) {
            const float* Ps = P + (size_t)s * PRED_BINS;
            float acc = tid == 0 ? mid * Ps[FH] : 0.f;
#pragma unroll
            for (int i = 0; i < FBINS; ++i) {
                const int k = tid + FT * i;
                acc = fmaf(pw[i], Ps[k], acc);
                acc = fmaf(pm[i], Ps[k == 0 ? FN : FN - k], acc);
            }
            double d = (double)acc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if ((tid & 31) == 0) red[tid >> 5] = d;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < FT / 32; ++w) tot += red[w];
                D[(size_t)s * d_stride + row0 + q] = (float)tot;
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ void push_tail(const FftParams& p, uint32_t series, uint32_t k, uint32_t tau,
                                          float rho)
{
    unsigned int i = atomicAdd(p.cand_count, 1u);
    if (i < p.cand_cap) p.cand[i] = Candidate{series, k, tau, rho};
}

// running max |rho| with its first lag, as the packed key of pack_max (|rho|
// >= 0, so its bits order as its values; then the lower lag): one unsigned
// 64-bit max per update, whatever order the lags arrive in
__device__ __forceinline__ void track_max(float a, uint32_t tau, unsigned long long& best)
{
    const unsigned long long key = pack_max(a, tau);
    best = key > best ? key : best;
}

// the largest of the warp's packed keys: the largest value bits, then among
// the lanes that hold them the largest low word (the earliest lag)
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long k)
{
    const uint32_t hi = __reduce_max_sync(0xffffffffu, (uint32_t)(k >> 32));
    const uint32_t lo = __reduce_max_sync(0xffffffffu, (uint32_t)(k >> 32) == hi ? (uint32_t)k : 0u);
    return ((unsigned long long)hi << 32) | lo;
}

// the warp's largest of the non-negative g (float bits order as values)
__device__ __forceinline__ float warp_max_abs(float g)
{
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(g)));
}

// segment spectrum of NX bins into shared memory (16-byte asynchronous copies)
template <int NX>
__device__ __forceinline__ void stage_spectrum(const Smem& m, const float2* src)
{
    for (int c = threadIdx.x; c < NX / 2; c += FT) cp_async16(m.x + 2 * c, src + 2 * c);
}

// a 128-byte line from DRAM into L2 (no register, no wait)
__device__ __forceinline__ void prefetch_l2(const void* g)
{
    asm volatile("prefetch.global.L2 [%0];\n" ::"l"(g));
}

// warp reduction of a packed max key and a sum, then one atomic each per warp
__device__ __forceinline__ void publish(unsigned long long key, double d, unsigned long long* vmax,
                                       double* sumsq)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        key = ok > key ? ok : key;
        d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(vmax, key);
        atomicAdd(sumsq, d);
    }
}

// The transform of an item in both correlation kernels alternates between the
// two work arrays, so that no pass waits for the reads of the one before:
//   product spectrum from x: own bins in registers, mirrors into z   barrier 1
//   (the next segment's spectrum starts to arrive in x)
//   pass 1: registers and the mirrors read from z, into z2           barrier 2
//   pass 2: z2 into z                                                 barrier 3
//   pass 3: z into z2 (and the next spectrum has arrived)             barrier 4
//   final radix-2 stage and epilogue read z2.
// Each array's last reads come before the barrier that precedes its next
// write: z is read by pass 3 (before barrier 4) and written by the next item's
// product spectrum; z2 is read by the epilogue and written only after the next
// item's barrier 1; x is read by the product spectrum and refilled after
// barrier 1.  Four barriers per item.  The window norms (the per-segment copy,
// 16-byte aligned rows, carrying 1/F) are read from L2 into registers, half of
// them while pass 3 runs and half while the first half of the epilogue runs.

// this thread's norms for the lag pairs t = 2 (tid + 512 (I0 + u) + 4096 h),
// u < 4, of the real route (zero past the segment's nv lags)
template <int I0>
__device__ __forceinline__ void load_norm_pairs(const float* __restrict__ nrm, uint32_t nv, float2 (&iv)[8])
{
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t t = 2u * (uint32_t)(threadIdx.x + FT * (I0 + u) + FH * h);
            iv[2 * u + h] = t < nv ? __ldg(reinterpret_cast<const float2*>(nrm + t)) : make_float2(0.f, 0.f);
        }
}

// the same for the lags t = tid + 512 (I0 + u) + 4096 h of the pair route
template <int I0>
__device__ __forceinline__ void load_norms(const float* __restrict__ nrm, uint32_t nv, float (&iv)[8])
{
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t t = (uint32_t)(threadIdx.x + FT * (I0 + u) + FH * h);
            iv[2 * u + h] = t < nv ? __ldg(nrm + t) : 0.f;
        }
}

// The correlation of the real route (plain banks).  Each CTA walks its items
// (template row, series, segment) in order; while the FFT of one segment
// runs, the spectrum of the next one arrives in shared memory.
// DENSE: a series of the launch keeps the dense output rho (a compile-time
// copy, so that the common case carries no per-lag test for it)
template <bool DENSE>
__global__ void __launch_bounds__(FT, 1) k_corr_rfft(const __grid_constant__ FftParams p)
{
    const Smem m = smem_setup<true>(p.tw);
    const int tid = threadIdx.x;
    const float2 base_f = thread_root(4096.0);
    const float2 base_r = thread_root(8192.0);
    const uint32_t n_rows = p.k_hi - p.k_lo;
    uint32_t row = blockIdx.x;
    if (row >= n_rows || p.n_ser == 0) return;
    int s = 0;
    uint32_t j = 0;
    stage_spectrum<FN>(m, p.ser[0].spec);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    float2 hk[FBINS], hp[FBINS], hm = make_float2(0.f, 0.f);
    uint32_t k = 0;
    float thr = 0.f;
    // the warp's packed max key over the series so far (0: none yet) and its
    // value: a lag below both it and the tail threshold changes nothing
    unsigned long long best = 0ull;
    float best_v = 0.f;
    // per-thread sum of rho^2 over a series (a few thousand terms of similar
    // size: FP32 is ample); the sum over threads is FP64
    float ss = 0.f;
    bool new_row = true, new_series = true;

    for (;;) {
        const FftSeries& S = p.ser[s];
        if (new_row) {
            k = p.k_lo + row;
            const float2* H = p.hspec + (size_t)(k - p.hrow0) * FN;
#pragma unroll
            for (int i = 0; i < FBINS; ++i) {
                const int f = tid + FT * i;
                hk[i] = H[f];
                hp[i] = H[(FN - f) & (FN - 1)];
            }
            if (tid == 0) hm = H[FH];
        }
        const uint32_t o = k - p.k_begin;
        (void)BF_BOUNDS(p.err, o < p.k_end - p.k_begin && k >= p.hrow0 && j < S.nseg);
        if (new_series) {
            thr = S.sigma_pred ? S.kappa * S.sigma_pred[o] : p.thr;
            best = 0ull;
            best_v = 0.f;
            ss = 0.f;
        }
        const uint32_t t0 = j * p.V;
        const uint32_t nv = min(p.V, S.L - t0);
        const float* nrm = S.inv + (size_t)j * p.Vp;     // (BF_BOUNDS above: j < nseg)
        // the item after this one
        uint32_t np = row, nj = j + 1;
        int ns = s;
        if (nj >= S.nseg) {
            nj = 0;
            if (++ns >= p.n_ser) {
                ns = 0;
                np = row + gridDim.x;
            }
        }
        // Y = X conj(H) over all F bins, and the packed spectrum
        // Z'[f] = A + i w B, Z'[N - f] = conj(A - i w B), with A = Y[f] +
        // conj Y[N-f], B = Y[f] - conj Y[N-f], w = e^{i pi f / N}: twice the
        // transform of c[2n] + i c[2n+1].  The first pass of the FFT reads
        // Z'[tid + 512 r]: for r < 8 this thread's own, kept in registers; for
        // r >= 8 those of the mirror thread 512 - tid (thread 0: its own
        // mirrors and the middle bin), exchanged through shared memory in an
        // unpadded [8][512] layout of its own: reader j finds Z'[j + 512 r] at
        // (r - 8) 512 + j, which writer tid fills for its bin r' at
        // (8 - r') 512 - tid (the middle bin at 0).  A half-warp then writes,
        // and reads, 16 consecutive values: no bank conflict either way.
        float vr[16], vi[16];
#pragma unroll
        for (int r = 0; r < FBINS; ++r) {
            const int f = tid + FT * r;
            if (tid == 0 && r == 0) {
                // DC and Nyquist (real): Z'[0] = (Y0 + YN) + i (Y0 - YN);
                // middle bin: Z'[N/2] = 2 conj(Y[N/2]) = 2 conj(X) H
                const float2 x0 = m.x[0];
                const float y0 = x0.x * hk[0].x, yn = x0.y * hk[0].y;
                vr[0] = y0 + yn;
                vi[0] = y0 - yn;
                const float2 xm = m.x[FH];
                m.z[0] = make_float2(2.f * (xm.x * hm.x + xm.y * hm.y), 2.f * (xm.x * hm.y - xm.y * hm.x));
            } else {
                const float2 xk = m.x[f], xq = m.x[FN - f];
                const float ykr = xk.x * hk[r].x + xk.y * hk[r].y, yki = xk.y * hk[r].x - xk.x * hk[r].y;
                const float yqr = xq.x * hp[r].x + xq.y * hp[r].y, yqi = xq.y * hp[r].x - xq.x * hp[r].y;
                const float ar = ykr + yqr, ai = yki - yqi;
                const float br = ykr - yqr, bi = yki + yqi;
                const float2 w = cmul(base_r, root32(r));
                const float wbr = w.x * br - w.y * bi, wbi = w.x * bi + w.y * br;
                vr[r] = ar - wbi;
                vi[r] = ai + wbr;
                m.z[(FBINS - r) * FT - tid] = make_float2(ar + wbi, wbr - ai);
            }
        }
        __syncthreads();                            // 1
        if (np < n_rows) stage_spectrum<FN>(m, p.ser[ns].spec + (size_t)nj * FN);
        cp_async_commit();
        if (np != row && np < n_rows)               // the next row's template spectrum into L2 (64 KiB)
            prefetch_l2(p.hspec + (size_t)(p.k_lo + np - p.hrow0) * FN + 16 * tid);
#pragma unroll
        for (int r = FBINS; r < 16; ++r) {
            const float2 v = m.z[(r - FBINS) * FT + tid];
            vr[r] = v.x;
            vi[r] = v.y;
        }
        pass16_from<1, 1>(m, m.z2, vr, vi);               // 2
        pass16<1, 16, -1, false>(m, m.z2, m.z);           // 3
        float2 iv0[8], iv1[8];
        load_norm_pairs<0>(nrm, nv, iv0);
        pass16<1, 256, 0, false>(m, m.z, m.z2);           // 4, and the next segment's spectrum
        load_norm_pairs<4>(nrm, nv, iv1);
        float pa = 0.f;
        // lag pairs t = 2 (tid + 512 i + 4096 h) for i = i0 + u, with norms iv
        auto lags = [&](const int i0, const float2 (&iv)[8]) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u;
                float2 w = final_tw<1>(base_f, u);     // e^{i pi (tid + 512 u) / 4096} ...
                if (i0) w = make_float2(-w.y, w.x);    // ... times e^{i pi / 2} for i = 4 + u
                float2 z[2];
                fft_final(m.z2, i, w, z[0], z[1]);
                // z = c[2n] + i c[2n + 1]: the lag pairs t = 2 (tid + 512 i + 4096 h);
                // norms carry 1/F (k_fft_flags), and the norm of t + 1 is 0 when t
                // is the segment's last lag, so rb is 0 there
                float ra[2], rb[2], g = 0.f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t t = 2u * (uint32_t)(tid + FT * i + FH * h);
                    ra[h] = rb[h] = 0.f;
                    if (t < nv) {
                        ra[h] = z[h].x * iv[2 * u + h].x;
                        rb[h] = z[h].y * iv[2 * u + h].y;
                        if (DENSE && S.rho) {
                            const uint32_t tau = t0 + t;
                            const bool two = t + 1 < nv;
                            if (BF_BOUNDS(p.err, tau + (two ? 1u : 0u) < S.L)) {
                                S.rho[(size_t)o * S.L + tau] = ra[h];
                                if (two) S.rho[(size_t)o * S.L + tau + 1] = rb[h];
                            }
                        }
                    }
                    pa = fmaf(ra[h], ra[h], pa);
                    pa = fmaf(rb[h], rb[h], pa);
                    g = fmaxf(g, fmaxf(fabsf(ra[h]), fabsf(rb[h])));
                }
                // only lags reaching the warp's running max (ties included: an
                // earlier lag wins them) or the tail threshold need their keys
                if (warp_max_abs(g) >= fminf(thr, best_v)) {
                    unsigned long long lk = 0ull;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t t = 2u * (uint32_t)(tid + FT * i + FH * h);
                        if (t < nv) {
                            const uint32_t tau = t0 + t;
                            const float aa = fabsf(ra[h]), ab = fabsf(rb[h]);
                            // the pair's larger |rho|, the earlier lag on ties
                            const bool second = ab > aa;
                            track_max(second ? ab : aa, second ? tau + 1 : tau, lk);
                            if (fmaxf(aa, ab) >= thr) {
                                if (aa >= thr) push_tail(p, S.series_id, k, tau, ra[h]);
                                if (t + 1 < nv && ab >= thr) push_tail(p, S.series_id, k, tau + 1, rb[h]);
                            }
                        }
                    }
                    lk = warp_max_key(lk);
                    best = lk > best ? lk : best;
                    best_v = __uint_as_float((uint32_t)(best >> 32));
                }
            }
        };
        lags(0, iv0);
        lags(4, iv1);
        ss += pa;
        if (nj == 0)                                // last segment of this series: publish
            publish(best, (double)ss, S.vmax + o, S.sumsq + o);
        if (np >= n_rows) break;
        new_row = np != row;
        new_series = nj == 0;
        row = np;
        s = ns;
        j = nj;
    }
}

// The correlation of the pair route (quadrature banks): a template and its
// quadrature partner in one complex transform, |rho| = |c_cos + i c_sin| /
// |window|.  Each CTA walks its items (pair, series, segment) in order, with
// the next segment's spectrum staged and the norms read as above.  DENSE as
// in k_corr_rfft.
template <bool DENSE>
__global__ void __launch_bounds__(FT, 1) k_corr_fft_quad(const __grid_constant__ FftParams p)
{
    const Smem m = smem_setup<true>(p.tw);
    const int tid = threadIdx.x;

    const float2 base_f = thread_root(4096.0);
    const uint32_t n_pairs = (p.k_hi - p.k_lo + 1) / 2;
    uint32_t pair = blockIdx.x;
    if (pair >= n_pairs || p.n_ser == 0) return;
    int s = 0;
    uint32_t j = 0;
    stage_spectrum<FH>(m, p.ser[0].spec);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    float2 ha[FBINS], hb[FBINS];
    uint32_t ka = 0;
    float thr = 0.f;
    unsigned long long best = 0ull;             // the warp's packed max key, as above
    float best_v = 0.f;
    float ss = 0.f;
    bool new_pair = true, new_series = true;

    for (;;) {
        const FftSeries& S = p.ser[s];
        if (new_pair) {
            ka = p.k_lo + 2 * pair;
#pragma unroll
            for (int i = 0; i < FBINS; ++i) {
                const int f = tid + FT * i;
                ha[i] = p.hspec[(size_t)(ka - p.hrow0) * FH + f];
                hb[i] = p.hspec[(size_t)(ka + 1 - p.hrow0) * FH + f];
            }
        }
        const uint32_t la = (ka - p.k_begin) >> 1;           // output index of the pair
        (void)BF_BOUNDS(p.err, ka + 1 < p.k_end && ka >= p.hrow0 && j < S.nseg);
        if (new_series) {
            thr = S.sigma_pred ? S.kappa * S.sigma_pred[la] : p.thr;
            best = 0ull;
            best_v = 0.f;
            ss = 0.f;
        }
        const uint32_t t0 = j * p.V;
        const uint32_t nv = min(p.V, S.L - t0);
        const float* nrm = S.inv + (size_t)j * p.Vp;
        uint32_t np = pair, nj = j + 1;
        int ns = s;
        if (nj >= S.nseg) {
            nj = 0;
            if (++ns >= p.n_ser) {
                ns = 0;
                np = pair + gridDim.x;
            }
        }
        // Z = X conj(H_a) + i X conj(H_b); Z[F - f] = conj(Ya) + i conj(Yb),
        // exchanged with the mirror thread as in k_corr_rfft
        float vr[16], vi[16];
#pragma unroll
        for (int i = 0; i < FBINS; ++i) {
            const float2 x = m.x[tid + FT * i];
            if (tid == 0 && i == 0) {
                // DC (x.x) and Nyquist (x.y): real products
                vr[0] = x.x * ha[0].x;
                vi[0] = x.x * hb[0].x;
                m.z[0] = make_float2(x.y * ha[0].y, x.y * hb[0].y);
            } else {
                const float yar = x.x * ha[i].x + x.y * ha[i].y;
                const float yai = x.y * ha[i].x - x.x * ha[i].y;
                const float ybr = x.x * hb[i].x + x.y * hb[i].y;
                const float ybi = x.y * hb[i].x - x.x * hb[i].y;
                vr[i] = yar - ybi;
                vi[i] = yai + ybr;
                m.z[(FBINS - i) * FT - tid] = make_float2(yar + ybi, ybr - yai);
            }
        }
        __syncthreads();                            // 1
        if (np < n_pairs) stage_spectrum<FH>(m, p.ser[ns].spec + (size_t)nj * FH);
        cp_async_commit();
        if (np != pair && np < n_pairs)             // the next pair's two spectra into L2 (64 KiB)
            prefetch_l2(p.hspec + (size_t)(p.k_lo + 2 * np - p.hrow0) * FH + 16 * tid);
#pragma unroll
        for (int r = FBINS; r < 16; ++r) {
            const float2 v = m.z[(r - FBINS) * FT + tid];
            vr[r] = v.x;
            vi[r] = v.y;
        }
        pass16_from<1, 1>(m, m.z2, vr, vi);               // 2
        pass16<1, 16, -1, false>(m, m.z2, m.z);           // 3
        float iv0[8], iv1[8];
        load_norms<0>(nrm, nv, iv0);
        pass16<1, 256, 0, false>(m, m.z, m.z2);           // 4, and the next segment's spectrum
        load_norms<4>(nrm, nv, iv1);
        float pa = 0.f;
        auto lags = [&](const int i0, const float (&iv)[8]) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u;
                float2 w = final_tw<1>(base_f, u);
                if (i0) w = make_float2(-w.y, w.x);
                float2 z[2];
                fft_final(m.z2, i, w, z[0], z[1]);
                float r[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t t = (uint32_t)(tid + FT * i + FH * h);
                    r[h] = 0.f;
                    if (t < nv) {
                        const uint32_t tau = t0 + t;
                        r[h] = sqrtf(z[h].x * z[h].x + z[h].y * z[h].y) * iv[2 * u + h];   // norms carry 1/F
                        pa = fmaf(r[h], r[h], pa);
                        if (DENSE && S.rho && BF_BOUNDS(p.err, tau < S.L)) S.rho[(size_t)la * S.L + tau] = r[h];
                    }
                }
                if (warp_max_abs(fmaxf(r[0], r[1])) >= fminf(thr, best_v)) {
                    unsigned long long lk = 0ull;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t t = (uint32_t)(tid + FT * i + FH * h);
                        if (t < nv) {
                            track_max(r[h], t0 + t, lk);
                            if (r[h] >= thr) push_tail(p, S.series_id, ka >> 1, t0 + t, r[h]);
                        }
                    }
                    lk = warp_max_key(lk);
                    best = lk > best ? lk : best;
                    best_v = __uint_as_float((uint32_t)(best >> 32));
                }
            }
        };
        lags(0, iv0);
        lags(4, iv1);
        ss += pa;
        if (nj == 0)
            publish(best, (double)ss, S.vmax + la, S.sumsq + la);
        if (np >= n_pairs) break;
        new_pair = np != pair;
        new_series = nj == 0;
        pair = np;
        s = ns;
        j = nj;
    }
}

// Lags whose window holds less than 1/FFT_FIX_RATIO2 of the energy of its
// FFT segment (e.g. a quiet stretch or the tapered edge of a loud chirp next to
// silence): the transform's rounding error scales with the segment, so there it
// would swamp rho.  Their inverse norm is set to 0, so the correlation kernel
// gives them rho = 0 (no tail, nothing to the sum of squares, never above the
// true maximum), and they are listed, with the norm, for k_fft_fixup.  The
// energies come from the FP64 prefix of x^2.  One grid row per series.
// Every norm is also written, times the inverse transform's scale (a power of
// two, so exactly), to the per-segment copy the correlation kernel reads:
// segment j's lags at inv_seg[j Vp ..), Vp = V rounded up to a multiple of 4,
// so every segment starts 16-byte aligned; past a segment's last lag its row
// holds zeros, so that the real route reads whole pairs (t, t + 1) of norms.
__global__ void __launch_bounds__(256) k_fft_flags(const __grid_constant__ FftSeriesBatch b)
{
    const int i = blockIdx.y;
    if (i >= b.n) return;
    const uint64_t L = b.L[i], N = b.N[i];
    const double* S = b.S[i];
    float* inv = b.inv[i];
    const uint32_t lane = threadIdx.x & 31;
    {
        // the zeros: Vp - V per full segment, Vp - (its lags) in the last one
        const uint64_t nseg = (L + b.V - 1) / b.V;
        const uint64_t last = L - (nseg - 1) * b.V;
        const uint64_t padv = b.Vp - b.V, n_full = (nseg - 1) * padv;
        const uint64_t n_pad = n_full + (b.Vp - last);
        for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n_pad;
             q += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t pos = q < n_full ? (q / padv) * b.Vp + b.V + q % padv
                                            : (nseg - 1) * b.Vp + last + (q - n_full);
            if (BF_BOUNDS(b.err, pos < nseg * b.Vp)) b.inv_seg[i][pos] = 0.f;
        }
    }
    // the loop bound is uniform over a warp, so each warp appends its lanes'
    // lags together, in lag order (the fixup reads them as coalesced runs)
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < L; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = base + threadIdx.x;
        bool flag = false;
        float iv = 0.f;
        if (t < L) {
            iv = inv[t];
            const uint64_t j = t / b.V;                 // the segment
            const uint64_t a = j * b.V;                 // its first sample
            if (iv > 0.f) {                             // empty window: rho = 0 exactly
                const uint64_t e = min(a + (uint64_t)b.F, N);
                const double E = S[e] - S[a];
                flag = E * (double)iv * (double)iv > FFT_FIX_RATIO2;
            }
            b.inv_seg[i][j * b.Vp + (t - a)] = flag ? 0.f : iv * b.scale;
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, flag);
        if (mask == 0u) continue;
        uint32_t slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(b.n_fix + i, (uint32_t)__popc(mask));   // each lag once: < L entries
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        const uint32_t slot = slot0 + __popc(mask & ((1u << lane) - 1u));
        if (flag && BF_BOUNDS(b.err, slot < L)) {
            inv[t] = 0.f;
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
    cudaError_t e = cudaFuncSetAttribute(k_corr_rfft<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RCORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_corr_rfft<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RCORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_corr_fft_quad<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_corr_fft_quad<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_series<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_series<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_bank_real, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CORR_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_bank_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_welch_segments, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_template_power_dot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM);
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

uint32_t fft_seg_len(bool quad) { return quad ? FN : FR; }
uint32_t fft_spec_bins(bool quad) { return quad ? FH : FN; }

// Spectra of template rows [row0, row0 + nrows) into out[0 ..] (fft_spec_bins
// complex values per row), through `scratch`, room for `scratch_rows`
// synthesised rows of 8192 samples.  The pair route rounds nrows up to even:
// an odd tail pairs with a zero row whose spectrum is not written.
// Asynchronous on st.
static cudaError_t template_spectra(const bf_bank* bank, size_t row0, size_t nrows, float* scratch,
                                    size_t scratch_rows, const float2* tw, float2* out, int n_sm,
                                    cudaStream_t st)
{
    const size_t bins = fft_spec_bins(bank->quad);
    if (bank->M > (uint32_t)FH) return cudaErrorInvalidValue;     // the route's limit (checked by the callers)
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < nrows && e == cudaSuccess; k += scratch_rows) {
        const size_t kc = std::min(scratch_rows, nrows - k);     // rows of this sub-chunk
        const size_t nr = bank->quad ? kc + (kc & 1) : kc;        // scratch_rows is even
        e = launch_bank_synth(bank->d_params, (uint32_t)(row0 + k), bank->quad, (uint32_t)kc, (uint32_t)nr,
                              bank->M, FN, bank->fs, scratch, nullptr, nullptr, st);
        if (e != cudaSuccess) break;
        const uint32_t items = (uint32_t)(bank->quad ? nr / 2 : nr);
        const unsigned grid = std::min<uint32_t>(items, (uint32_t)n_sm);
        count_launches(1);
        if (bank->quad) k_fft_bank_pair<<<grid, FT, FFT_SMEM, st>>>(scratch, (uint32_t)kc, items, tw, out + k * bins);
        else k_fft_bank_real<<<grid, FT, CORR_SMEM, st>>>(scratch, (uint32_t)kc, bank->M, tw, out + k * bins);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t fft_template_spectra(const bf_bank* bank, size_t row0, size_t nrows, float* scratch,
                                 size_t scratch_rows, const float2* tw, float2* out, int n_sm, cudaStream_t st)
{
    return template_spectra(bank, row0, nrows, scratch, scratch_rows, tw, out, n_sm, st);
}

// Spectra of every template of the bank, [rows (rounded up to even for the
// pair route)][fft_spec_bins] complex, computed once and kept with the bank.
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
    const size_t K2 = bank->quad ? bank->rows + (bank->rows & 1) : bank->rows;
    const size_t bins = fft_spec_bins(bank->quad);
    Allocator& mem = *ctx->mem;
    float2* spec = static_cast<float2*>(mem.alloc(K2 * bins * sizeof(float2)));
    const size_t chunk = std::min<size_t>(4096, K2 + (K2 & 1));
    float* rows = static_cast<float*>(mem.alloc(chunk * FN * sizeof(float)));
    if (!spec || !rows) {
        mem.release(spec);
        mem.release(rows);
        set_error("out of device memory for the template spectra (%zu MB)", (K2 * bins * 8) >> 20);
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

uint32_t fft_lags_per_seg(uint32_t M, bool quad) { return fft_seg_len(quad) - M + 1; }
uint32_t fft_norm_stride(uint32_t M, bool quad) { return (fft_lags_per_seg(M, quad) + 3) & ~3u; }
// 1/F for the real route: the inverse transform is unnormalised and the
// even/odd split forms twice the packed spectrum; 1/N for the pair route
float fft_inverse_scale(bool quad) { return 1.f / (float)fft_seg_len(quad); }

size_t fft_series_bytes(uint32_t L, uint32_t M, bool quad)
{
    const size_t nseg = fft_segments(L, M, quad);
    return nseg * fft_spec_bins(quad) * sizeof(float2) + nseg * fft_norm_stride(M, quad) * sizeof(float);
}

uint32_t fft_segments(uint32_t L, uint32_t M, bool quad)
{
    const uint64_t V = fft_lags_per_seg(M, quad);
    return (uint32_t)(((uint64_t)L + V - 1) / V);          // L may be close to 2^32
}

uint32_t welch_segments(uint64_t N)
{
    return N >= (uint64_t)PRED_F ? (uint32_t)((N - PRED_F) / (PRED_F / 2) + 1) : 1u;
}

cudaError_t launch_welch(const WelchBatch& b, int n_sm, cudaStream_t st)
{
    const uint32_t total = b.seg_begin[b.n];
    if (b.n == 0 || total == 0) return cudaSuccess;
    count_launches(2);
    k_welch_segments<<<std::min<uint32_t>(total, (uint32_t)n_sm), FT, FFT_SMEM, st>>>(b, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_welch_mean<<<dim3((PRED_BINS + 255) / 256, (unsigned)b.n), 256, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_template_power_dot(const float* rows, uint32_t n_rows, const float2* tw, const float* P,
                                      uint32_t n_ser, float* D, uint32_t d_stride, uint32_t row0, int n_sm,
                                      cudaStream_t st)
{
    if (n_rows == 0 || n_ser == 0) return cudaSuccess;
    count_launches(1);
    k_template_power_dot<<<std::min<uint32_t>(n_rows, (uint32_t)n_sm), FT, FFT_SMEM, st>>>(
        rows, n_rows, tw, P, n_ser, D, d_stride, row0);
    return cudaGetLastError();
}

cudaError_t launch_fft_series(const FftSeriesBatch& b, uint32_t total_segments, int n_sm, cudaStream_t st)
{
    if (total_segments == 0) return cudaSuccess;
    const unsigned grid = std::min<uint32_t>(total_segments, (uint32_t)n_sm);
    count_launches(1);
    if (b.quad) k_fft_series<false><<<grid, FT, FFT_SMEM, st>>>(b, total_segments);
    else k_fft_series<true><<<grid, FT, FFT_SMEM, st>>>(b, total_segments);
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
    const uint32_t items = p.quad ? (p.k_hi - p.k_lo + 1) / 2 : p.k_hi - p.k_lo;
    if (items == 0 || p.n_ser == 0) return cudaSuccess;
    const unsigned grid = std::min<unsigned>(items, (unsigned)n_sm);
    count_launches(1);
    bool dense = false;
    for (int i = 0; i < p.n_ser; ++i) dense = dense || p.ser[i].rho != nullptr;
    if (p.quad) {
        if (dense) k_corr_fft_quad<true><<<grid, FT, CORR_SMEM, st>>>(p);
        else k_corr_fft_quad<false><<<grid, FT, CORR_SMEM, st>>>(p);
    } else {
        if (dense) k_corr_rfft<true><<<grid, FT, RCORR_SMEM, st>>>(p);
        else k_corr_rfft<false><<<grid, FT, RCORR_SMEM, st>>>(p);
    }
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
// chunk by chunk (512 MiB of spectra: 8192 rows of the real route, 16384 of
// the pair route) into a two-slot ring on the auxiliary stream, and chunk c is
// correlated against every series batch on the main stream while chunk c+1 is
// made.  Events order the reuse of a slot after the launches that read it.
constexpr size_t FFT_CHUNK_BYTES = size_t(512) << 20;
constexpr size_t FFT_SYNTH_ROWS = 4096;

bf_status fft_ring_prepare(bf_ctx* ctx, const bf_bank* bank, uint32_t row_begin, uint32_t row_end,
                           std::vector<void*>& keep, FftRing* ring)
{
    const size_t bins = fft_spec_bins(bank->quad);
    const size_t n_rows = row_end - row_begin;
    ring->chunk = std::min(FFT_CHUNK_BYTES / (bins * sizeof(float2)), n_rows + (n_rows & 1));
    ring->n_chunks = (n_rows + ring->chunk - 1) / ring->chunk;
    ring->synth_rows = std::min(FFT_SYNTH_ROWS, ring->chunk + (ring->chunk & 1));    // even
    Allocator& mem = *ctx->mem;
    ring->scratch = static_cast<float*>(mem.alloc(ring->synth_rows * FN * sizeof(float)));
    if (ring->scratch) keep.push_back(ring->scratch);
    for (int i = 0; i < 2 && i < (int)ring->n_chunks; ++i) {
        ring->slot[i] = static_cast<float2*>(mem.alloc((ring->chunk + 2) * bins * sizeof(float2)));
        if (ring->slot[i]) keep.push_back(ring->slot[i]);
    }
    if (!ring->scratch || !ring->slot[0] || (ring->n_chunks > 1 && !ring->slot[1])) {
        set_error("out of device memory for the template-spectra ring");
        return BF_ENOMEM;
    }
    cudaError_t e = ring->ev.create();
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "ring events");
}

cudaError_t fft_correlate_chunked(bf_ctx* ctx, const bf_bank* bank, std::vector<FftParams>& batches,
                                  uint32_t row_begin, uint32_t row_end, const FftRing& ring,
                                  cudaStream_t st)
{
    const bool quad = bank->quad;
    const float2* tw = batches.empty() ? nullptr : batches[0].tw;
    const RingEvents& ev = ring.ev;
    cudaError_t e = cudaEventRecord(ev.start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux, ev.start, 0);
    for (size_t c = 0; c < ring.n_chunks && e == cudaSuccess; ++c) {
        const int sl = (int)(c & 1);
        const uint32_t c0 = row_begin + (uint32_t)(c * ring.chunk);
        const uint32_t c1 = (uint32_t)std::min<size_t>(c0 + ring.chunk, row_end);
        // the pair route makes the spectra of the even-aligned row pairs that a
        // stored bank uses, partner rows outside the slice included (each
        // spectrum carries its partner's rounding), so the outputs equal the
        // stored bank's; the real route makes one row per transform
        const uint32_t s0 = quad ? c0 & ~1u : c0;
        const uint32_t s1 = quad ? (uint32_t)std::min<size_t>((c1 + 1) & ~1u, bank->rows) : c1;
        if (c >= 2) e = cudaStreamWaitEvent(ctx->aux, ev.used[sl], 0);
        if (e == cudaSuccess)
            e = template_spectra(bank, s0, s1 - s0, ring.scratch, ring.synth_rows, tw, ring.slot[sl], ctx->n_sm,
                                 ctx->aux);
        if (e == cudaSuccess) e = cudaEventRecord(ev.made[sl], ctx->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev.made[sl], 0);
        for (FftParams& p : batches) {
            if (e != cudaSuccess) break;
            p.hspec = ring.slot[sl];
            p.hrow0 = s0;
            p.k_lo = c0;
            p.k_hi = c1;
            e = launch_corr_fft(p, ctx->n_sm, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev.used[sl], st);
    }
    return e;
}

}  // namespace bfi
