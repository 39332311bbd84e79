// Tensor-core correlation (tcgen05, TMEM accumulators, bulk-async copies) with
// the fused epilogue.  The sliding correlation of Sect. 2.1 is a dense
// contraction C[k, tau] = sum_m h_k[m] x[tau + m]; here it runs as an implicit
// GEMM with templates as the MMA M dimension (A operand, 128 per tile), lags
// as N (B operand, MMAs of N = 256; 512 or 256 lags per tile, see Geo) and
// template samples as K.
//
// The lag operand is a Hankel matrix, B[n][m] = x[lag0 + n + m].  It is never
// materialised: the series is kept as overlapping "split rows" (row w = the
// eight samples x[w .. w+7]; see prep.cu), so the 8x8 core matrix of lags
// n0..n0+7 and samples m0..m0+7 is row block (lag0 + n0 + m0) .. +7, i.e. 128
// contiguous bytes, and both descriptor strides (next 8 lags, next 8 samples)
// are 128 B.  One bulk copy of 568 rows stages a whole 512-lag x 64-sample
// block; the core matrices overlap in shared memory, which the MMA only reads.
//
// Precision: BF_BF16 issues one MMA (x_hi * h_hi); BF_SPLIT_BF16 and
// BF_SPLIT_FP16 issue three (x_hi h_hi + x_hi h_lo + x_lo h_hi), dropping only
// x_lo h_lo (relative size 2^-16 or less), into FP32 accumulators that take
// the K range in chunks (KRange / n_chunks below): the tensor core's own
// accumulation truncates, and the chunks are added with rounding to nearest.
//
// Warp roles (320 threads, one CTA per SM, persistent over tiles):
//   warp 0  producer: bulk copies of template and series blocks per stage
//   warp 1  allocates TMEM, one lane issues tcgen05.mma and commits
//   warps 2-9 epilogue: folds the K chunks of a tile, then tcgen05.ld of its
//            FP32 accumulator; two warps per TMEM lane quadrant, each thread
//            owning one template row and half of the lags: rho = C *
//            inv_norm, running max/argmax (ties to the smallest lag), sum of
//            rho^2, tails.  Four independent accumulator chains per thread
//            keep the ALU busy.  With 256-lag tiles the two TMEM buffers
//            alternate, so a tile's epilogue runs under the next tile's MMAs.
// Every mbarrier wait is bounded in time; on expiry the kernel records an
// error code in the status word, drains its own copies and MMAs, frees TMEM
// and returns.
#include "corr_common.cuh"

namespace bfi {

namespace {

constexpr uint32_t A_BYTES = TILE_BYTES_A;                   // 16384 B per k-block
constexpr uint32_t round1k(uint32_t b) { return (b + 1023u) & ~1023u; }

// Shared-memory and TMEM geometry of a tile of LT lags.  LT = 512: one
// accumulator of 512 columns (two N = 256 MMAs per step) fills TMEM, and the
// next tile's MMAs wait for the epilogue.  LT = 256: two accumulators of 256
// columns used alternately, so the epilogue of one tile overlaps the MMAs of
// the next, at twice the template-operand traffic per lag.
template <int LT>
struct Geo {
    static constexpr uint32_t NSUB = LT / 256;                 // N = 256 MMAs per step
    static constexpr uint32_t NBUF = 512 / LT;                 // accumulators in TMEM
    static constexpr uint32_t B_ROWS = LT + TC_BK - 8;         // split rows per stage
    static constexpr uint32_t B_BYTES = B_ROWS * 16;
    static constexpr uint32_t OFF_AHI = 0;
    static constexpr uint32_t OFF_ALO = A_BYTES;
    static constexpr uint32_t OFF_BHI = 2 * A_BYTES;
    static constexpr uint32_t OFF_BLO = 2 * A_BYTES + B_BYTES;
    static constexpr uint32_t STAGE_BYTES = round1k(2 * A_BYTES + 2 * B_BYTES);
    static constexpr uint32_t STAGES = LT == 512 ? 4 : 5;
    static constexpr uint32_t OFF_INV = STAGES * STAGE_BYTES;  // LT floats
    static constexpr uint32_t OFF_BAR = OFF_INV + LT * 4;
    static constexpr uint32_t N_BARS = 2 * STAGES + 2 * NBUF + 1;
    static constexpr uint32_t SMEM = OFF_BAR + N_BARS * 8 + 16 + 1024;   // + alignment slack
};
static_assert(Geo<512>::STAGE_BYTES == 51200, "stage layout");
static_assert(Geo<512>::SMEM <= 232448 && Geo<256>::SMEM <= 232448, "shared memory per CTA");
constexpr uint64_t TIMEOUT_NS = 10ull * 1000 * 1000 * 1000;
constexpr uint32_t TMEM_COLS = 512;

// instruction descriptors, kind::f16, D = F32, both operands K-major, N = 256,
// M = 128: A = B = BF16 (formats 1), or A = B = FP16 (formats 0)
constexpr uint32_t IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) |
                                ((128u >> 4) << 24);
constexpr uint32_t IDESC_F16 = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait.  Returns false on timeout or when another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          volatile int* abort_flag, bool honour_abort = true,
                                          uint64_t limit_ns = TIMEOUT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (honour_abort && *abort_flag) return false;
            if (globaltimer() - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                     // descriptor version (tcgen05)
    return d;                                   // base offset 0, no swizzle
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Issues a 32-lane x 32-column TMEM load; the registers are valid only after
// tmem_wait(r) (the load completes asynchronously).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}

// Waits for this thread's outstanding TMEM loads.  The registers of the load
// in flight are passed as read-write operands so that no use of them can be
// scheduled before the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// TMEM stores complete after tmem_st_wait().
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 64-column forms of the TMEM load and store, for the fold of a K chunk
__device__ __forceinline__ void tmem_ld64_async(uint32_t taddr, uint32_t (&r)[64])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait64(uint32_t (&r)[64])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]), "+r"(r[40]), "+r"(r[41]), "+r"(r[42]), "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]), "+r"(r[48]), "+r"(r[49]), "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]), "+r"(r[56]), "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_st64(uint32_t taddr, const uint32_t (&r)[64])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x64.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63,%64};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31]), "r"(r[32]), "r"(r[33]), "r"(r[34]), "r"(r[35]), "r"(r[36]), "r"(r[37]), "r"(r[38]), "r"(r[39]), "r"(r[40]), "r"(r[41]), "r"(r[42]), "r"(r[43]), "r"(r[44]), "r"(r[45]), "r"(r[46]), "r"(r[47]), "r"(r[48]), "r"(r[49]), "r"(r[50]), "r"(r[51]), "r"(r[52]), "r"(r[53]), "r"(r[54]), "r"(r[55]), "r"(r[56]), "r"(r[57]), "r"(r[58]), "r"(r[59]), "r"(r[60]), "r"(r[61]), "r"(r[62]), "r"(r[63])
                 : "memory");
}


constexpr uint32_t EPI_THREADS = TC_THREADS - 64;            // 256

// OR of a predicate over the epilogue threads (named barrier 1)
__device__ __forceinline__ bool epilogue_any(bool pred)
{
    uint32_t res;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(res)
        : "r"((uint32_t)pred), "n"(EPI_THREADS)
        : "memory");
    return res != 0;
}

__device__ __forceinline__ void epilogue_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
}

// running reductions of one template row over its lags, in 4 chains
struct EpiState {
    float bv[4];          // max |rho| per chain (-1: nothing seen)
    uint32_t bi[4];       // its column (first on ties within the chain)
    float ss[4];          // sum of rho^2
};

// 32 accumulator columns c0 .. c0+31 of one template row: running max/argmax
// and sum of squares; returns the largest |rho| of the chunk so that the tail
// test costs one branch per chunk.  DENSE also stores every rho.
template <bool FULL, bool DENSE>
__device__ __forceinline__ float epi_chunk(const uint32_t (&r)[32], const float* __restrict__ inv,
                                           uint32_t c0, uint32_t nvalid, EpiState& st,
                                           float* __restrict__ rho_row)
{
    float cmax = 0.f;
#pragma unroll
    for (uint32_t j4 = 0; j4 < 32; j4 += 4) {
        const float4 iv = *reinterpret_cast<const float4*>(inv + c0 + j4);
        const float ivs[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
        for (uint32_t u = 0; u < 4; ++u) {
            const uint32_t j = j4 + u;
            if (!FULL && c0 + j >= nvalid) continue;
            const float v = __uint_as_float(r[j]) * ivs[u];
            const float a = fabsf(v);
            if (a > st.bv[u]) {
                st.bv[u] = a;
                st.bi[u] = c0 + j;
            }
            st.ss[u] = fmaf(v, v, st.ss[u]);
            cmax = fmaxf(cmax, a);
            if (DENSE) rho_row[c0 + j] = v;
        }
    }
    return cmax;
}

// rare path: push every tail of a chunk whose largest |rho| reached thr
__device__ __forceinline__ void epi_tails(const uint32_t (&r)[32], const float* __restrict__ inv,
                                          uint32_t c0, uint32_t nvalid, float thr,
                                          const CorrParams& p, uint32_t series, uint32_t k,
                                          uint32_t lag0)
{
#pragma unroll
    for (uint32_t j = 0; j < 32; ++j) {     // unrolled: r stays in registers
        const float v = __uint_as_float(r[j]) * inv[c0 + j];
        if (c0 + j < nvalid && fabsf(v) >= thr) push_candidate(p, series, k, lag0 + c0 + j, v);
    }
}

// Quadrature banks: the rows of a pair (cosine, sine) sit in lanes 2i, 2i+1
// of a warp over the same 32 columns.  One exchange per column gives the even
// lane columns 0..15 and the odd lane columns 16..31 of both rows; each lane
// reduces the magnitude sqrt(c^2 + s^2) over its half.  q[] keeps the
// unnormalised magnitudes for the rare tail path.
template <bool FULL, bool DENSE>
__device__ __forceinline__ float epi_chunk_quad(const uint32_t (&r)[32], const float* __restrict__ inv,
                                                uint32_t c0, uint32_t nvalid, bool odd, EpiState& st,
                                                float* __restrict__ rho_row, float (&q)[16])
{
    const uint32_t cb = c0 + (odd ? 16u : 0u);
    float cmax = 0.f;
#pragma unroll
    for (uint32_t j = 0; j < 16; ++j) {
        const uint32_t send = odd ? r[j] : r[16 + j];
        const uint32_t recv = __shfl_xor_sync(0xffffffffu, send, 1);
        const float c = __uint_as_float(odd ? recv : r[j]);
        const float sn = __uint_as_float(odd ? r[16 + j] : recv);
        q[j] = sqrtf(c * c + sn * sn);
    }
#pragma unroll
    for (uint32_t j = 0; j < 16; ++j) {
        const uint32_t u = j & 3;
        if (!FULL && cb + j >= nvalid) continue;
        const float v = q[j] * inv[cb + j];
        if (v > st.bv[u]) {
            st.bv[u] = v;
            st.bi[u] = cb + j;
        }
        st.ss[u] = fmaf(v, v, st.ss[u]);
        cmax = fmaxf(cmax, v);
        if (DENSE) rho_row[cb + j] = v;
    }
    return cmax;
}

__device__ __forceinline__ void epi_tails_quad(const float (&q)[16], const float* __restrict__ inv,
                                               uint32_t cb, uint32_t nvalid, float thr,
                                               const CorrParams& p, uint32_t series, uint32_t chirp,
                                               uint32_t lag0)
{
#pragma unroll
    for (uint32_t j = 0; j < 16; ++j) {
        const float v = q[j] * inv[cb + j];
        if (cb + j < nvalid && v >= thr) push_candidate(p, series, chirp, lag0 + cb + j, v);
    }
}

__device__ __forceinline__ void record_error(int* err, int code)
{
    atomicCAS(err, 0, code);
}

struct TileCoord {
    const Seg* s;
    uint32_t tt, lag0;
};

// The K blocks of template tile tt that hold nonzero samples (all of them
// without a range table); the host guarantees lo < hi <= n_kb.  Skipped blocks
// are zero in every row of the tile, so the outputs are the full loop's.
struct KRange {
    uint32_t lo, hi;
};

__device__ __forceinline__ KRange k_range(const Seg& s, uint32_t tt, uint32_t n_kb)
{
    if (!s.tile_kb) return {0u, n_kb};
    const uint32_t r = s.tile_kb[tt];
    return {r & 0xffffu, min(r >> 16, n_kb)};
}

// K blocks (64 samples each) accumulated in one TMEM accumulator before the
// epilogue folds them into the tile's sum (2^p.kchunk_log2 blocks).  The
// tensor core adds each MMA's product sum to its FP32 accumulator with
// truncation, so each addition may lose part of an ulp of the running sum: on a
// matched window (rho near 1) the loss grows with the number of additions into
// one accumulator, about -5e-9 M at rho = 1 for M samples.  Chunks of C samples
// hold it near the loss of a C-sample template whatever M is (C = 2048 for
// split-BF16: about 1.1e-5; C = 1024 for split-FP16, whose loss per addition is
// larger: about 8e-6); the fold of the partial sums is one FP32 addition
// rounded to nearest.  Each fold stalls the MMAs for about 1.6K cycles: 0.6 %
// of the kernel at M = 4096 with C = 2048, 3-6 % with C = 1024.
//
// Chunks of a tile's K range [lo, hi) are its intersections with the aligned
// block ranges [c 2^k, (c + 1) 2^k), so that a tile whose range was narrowed to
// its templates' support adds the same partial sums as one that runs every
// block (the skipped blocks are zero).  The split routes only (a second
// accumulator is needed); plain BF16, whose operand rounding is far larger
// than the accumulation's, keeps one chunk, so its two tile shapes add in the
// same order.
template <int NPROD, uint32_t NBUF>
__device__ __forceinline__ uint32_t n_chunks(KRange kr, uint32_t lg)
{
    return NPROD == 3 && NBUF == 2 ? ((kr.hi - 1) >> lg) - (kr.lo >> lg) + 1 : 1u;
}

template <int NPROD, uint32_t NBUF>
__device__ __forceinline__ KRange chunk_range(KRange kr, uint32_t ch, uint32_t lg)
{
    if (!(NPROD == 3 && NBUF == 2)) return kr;
    const uint32_t a = ((kr.lo >> lg) + ch) << lg;
    return {max(kr.lo, a), min(kr.hi, a + (1u << lg))};
}

template <int LT>
__device__ __forceinline__ TileCoord tile_coord(const CorrParams& p, uint64_t t)
{
    const Seg* s = &p.seg[find_seg(p, t)];
    const uint64_t local = t - s->tile_begin;
    TileCoord c;
    c.s = s;
    c.tt = s->tt0 + (uint32_t)(local / s->n_lag_tiles);
    c.lag0 = (uint32_t)(local % s->n_lag_tiles) * LT;
    return c;
}

}  // namespace

template <int NPROD, int LT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_corr_tc(const __grid_constant__ CorrParams p)
{
    using G = Geo<LT>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* sh_inv = reinterpret_cast<float*>(sm + G::OFF_INV);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + G::OFF_BAR + G::N_BARS * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + G::OFF_BAR + G::N_BARS * 8 + 4);

    const uint32_t base = smem_u32(sm);
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](uint32_t st) { return bar0 + 8 * st; };
    auto empty_bar = [&](uint32_t st) { return bar0 + 8 * (G::STAGES + st); };
    auto tfull_bar = [&](uint32_t b) { return bar0 + 8 * (2 * G::STAGES + b); };
    auto tempty_bar = [&](uint32_t b) { return bar0 + 8 * (2 * G::STAGES + G::NBUF + b); };
    const uint32_t drain_bar = bar0 + 8 * (2 * G::STAGES + 2 * G::NBUF);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (uint32_t st = 0; st < G::STAGES; ++st) {
            mbar_init(full_bar(st), 1);
            mbar_init(empty_bar(st), 1);
        }
        for (uint32_t b = 0; b < G::NBUF; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), EPI_THREADS);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            uint64_t issued = 0;
            bool ok = true;
            for (uint64_t t = blockIdx.x; ok && t < p.total_tiles; t += gridDim.x) {
                const TileCoord c = tile_coord<LT>(p, t);
                const uint32_t n_kb = c.s->M_pad / TC_BK;
                const KRange kr = k_range(*c.s, c.tt, n_kb);
                const size_t tt_rel = c.tt - c.s->bank_k0 / TC_TILE_T;
                const uint8_t* a_hi = c.s->bank_hi + tt_rel * n_kb * A_BYTES;
                const uint8_t* a_lo = c.s->bank_lo + tt_rel * n_kb * A_BYTES;
                for (uint32_t kb = kr.lo; kb < kr.hi; ++kb) {
                    if (!mbar_wait(empty_bar(st), ph ^ 1, abort_flag)) {
                        if (!*abort_flag) record_error(p.err, DEV_TIMEOUT_EMPTY);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t sbase = base + st * G::STAGE_BYTES;
                    const uint32_t bytes = NPROD == 3 ? 2 * (A_BYTES + G::B_BYTES) : A_BYTES + G::B_BYTES;
                    mbar_expect_tx(full_bar(st), bytes);
                    const uint64_t w0 = (uint64_t)c.lag0 + (uint64_t)kb * TC_BK;
                    bulk_g2s(sbase + G::OFF_AHI, a_hi + (size_t)kb * A_BYTES, A_BYTES, full_bar(st));
                    bulk_g2s(sbase + G::OFF_BHI, c.s->yhi + w0, G::B_BYTES, full_bar(st));
                    if (NPROD == 3) {
                        bulk_g2s(sbase + G::OFF_ALO, a_lo + (size_t)kb * A_BYTES, A_BYTES, full_bar(st));
                        bulk_g2s(sbase + G::OFF_BLO, c.s->ylo + w0, G::B_BYTES, full_bar(st));
                    }
                    ++issued;
                    if (++st == G::STAGES) { st = 0; ph ^= 1; }
                }
            }
            if (!ok) {
                // let copies already in flight land before shared memory is released
                uint64_t first = issued > G::STAGES ? issued - G::STAGES : 0;
                for (uint64_t i = first; i < issued; ++i)
                    mbar_wait(full_bar((uint32_t)(i % G::STAGES)), (uint32_t)((i / G::STAGES) & 1),
                              abort_flag, false);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            uint32_t x = 0;             // the base accumulator of the next tile
            uint32_t mph = 0;           // bit b: phase of the waits on tempty[b]
            bool ok = true;
            for (uint64_t t = blockIdx.x; ok && t < p.total_tiles; t += gridDim.x) {
                const TileCoord c = tile_coord<LT>(p, t);
                const KRange kr = k_range(*c.s, c.tt, c.s->M_pad / TC_BK);
                const uint32_t n_ch = n_chunks<NPROD, G::NBUF>(kr, p.kchunk_log2);
                for (uint32_t ch = 0; ok && ch < n_ch; ++ch) {
                    // chunk 0 into the base accumulator, later chunks into the
                    // other one, which the epilogue folds into the base
                    const uint32_t b = ch == 0 ? x : x ^ 1u;
                    if (!mbar_wait(tempty_bar(b), ((mph >> b) & 1) ^ 1, abort_flag)) {
                        if (!*abort_flag) record_error(p.err, DEV_TIMEOUT_TMEM);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    mph ^= 1u << b;
                    fence_after();
                    const KRange cr = chunk_range<NPROD, G::NBUF>(kr, ch, p.kchunk_log2);
                    const uint32_t kb0 = cr.lo, kb1 = cr.hi;
                    for (uint32_t kb = kb0; kb < kb1; ++kb) {
                        if (!mbar_wait(full_bar(st), ph, abort_flag)) {
                            if (!*abort_flag) record_error(p.err, DEV_TIMEOUT_FULL);
                            *abort_flag = 1;
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t sbase = base + st * G::STAGE_BYTES;
#pragma unroll
                        for (uint32_t kk = 0; kk < TC_BK / 16; ++kk) {
                            const uint64_t ahi = make_desc(sbase + G::OFF_AHI + kk * 256, 128, 1024);
                            const uint64_t alo = make_desc(sbase + G::OFF_ALO + kk * 256, 128, 1024);
#pragma unroll
                            for (uint32_t h = 0; h < G::NSUB; ++h) {
                                const uint32_t boff = h * 256 * 16 + kk * 256;
                                const uint64_t bhi = make_desc(sbase + G::OFF_BHI + boff, 128, 128);
                                const uint64_t blo = make_desc(sbase + G::OFF_BLO + boff, 128, 128);
                                const uint32_t d = tmem + b * 256 + h * 256;
                                mma_f16(d, ahi, bhi, p.idesc, (kb != kb0) | (kk != 0));
                                if (NPROD == 3) {
                                    mma_f16(d, ahi, blo, p.idesc, 1);
                                    mma_f16(d, alo, bhi, p.idesc, 1);
                                }
                            }
                        }
                        mma_commit(empty_bar(st));
                        if (++st == G::STAGES) { st = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(tfull_bar(b));
                }
                if (G::NBUF == 2) x ^= 1u;      // the next tile's base is this tile's other one
            }
            // drain: every MMA issued by this thread completes before TMEM is freed
            mma_commit(drain_bar);
            mbar_wait(drain_bar, 0, abort_flag, false);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const uint32_t q = warp & 3;                       // TMEM lane quadrant
        const uint32_t half = (warp - 2) >> 2;             // columns [half LT/2, (half+1) LT/2)
        const uint32_t row = q * 32 + lane;                // template row of the tile
        const uint32_t e = threadIdx.x - 64;               // 0 .. EPI_THREADS-1
        uint32_t x = 0;                 // the base accumulator of this tile
        uint32_t eph = 0;               // bit b: phase of the waits on tfull[b]
        for (uint64_t t = blockIdx.x; t < p.total_tiles; t += gridDim.x) {
            const TileCoord c = tile_coord<LT>(p, t);
            const Seg& s = *c.s;
            const uint32_t nvalid = min((uint32_t)LT, s.L - c.lag0);
            // split-FP16 operands were scaled by 2^s (series) and 2^8 (templates)
            const float oscale = s.xmax ? ldexpf(1.f, -(f16_series_shift(*s.xmax) + 8)) : 1.f;
            epilogue_sync();
            for (uint32_t j = e; j < (uint32_t)LT; j += EPI_THREADS)
                sh_inv[j] = j < nvalid ? s.inv_norm[c.lag0 + j] * oscale : 0.f;
            epilogue_sync();
            static_assert((LT / 2) % 64 == 0, "chunk pairs per warp");
            const uint32_t cbeg = half * (LT / 2), cend = cbeg + LT / 2;
            uint32_t ra[32], rb[32];
            // chunk 0 of the K range is in the base accumulator x; each later
            // chunk arrives in the other one and is added into x here (FP32,
            // round to nearest), which frees it for the MMA warp
            const uint32_t n_ch = n_chunks<NPROD, G::NBUF>(k_range(s, c.tt, s.M_pad / TC_BK), p.kchunk_log2);
            bool ok = true;
            for (uint32_t ch = 0; ch < n_ch; ++ch) {
                const uint32_t b = ch == 0 ? x : x ^ 1u;
                ok = mbar_wait(tfull_bar(b), (eph >> b) & 1, abort_flag);
                eph ^= 1u << b;
                if (epilogue_any(!ok)) {   // all epilogue threads leave together
                    ok = false;
                    break;
                }
                fence_after();
                if (ch == 0) continue;
                const uint32_t tx = tmem + ((q * 32) << 16) + x * 256;
                const uint32_t ty = tmem + ((q * 32) << 16) + b * 256;
#pragma unroll 1
                for (uint32_t c0 = cbeg; c0 < cend; c0 += 64) {
                    uint32_t fx[64], fy[64];
                    __syncwarp();
                    tmem_ld64_async(tx + c0, fx);
                    tmem_ld64_async(ty + c0, fy);
                    tmem_wait64(fx);
                    tmem_wait64(fy);
#pragma unroll
                    for (int i = 0; i < 64; ++i)
                        fx[i] = __float_as_uint(__uint_as_float(fx[i]) + __uint_as_float(fy[i]));
                    tmem_st64(tx + c0, fx);
                }
                tmem_st_wait();
                fence_before();
                mbar_arrive(tempty_bar(b));
            }
            if (!ok) {
                if (!*abort_flag) record_error(p.err, DEV_TIMEOUT_TMEM);
                *abort_flag = 1;
                break;
            }
            const uint32_t buf = x;
            if (G::NBUF == 2) x ^= 1u;          // the next tile's base
            const uint32_t k = c.tt * TC_TILE_T + row;
            const bool keep = k >= s.k_begin && k < s.k_end;
            const bool full = nvalid == (uint32_t)LT;
            const bool quad = s.quad != 0, odd = (lane & 1) != 0;
            // output index: the row, or the quadrature pair of the row
            const uint32_t o = quad ? (k - s.k_begin) >> 1 : k - s.k_begin;
            float* const rho_row = (s.rho != nullptr && keep) ? s.rho + (size_t)o * s.L + c.lag0 : nullptr;
            const bool dense = rho_row != nullptr;
            const float thr = !keep ? INFINITY : (s.sigma_pred ? s.kappa * s.sigma_pred[o] : p.thr);
            const uint32_t series = s.series_id, lag0 = c.lag0;
            EpiState st;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                st.bv[u] = -1.f;
                st.bi[u] = 0;
                st.ss[u] = 0.f;
            }
            const uint32_t taddr = tmem + ((q * 32) << 16) + buf * 256;
            // software pipeline over the chunks of 32 columns: the load of
            // chunk i+1 is in flight while chunk i is reduced; the accumulator
            // is handed back to the MMA warp as soon as the last load has landed
            auto reduce = [&](const uint32_t (&r)[32], uint32_t cc) {
                if (cc >= nvalid) return;
                float cmax;
                if (quad) {
                    float q[16];
                    if (dense) cmax = epi_chunk_quad<false, true>(r, sh_inv, cc, nvalid, odd, st, rho_row, q);
                    else if (full) cmax = epi_chunk_quad<true, false>(r, sh_inv, cc, nvalid, odd, st, nullptr, q);
                    else cmax = epi_chunk_quad<false, false>(r, sh_inv, cc, nvalid, odd, st, nullptr, q);
                    if (cmax >= thr)
                        epi_tails_quad(q, sh_inv, cc + (odd ? 16u : 0u), nvalid, thr, p, series, k >> 1, lag0);
                    return;
                }
                if (dense) cmax = epi_chunk<false, true>(r, sh_inv, cc, nvalid, st, rho_row);
                else if (full) cmax = epi_chunk<true, false>(r, sh_inv, cc, nvalid, st, nullptr);
                else cmax = epi_chunk<false, false>(r, sh_inv, cc, nvalid, st, nullptr);
                if (cmax >= thr) epi_tails(r, sh_inv, cc, nvalid, thr, p, series, k, lag0);
            };
            __syncwarp();
            tmem_ld32_async(taddr + cbeg, ra);
            tmem_wait(ra);
#pragma unroll 1
            for (uint32_t c0 = cbeg; c0 < cend; c0 += 64) {
                __syncwarp();
                tmem_ld32_async(taddr + c0 + 32, rb);
                reduce(ra, c0);
                tmem_wait(rb);
                const bool more = c0 + 64 < cend;
                if (more) {
                    __syncwarp();
                    tmem_ld32_async(taddr + c0 + 64, ra);
                } else {
                    fence_before();
                    mbar_arrive(tempty_bar(buf));     // every column of this thread is read
                }
                reduce(rb, c0 + 32);
                if (more) tmem_wait(ra);
            }
            // merge the chains: largest |rho|, smallest column on ties
            float bv = st.bv[0];
            uint32_t bi = st.bi[0];
#pragma unroll
            for (int u = 1; u < 4; ++u)
                if (st.bv[u] > bv || (st.bv[u] == bv && st.bi[u] < bi)) {
                    bv = st.bv[u];
                    bi = st.bi[u];
                }
            float ssum = (st.ss[0] + st.ss[1]) + (st.ss[2] + st.ss[3]);
            if (quad) {
                // merge the two halves of the pair into the even lane
                const float obv = __shfl_xor_sync(0xffffffffu, bv, 1);
                const uint32_t obi = __shfl_xor_sync(0xffffffffu, bi, 1);
                ssum += __shfl_xor_sync(0xffffffffu, ssum, 1);
                if (obv > bv || (obv == bv && obi < bi)) {
                    bv = obv;
                    bi = obi;
                }
            }
            if (keep && bv >= 0.f && !(quad && odd) &&
                BF_BOUNDS(p.err, c.lag0 + bi < s.L && (size_t)c.tt * TC_TILE_T >= s.bank_k0)) {
                atomicMax(s.vmax + o, pack_max(bv, c.lag0 + bi));
                atomicAdd(s.sumsq + o, (double)ssum);
            }
        }
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

template <int NPROD, int LT>
static cudaError_t set_attr()
{
    return cudaFuncSetAttribute(k_corr_tc<NPROD, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Geo<LT>::SMEM);
}

static bool g_attr_done = false;

cudaError_t corr_tc_set_attributes()
{
    if (g_attr_done) return cudaSuccess;
    cudaError_t e = set_attr<1, 512>();
    if (e == cudaSuccess) e = set_attr<1, 256>();
    if (e == cudaSuccess) e = set_attr<3, 256>();
    if (e == cudaSuccess) g_attr_done = true;
    return e;
}

// Self-test of the bounded wait above: one mbarrier expecting one arrival,
// which thread 0 of warp 1 makes only when `signal` is set, and warp 0 waiting
// on it with the given limit.  A timeout is recorded in the status word as in
// the correlation kernel; waited[0] gets the nanoseconds spent waiting.
__global__ void k_wait_selftest(int* err, int signal, uint64_t limit_ns, unsigned long long* waited)
{
    __shared__ __align__(8) uint64_t bar_storage;
    __shared__ int abort_word;
    const uint32_t bar = smem_u32(&bar_storage);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        abort_word = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 32 && signal) mbar_arrive(bar);
    if (threadIdx.x == 0) {
        const uint64_t t0 = globaltimer();
        const bool ok = mbar_wait(bar, 0, reinterpret_cast<volatile int*>(&abort_word), true, limit_ns);
        *waited = globaltimer() - t0;
        if (!ok) record_error(err, DEV_TIMEOUT_FULL);
    }
}

cudaError_t launch_wait_selftest(int* err, int signal, uint64_t limit_ns, unsigned long long* waited,
                                 cudaStream_t st)
{
    count_launches(1);
    k_wait_selftest<<<1, 64, 0, st>>>(err, signal, limit_ns, waited);
    return cudaGetLastError();
}

uint32_t tc_idesc(int precision) { return precision == BF_SPLIT_FP16 ? IDESC_F16 : IDESC_BF16; }

cudaError_t launch_corr_tc(const CorrParams& p, int nprod, int lt, int n_sm, cudaStream_t st)
{
    if (p.total_tiles == 0) return cudaSuccess;
    cudaError_t ea = corr_tc_set_attributes();
    if (ea != cudaSuccess) return ea;
    const unsigned grid = (unsigned)(p.total_tiles < (uint64_t)n_sm ? p.total_tiles : (uint64_t)n_sm);
    count_launches(1);
    // the split routes need the second accumulator for their K chunks, so
    // they run the 256-lag shape only
    if (nprod == 3 && lt != 256) return cudaErrorInvalidValue;
    if (lt == 256) {
        if (nprod == 3) k_corr_tc<3, 256><<<grid, TC_THREADS, Geo<256>::SMEM, st>>>(p);
        else k_corr_tc<1, 256><<<grid, TC_THREADS, Geo<256>::SMEM, st>>>(p);
    } else {
        k_corr_tc<1, 512><<<grid, TC_THREADS, Geo<512>::SMEM, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace bfi
