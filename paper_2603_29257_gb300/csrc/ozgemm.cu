// FP64 GEMM by the Ozaki splitting scheme on tcgen05 (sm_103a), kind::f16
// with bf16 operands and FP32 accumulators in tensor memory.
//
// Splitting (per row r, exponent e = the row's largest binary exponent):
// Y = round(x * 2^(7 + 8(S-1) - e)) is an integer with |Y| <= 2^(7+8(S-1));
// its balanced base-256 digits q_0 (most significant) .. q_{S-1} lie in
// [-128, 128] and are exact in bf16.  All of it is integer arithmetic on the
// FP64 bit pattern.
//
// Slices are stored pre-scaled, q_s 2^(-8s) (exact in bf16).  Product: with A
// and B split the same way,
//   sum_k a_mk b_nk ~= 2^(eA_m + eB_n - 14) * sum_{d<S} P_d,
//   P_d = sum_k sum_{s+t=d} qA_s qB_t 2^(-8d)   (the terms s + t >= S are dropped).
// Each digit product is at most 2^14 in magnitude, so over a chunk of K with
// (d+1) * kc <= 1024 the sum P_d is an integer multiple of 2^(-8d) below
// 2^(24-8d): exact in FP32.  The kernel keeps one FP32 accumulator in tensor
// memory for each leading diagonal d < NE (NE = S for S <= 4, S - 2 above)
// and one shared accumulator for the remaining diagonals, whose FP32 rounding
// (2^-24 of a sum already scaled by 2^(-8 NE)) stays far below the slicing
// error; after each chunk every accumulator is added into a double-FP32
// (hi, lo) pair per output by error-free two-sums.
//
// CTA: 10 warps, a 128 x 64 output tile.  Warp 0 (one lane) streams the
// slices of 128 A rows and 64 B rows for one K block of 32 per stage with TMA
// (boxes of 64 bf16 = two slices, 128-byte swizzle) into a ring of shared
// memory; warp 1 (one lane) issues the S(S+1)/2 slice products per stage as
// tcgen05.mma (M = 128, N = 64, K = 16) into the S accumulators; warps 2..9
// drain the accumulators after each chunk (warp w reads TMEM lanes
// 32 (w mod 4) .. +31, half of the columns) and write the scaled FP64 tile at
// the end.  With S <= 4 the accumulators are double-buffered, so that draining
// one chunk overlaps the products of the next.  Every wait is bounded (about
// 1 s, or the launch's own limit): a timeout records an error code in *err and
// the CTA goes to its teardown, which waits (bounded) for its own copies and
// products in flight and always frees tensor memory.
#include "ozgemm.cuh"
#include "tcptx.cuh"

#include <algorithm>

namespace tr {
namespace {

using namespace ptx;

constexpr int OZ_TBYTES = 8 * 32 * 33 * 4;  // epilogue transpose buffers: 8 warps x 32 x 33 floats

constexpr int oz_stages(int stage)
{
    return 4 * stage + OZ_TBYTES + 1280 <= 227 * 1024 ? 4 : 3 * stage + OZ_TBYTES + 1280 <= 227 * 1024 ? 3 : 2;
}

template <int S, int BN>
struct OzCfg {
    static constexpr int SP = (S + 1) & ~1;            // slices per K block, padded to even
    static constexpr int NBOX = SP / 2;                // TMA boxes per operand per stage
    static constexpr int ABOX = 128 * 128;             // bytes: 128 rows x 128 B
    static constexpr int BBOX = BN * 128;
    static constexpr int STAGE = NBOX * (ABOX + BBOX);
    static constexpr int STAGES = oz_stages(STAGE);
    // exactly summed leading diagonals; the rest share one FP32 accumulator whose
    // rounding (2^-24 of sums scaled by 2^(-8 NE)) stays far below the slicing
    // error 2^(-8S) even after the cancellation of the AO-to-MO sums (~2^14)
    static constexpr int NE = S <= 4 ? S : S - 2;
    static constexpr int NACC = NE + (S > NE ? 1 : 0); // plus one shared tail accumulator
    static constexpr int CK = 1024 / NE / 32;          // K blocks per exactly summed chunk
    static constexpr int NC = BN / 2;                  // output columns per epilogue warp
    static constexpr int NBUF = 2 * NACC * BN <= 512 ? 2 : 1;  // accumulator sets in tensor memory
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + OZ_TBYTES + 1024 + 256;
    static_assert(S >= 2 && S <= OZ_MAX_SLICES, "slices");
    static_assert(NACC * BN <= 512, "tensor memory holds the accumulators");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(STAGES >= 2 && CK >= 1 && NC == 32, "pipeline");
};

struct OzArgs {
    long long ntiles;              // tiles: N tiles x M tiles x batch entries x K splits
    int ntn, ntm;
    int M, N, nkb;                 // K blocks contracted per tile (all splits)
    int n2, ksplit, kchunk;        // batch b = b1 * n2 + b2; split s covers K blocks [s kchunk, ...)
    int kbA, kbB;                  // first K block of A and of B
    long long a0, a1, a2, c0, c1, c2;
    long long rowsA, rowsB;
    const int *eA, *eB;
    double *d;                     // output (or the split partials)
    long long s1, s2, ldm, ldn;
    double alpha;
    int accumulate;                // d += (instead of =)
    int *err;
    long long wait;                // pipeline wait limit in SM cycles
    int stall;                     // test of the bounded waits: the producer issues no loads
    const int *klist, *kcount;     // block-sparse K per N tile (null: every block)
    int kld;
};

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}

// The FP64 value of a float scaled by 2^n, as a bit pattern built with integer
// work (the FP64 pipe of this GPU is narrow): exact for zero and for normal
// floats whose scaled exponent stays in the normal FP64 range (ok = true).
__device__ __forceinline__ unsigned long long f2d_bits(float f, int n, bool &ok)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xFF;
    const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
    const int e = (int)ex + (1023 - 127) + n;
    const bool zero = (b << 1) == 0;
    ok = zero || (ex != 0 && ex != 0xFF && e > 0 && e < 2047);
    return zero ? sgn : (sgn | ((unsigned long long)(unsigned)e << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29));
}

// (hi + lo) 2^n for the rare pairs f2d_bits cannot take (subnormal, infinite or
// out-of-range results): an out-of-line call, so that the common path carries
// none of its FP64 instructions
__device__ __noinline__ double oz_pair_slow(float hi, float lo, int n)
{
    return scalbn((double)hi + (double)lo, n);
}

// (hi + lo) 2^n rounded once to FP64: both floats scaled exactly on their bit
// patterns, then one FP64 addition (the same value as adding first and scaling
// after).  Called by all 32 lanes of a warp; the warp takes the slow path only
// if one of its lanes needs it.
__device__ __forceinline__ double pair_scaled(float hi, float lo, int n)
{
    bool oh, ol;
    const unsigned long long bh = f2d_bits(hi, n, oh), bl = f2d_bits(lo, n, ol);
    if (__all_sync(0xffffffffu, oh && ol)) return __longlong_as_double((long long)bh) + __longlong_as_double((long long)bl);
    return oz_pair_slow(hi, lo, n);
}

// (hi, lo) += b with Knuth's error-free two-sum of hi and b (round-to-nearest
// intrinsics: no contraction or reassociation)
__device__ __forceinline__ void two_sum(float &hi, float &lo, float b)
{
    const float s = __fadd_rn(hi, b);
    const float bp = __fsub_rn(s, hi);
    const float ap = __fsub_rn(s, bp);
    const float err = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(b, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// Tile t of a persistent CTA: its output block, operand rows and K blocks
struct OzTile {
    int m0, n0, nt, split, b, b1, b2, kb_begin, nkb;
    long long arow, brow;
};

__device__ __forceinline__ OzTile oz_tile(const OzArgs &g, long long t, int BN)
{
    OzTile u;
    const int nt = (int)(t % g.ntn);
    const long long r = t / g.ntn;
    const int mt = (int)(r % g.ntm);
    const long long z = r / g.ntm;
    u.split = (int)(z % g.ksplit);
    u.b = (int)(z / g.ksplit);
    u.b1 = u.b / g.n2;
    u.b2 = u.b - u.b1 * g.n2;
    u.m0 = mt * 128;
    u.n0 = nt * BN;
    u.arow = g.a0 + g.a1 * u.b1 + g.a2 * u.b2 + u.m0;
    u.brow = g.c0 + g.c1 * u.b1 + g.c2 * u.b2 + u.n0;
    u.nt = nt;
    u.kb_begin = u.split * g.kchunk;
    u.nkb = g.kcount ? __ldg(g.kcount + nt) : max(0, min(g.nkb - u.kb_begin, g.kchunk));
    return u;
}

// One output element: MODE 0 stores v, 1 stores v alpha, 2 adds v, 3 adds v alpha
// (a separate instantiation per mode, so that no FP64 work of another mode is issued)
template <int MODE>
__device__ __forceinline__ void oz_put(double *o, double v, double alpha)
{
    if constexpr (MODE == 0) *o = v;
    else if constexpr (MODE == 1) *o = v * alpha;
    else if constexpr (MODE == 2) *o = *o + v;
    else *o = *o + v * alpha;
}

// Write of one epilogue warp's 32 x NC part of a tile: the double-FP32 sums
// (hi, lo) of its TMEM lanes (rows 32 quarter + lane) and columns
// half NC .. +NC, scaled by 2^(eA[row] + eB[col] - 14).  ldm == 1: lanes own
// consecutive output rows and write directly; otherwise the 32 x 32 block goes
// through the warp's float buffer (hi, then lo) so that lanes walk columns.
template <int MODE, int NC>
__device__ __forceinline__ void oz_write_tile(const OzArgs &g, const OzTile &u, const float (&hi)[NC],
                                              const float (&lo)[NC], float *fb, int quarter, int half, int lane,
                                              int ea, double *out, long long ldm, long long ldn, double alpha)
{
    if (ldm == 1) {
        const int rw = u.m0 + 32 * quarter + lane;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const int col = u.n0 + half * NC + j;
            const long long rb = u.brow + half * NC + j;
            const bool cok = col < g.N && rb < g.rowsB;
            const int eb = cok ? g.eB[rb] : 0;
            const double v = pair_scaled(hi[j], lo[j], ea - 14 + eb);
            if (rw < g.M && cok) oz_put<MODE>(out + (long long)rw + (long long)col * ldn, v, alpha);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) fb[lane * 33 + j] = hi[j];
    __syncwarp();
    float th[32];
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) th[rr] = fb[rr * 33 + lane];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) fb[lane * 33 + j] = lo[j];
    __syncwarp();
    const int col = u.n0 + half * NC + lane;
    const long long rb = u.brow + half * NC + lane;
    const bool cok = col < g.N && rb < g.rowsB;
    const int eb = cok ? g.eB[rb] - 14 : 0;
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) {
        const int er = __shfl_sync(0xffffffffu, ea, rr);
        const int rw = u.m0 + 32 * quarter + rr;
        const double v = pair_scaled(th[rr], fb[rr * 33 + lane], er + eb);
        if (rw < g.M && cok) oz_put<MODE>(out + (long long)rw * ldm + (long long)col * ldn, v, alpha);
    }
    __syncwarp();
}

// Persistent: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
// stage, chunk and barrier-phase counters run on across tiles, so that the
// epilogue of one tile (drained to registers, then written) overlaps the
// products of the next.
template <int S, int BN>
__global__ void __launch_bounds__(320, 1)
    oz_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, const OzArgs g)
{
    using C = OzCfg<S, BN>;
    constexpr int ST = C::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *tbuf = (float *)(smem + ST * C::STAGE);
    // barriers: full[ST], empty[ST], acc_full[NBUF], acc_empty[NBUF], drain
    uint64_t *bars = (uint64_t *)(smem + ST * C::STAGE + OZ_TBYTES);
    uint32_t *tslot = (uint32_t *)(bars + 2 * ST + 2 * C::NBUF + 1);
    const uint32_t FULL = sa(&bars[0]), EMPTY = sa(&bars[ST]);
    const uint32_t ACCF = sa(&bars[2 * ST]), ACCE = sa(&bars[2 * ST + C::NBUF]);
    const uint32_t DRAIN = sa(&bars[2 * ST + 2 * C::NBUF]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ntiles = g.ntiles;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * ST + C::NBUF; ++i) bar_init(sa(&bars[i]), 1);
        for (int i = 0; i < C::NBUF; ++i) bar_init(ACCE + 8 * i, 8);  // one arrival per epilogue warp
        bar_init(DRAIN, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tslot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            long long gk = 0;
            bool ok = !g.stall;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const OzTile u = oz_tile(g, t, BN);
                for (int kt = 0; kt < u.nkb; ++kt) {
                    const int s = (int)(gk % ST);
                    if (gk >= ST && !bar_wait(EMPTY + 8 * s, (uint32_t)(((gk / ST) - 1) & 1), g.err, 11, g.wait)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = FULL + 8 * s;
                    bar_expect(full, C::STAGE);
                    uint8_t *stg = smem + s * C::STAGE;
                    const int kb = g.klist ? __ldg(g.klist + (long long)u.nt * g.kld + kt) : u.kb_begin + kt;
                    const int xa = (g.kbA + kb) * C::SP * 32, xb = (g.kbB + kb) * C::SP * 32;
#pragma unroll
                    for (int j = 0; j < C::NBOX; ++j) {
                        tma2d(sa(stg + j * C::ABOX), &tA, xa + 64 * j, (int)u.arow, full);
                        tma2d(sa(stg + C::NBOX * C::ABOX + j * C::BBOX), &tB, xb + 64 * j, (int)u.brow, full);
                    }
                    ++gk;
                }
            }
            // copies still in flight complete before the CTA ends
            for (long long q = gk > ST ? gk - ST : 0; q < gk; ++q)
                bar_wait(FULL + 8 * (int)(q % ST), (uint32_t)((q / ST) & 1), g.err, 15);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, both
            // K-major, N = BN, M = 128
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            long long gk = 0, gch = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const OzTile u = oz_tile(g, t, BN);
                for (int kt = 0; kt < u.nkb; ++kt) {
                    const int s = (int)(gk % ST), kc = kt % C::CK, buf = (int)(gch % C::NBUF);
                    if (kc == 0 && gch >= C::NBUF) {
                        // the epilogue has drained the chunk that last used this accumulator set
                        if (!bar_wait(ACCE + 8 * buf, (uint32_t)(((gch / C::NBUF) - 1) & 1), g.err, 12, g.wait)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                    }
                    if (!bar_wait(FULL + 8 * s, (uint32_t)((gk / ST) & 1), g.err, 13, g.wait)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    uint8_t *stg = smem + s * C::STAGE;
                    const uint32_t abase = sa(stg), bbase = sa(stg + C::NBOX * C::ABOX);
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        // slice i of A: box i/2, byte offset 64 (i odd) inside the 128-byte row
                        const uint64_t dA = smem_desc(abase + (i >> 1) * C::ABOX) + 4 * (i & 1);
#pragma unroll
                        for (int tt = 0; tt + i < S; ++tt) {
                            const uint64_t dB = smem_desc(bbase + (tt >> 1) * C::BBOX) + 4 * (tt & 1);
                            const int ai = i + tt < C::NE ? i + tt : C::NE;  // accumulator of diagonal i + tt
                            const uint32_t acc = tmem + (uint32_t)((buf * C::NACC + ai) * BN);
                            // the first product into an accumulator in a chunk overwrites it:
                            // (0, d) for d < NE and (0, NE) for the tail
                            const bool first = kc == 0 && i == 0 && tt <= C::NE;
#pragma unroll
                            for (int h = 0; h < 2; ++h)
                                mma_bf16(acc, dA + 2 * h, dB + 2 * h, idesc, (first && h == 0) ? 0u : 1u);
                        }
                    }
                    commit(EMPTY + 8 * s);
                    ++gk;
                    if (kc == C::CK - 1 || kt == u.nkb - 1) {
                        commit(ACCF + 8 * buf);
                        ++gch;
                    }
                }
            }
            // every product issued has completed before tensor memory is freed, also
            // when a wait gave up and the epilogue no longer consumes them
            commit(DRAIN);
            bar_wait(DRAIN, 0, g.err, 16);
        }
        __syncwarp();
    } else {
        const int ew = warp - 2;        // 0..7
        const int quarter = warp & 3;   // TMEM lanes this warp may read
        const int half = ew >> 2;       // column half
        float *fb = tbuf + ew * 32 * 33;
        long long gch = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const OzTile u = oz_tile(g, t, BN);
            const int nch = (u.nkb + C::CK - 1) / C::CK;
            float hi[C::NC], lo[C::NC];
#pragma unroll
            for (int j = 0; j < C::NC; ++j) hi[j] = lo[j] = 0.f;
            for (int ch = 0; ch < nch; ++ch) {
                const int buf = (int)(gch % C::NBUF);
                if (!bar_wait(ACCF + 8 * buf, (uint32_t)((gch / C::NBUF) & 1), g.err, 14, g.wait)) {
                    ok = false;
                    break;
                }
                fence_after();
#pragma unroll
                for (int ai = 0; ai < C::NACC; ++ai) {
                    uint32_t r[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)((buf * C::NACC + ai) * BN + half * C::NC),
                              r);
#pragma unroll
                    for (int j = 0; j < 32; ++j) two_sum(hi[j], lo[j], __uint_as_float(r[j]));
                }
                fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(ACCE + 8 * buf);
                ++gch;
            }
            if (!ok) break;
            // tile write: the accumulators are in registers, tensor memory already
            // belongs to the next tile's products
            const int rl = 32 * quarter + lane;
            const long long ra = u.arow + rl;
            const int ea = (u.m0 + rl < g.M && ra < g.rowsA) ? g.eA[ra] : 0;
            double *out;
            long long ldm, ldn;
            double alpha;
            int acc;
            if (g.ksplit > 1) {  // split partials: [split][b][M][N] row-major, unscaled by alpha, stored
                const long long nb = g.ntiles / ((long long)g.ntn * g.ntm * g.ksplit);
                out = g.d + ((long long)u.split * nb + u.b) * (long long)g.M * g.N;
                ldm = g.N;
                ldn = 1;
                alpha = 1.0;
                acc = 0;
            } else {
                out = g.d + g.s1 * u.b1 + g.s2 * u.b2;
                ldm = g.ldm;
                ldn = g.ldn;
                alpha = g.alpha;
                acc = g.accumulate;
            }
            const int mode = (acc ? 2 : 0) + (alpha == 1.0 ? 0 : 1);
            switch (mode) {
                case 0: oz_write_tile<0, C::NC>(g, u, hi, lo, fb, quarter, half, lane, ea, out, ldm, ldn, alpha); break;
                case 1: oz_write_tile<1, C::NC>(g, u, hi, lo, fb, quarter, half, lane, ea, out, ldm, ldn, alpha); break;
                case 2: oz_write_tile<2, C::NC>(g, u, hi, lo, fb, quarter, half, lane, ea, out, ldm, ldn, alpha); break;
                default: oz_write_tile<3, C::NC>(g, u, hi, lo, fb, quarter, half, lane, ea, out, ldm, ldn, alpha); break;
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------- splitting

// e[r] = largest biased binary exponent field of row r (e zeroed beforehand):
// one warp per segment of 1024 values, combined by atomicMax, so that a few long
// rows still fill the GPU
constexpr int OZ_SEG = 1024;

// bmask (optional): K block kb of row r is read only where
// bmask[((r % mrows) / 64) * mld + kb] is set (the others hold zeros)
__global__ void oz_rowexp(const double *__restrict__ x, long long rows, int K, long long sr, long long sk,
                          int *__restrict__ e, const unsigned char *__restrict__ bmask, long long mrows, int mld)
{
    const int lane = threadIdx.x & 31;
    const int nseg = (K + OZ_SEG - 1) / OZ_SEG;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); t < rows * nseg; t += nw) {
        const long long r = t / nseg;
        const int k0 = (int)(t - r * nseg) * OZ_SEG, k1 = min(K, k0 + OZ_SEG);
        int mx = 0;
        const unsigned char *mk = bmask ? bmask + ((r % mrows) / 64) * mld : nullptr;
        for (int k = k0 + lane; k < k1; k += 32) {
            if (mk && !mk[k >> 5]) continue;  // the same block for the whole warp
            const long long bits = __double_as_longlong(x[r * sr + (long long)k * sk]);
            mx = max(mx, (int)((bits >> 52) & 0x7FF));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx > 0) atomicMax(e + r, mx);
    }
}

// biased exponent field -> frexp exponent (|x| < 2^e); 0 for a zero row
__global__ void oz_rowexp_finish(int *__restrict__ e, long long rows)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
        e[r] = e[r] ? e[r] - 1022 : 0;
}

// balanced base-256 digits of round(x * 2^(7 + 8(S-1) - e)), most significant first
template <int S>
__device__ __forceinline__ void oz_digits(double x, int e, int (&q)[S])
{
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    long long Y = 0;
    if (ex != 0) {  // zero and subnormal inputs give zero digits
        const long long M = (bits & ((1LL << 52) - 1)) | (1LL << 52);
        // x = +-M 2^(ex - 1075); |x| < 2^e keeps sh <= 2 (S <= 7)
        const int sh = ex - 1075 + 7 + 8 * (S - 1) - e;
        if (sh >= 0) Y = M << sh;
        else if (sh > -63) Y = (M + (1LL << (-sh - 1))) >> (-sh);
        if (bits < 0) Y = -Y;
    }
#pragma unroll
    for (int s = S - 1; s > 0; --s) {
        const int dgt = (int)((Y + 128) & 255) - 128;
        q[s] = dgt;
        Y = (Y - dgt) >> 8;
    }
    q[0] = (int)Y;
}

template <int S>
__global__ void oz_slice(const double *__restrict__ x, long long rows, int K, long long sr, long long sk,
                         const int *__restrict__ e, int nkb, int SP, long long L, uint16_t *__restrict__ q,
                         const unsigned char *__restrict__ bmask, long long mrows, int mld)
{
    const long long tot = rows * nkb * 32;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / (nkb * 32);
        const int rem = (int)(t - r * nkb * 32);
        const int kb = rem >> 5, kl = rem & 31, k = kb * 32 + kl;
        if (bmask && !bmask[((r % mrows) / 64) * mld + kb]) continue;  // a block no product reads
        int dg[S];
        if (k < K) {
            oz_digits<S>(x[r * sr + (long long)k * sk], e[r], dg);
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) dg[s] = 0;
        }
        uint16_t *o = q + r * L + (long long)kb * SP * 32 + kl;
#pragma unroll
        for (int s = 0; s < S; ++s)  // |digit| <= 128 times 2^(-8s): the upper half of its FP32 pattern is the exact bf16
            o[s * 32] = (uint16_t)(__float_as_uint((float)dg[s] * __int_as_float((127 - 8 * s) << 23)) >> 16);
        for (int s = S; s < SP; ++s) o[s * 32] = 0;
    }
}

// Many short rows: one block per row finds the row's exponent and slices it in
// the same pass (the row is re-read from L2), with the block mask as in oz_slice
template <int S>
__global__ void __launch_bounds__(256)
    oz_split_rowwise(const double *__restrict__ x, long long rows, int K, long long sr, long long sk,
                     int *__restrict__ e, int nkb, int SP, long long L, uint16_t *__restrict__ q,
                     const unsigned char *__restrict__ bmask, long long mrows, int mld)
{
    __shared__ int wmax[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const unsigned char *mk = bmask ? bmask + ((r % mrows) / 64) * mld : nullptr;
        const double *xr = x + r * sr;
        int mx = 0;
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            if (mk && !mk[k >> 5]) continue;
            mx = max(mx, (int)((__double_as_longlong(xr[(long long)k * sk]) >> 52) & 0x7FF));
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) wmax[warp] = mx;
        __syncthreads();
        mx = wmax[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) mx = max(mx, wmax[w]);
        const int er = mx ? mx - 1022 : 0;  // biased exponent field -> frexp exponent; 0 for a zero row
        if (threadIdx.x == 0) e[r] = er;
        // two neighbouring K values per thread: each slice is one 32-bit store
        // of two bf16 (row storage is 256-byte aligned, kl even)
        uint32_t *qr = (uint32_t *)(q + r * L);
        for (int t = threadIdx.x; t < nkb * 16; t += blockDim.x) {
            const int kb = t >> 4, kl = (t & 15) * 2, k = kb * 32 + kl;
            if (mk && !mk[kb]) continue;  // a block no product reads
            int d0[S], d1[S];
            if (k < K) {
                oz_digits<S>(xr[(long long)k * sk], er, d0);
            } else {
#pragma unroll
                for (int s2 = 0; s2 < S; ++s2) d0[s2] = 0;
            }
            if (k + 1 < K) {
                oz_digits<S>(xr[(long long)(k + 1) * sk], er, d1);
            } else {
#pragma unroll
                for (int s2 = 0; s2 < S; ++s2) d1[s2] = 0;
            }
            uint32_t *o = qr + ((long long)kb * SP * 32 + kl) / 2;
#pragma unroll
            for (int s2 = 0; s2 < S; ++s2) {
                const float w = __int_as_float((127 - 8 * s2) << 23);
                const uint32_t lo = __float_as_uint((float)d0[s2] * w) >> 16, hi = __float_as_uint((float)d1[s2] * w) >> 16;
                o[s2 * 16] = lo | (hi << 16);
            }
            for (int s2 = S; s2 < SP; ++s2) o[s2 * 16] = 0u;
        }
        __syncthreads();  // wmax is rewritten for the next row
    }
}

// d[s1 b1 + s2 b2 + r ldm + c ldn] (+)= alpha * sum over splits of ws[split][b][r][c]
__global__ void oz_split_reduce(const double *__restrict__ ws, int ksplit, int nb, int n2, int M, int N, double *d,
                                long long s1, long long s2, long long ldm, long long ldn, double alpha, int acc)
{
    const long long per = (long long)M * N, tot = (long long)nb * per;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const long long b = t / per, rc = t - b * per;
        const int r = (int)(rc / N), cc = (int)(rc - (long long)r * N);
        double sum = 0.0;
        for (int sp = 0; sp < ksplit; ++sp) sum += ws[((long long)sp * nb + b) * per + rc];
        const long long b1 = b / n2, b2 = b - b1 * n2;
        double *o = d + s1 * b1 + s2 * b2 + (long long)r * ldm + (long long)cc * ldn;
        *o = acc ? *o + alpha * sum : alpha * sum;
    }
}

// columns k0 .. k0+p of a sliced matrix whose rows are the source columns:
// element (r, k0 + j) = src[j * ld + r], with the row exponents already in e
template <int S>
__global__ void oz_slice_cols(const double *__restrict__ src, long long ld, long long rows, int k0, int p,
                              const int *__restrict__ e, int SP, long long L, uint16_t *__restrict__ q)
{
    const long long tot = rows * p;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / p;
        const int j = (int)(t - r * p), k = k0 + j;
        int dg[S];
        oz_digits<S>(src[(long long)j * ld + r], e[r], dg);
        uint16_t *o = q + r * L + (long long)(k >> 5) * SP * 32 + (k & 31);
#pragma unroll
        for (int s = 0; s < S; ++s)
            o[s * 32] = (uint16_t)(__float_as_uint((float)dg[s] * __int_as_float((127 - 8 * s) << 23)) >> 16);
    }
}

__global__ void fill_int(int *__restrict__ p, long long n, int v)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        p[t] = v;
}

template <int S, int BN>
void oz_launch(cudaStream_t st, dim3 grid, const OzMat &A, const OzMat &B, const OzArgs &g)
{
    using C = OzCfg<S, BN>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(oz_kernel<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    TR_CUDA(attr);
    oz_kernel<S, BN><<<grid, 320, C::SMEM, st>>>(A.m128, BN == 64 ? B.m64 : B.m128, g);
}

template <int S>
void oz_slice_launch(cudaStream_t st, const double *x, long long sr, long long sk, OzMat &m, unsigned blocks,
                     const unsigned char *bmask, long long mrows, int mld)
{
    oz_slice<S><<<blocks, 256, 0, st>>>(x, m.rows, m.K, sr, sk, m.e, m.nkb, m.SP, m.L, m.q, bmask, mrows, mld);
}

long long row_len(int K, int S) { return (long long)cdiv(K, 32) * (((S + 1) & ~1) * 32); }

}  // namespace

size_t oz_bytes(long long rows, int K, int S)
{
    const size_t qb = (size_t)rows * row_len(K, S) * 2;
    return ((qb + 255) & ~(size_t)255) + (((size_t)rows * 4 + 255) & ~(size_t)255);
}

void oz_bind(OzMat &m, void *storage, long long rows, int K, int S)
{
    TR_REQUIRE(S >= 2 && S <= OZ_MAX_SLICES, TR_EINVAL, "Ozaki split: slices must be 2..7");
    TR_REQUIRE(rows > 0 && rows < (1LL << 31) && K > 0, TR_EINVAL, "Ozaki split: bad shape");
    TR_REQUIRE(((uintptr_t)storage % 256) == 0, TR_EINVAL, "Ozaki split: storage must be 256-byte aligned");
    m.rows = rows;
    m.K = K;
    m.S = S;
    m.SP = (S + 1) & ~1;
    m.nkb = cdiv(K, 32);
    m.L = row_len(K, S);
    m.q = (uint16_t *)storage;
    const size_t qb = (size_t)rows * m.L * 2;
    m.e = (int *)((uint8_t *)storage + ((qb + 255) & ~(size_t)255));
    tma_encode_2d(m.m128, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m.q, rows, m.L, m.L * 2, 64, 128);
    tma_encode_2d(m.m64, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m.q, rows, m.L, m.L * 2, 64, 64);
}

void oz_split(Prof &prof, cudaStream_t st, const char *name, const double *x, long long sr, long long sk, OzMat &m,
              const unsigned char *bmask, long long mrows, int mld)
{
    TR_REQUIRE(m.q && m.e, TR_EINVAL, "Ozaki split: unbound operand");
    TR_REQUIRE(!bmask || (mrows >= 1 && mld >= m.nkb), TR_EINVAL, "Ozaki split: bad block mask");
    if (m.rows >= 152LL * 8 && m.K <= 16384) {
        // many short rows (integral and half-transform chunks): one fused pass
        const unsigned blocks = (unsigned)std::min<long long>(m.rows, 152LL * 8);
        int tok = prof.begin(st, name, 0, 8.0 * m.rows * m.K + 2.0 * m.rows * m.L);
        switch (m.S) {
#define TR_OZR(SS) \
    case SS: oz_split_rowwise<SS><<<blocks, 256, 0, st>>>(x, m.rows, m.K, sr, sk, m.e, m.nkb, m.SP, m.L, m.q, bmask, mrows, mld); break;
        TR_OZR(2) TR_OZR(3) TR_OZR(4) TR_OZR(5) TR_OZR(6)
        default: oz_split_rowwise<7><<<blocks, 256, 0, st>>>(x, m.rows, m.K, sr, sk, m.e, m.nkb, m.SP, m.L, m.q, bmask,
                                                             mrows, mld);
            break;
#undef TR_OZR
        }
        TR_CHECK_LAUNCH(name);
        prof.end(st, tok);
        return;
    }
    const long long nwarps = m.rows * cdiv(m.K, OZ_SEG);
    const unsigned rb = (unsigned)std::min<long long>(cdiv(nwarps, 8), 152LL * 32);
    TR_CUDA(cudaMemsetAsync(m.e, 0, sizeof(int) * m.rows, st));
    TR_LAUNCH(prof, st, "oz_rowexp", 0, 8.0 * m.rows * m.K,
              oz_rowexp<<<rb, 256, 0, st>>>(x, m.rows, m.K, sr, sk, m.e, bmask, mrows, mld));
    oz_rowexp_finish<<<(unsigned)std::min<long long>(cdiv(m.rows, 256), 152LL * 8), 256, 0, st>>>(m.e, m.rows);
    const long long tot = m.rows * m.nkb * 32;
    const unsigned blocks = (unsigned)std::min<long long>(cdiv(tot, 256), 152LL * 16);
    int tok = prof.begin(st, name, 0, 8.0 * m.rows * m.K + 2.0 * m.rows * m.L);
    switch (m.S) {
    case 2: oz_slice_launch<2>(st, x, sr, sk, m, blocks, bmask, mrows, mld); break;
    case 3: oz_slice_launch<3>(st, x, sr, sk, m, blocks, bmask, mrows, mld); break;
    case 4: oz_slice_launch<4>(st, x, sr, sk, m, blocks, bmask, mrows, mld); break;
    case 5: oz_slice_launch<5>(st, x, sr, sk, m, blocks, bmask, mrows, mld); break;
    case 6: oz_slice_launch<6>(st, x, sr, sk, m, blocks, bmask, mrows, mld); break;
    default: oz_slice_launch<7>(st, x, sr, sk, m, blocks, bmask, mrows, mld); break;
    }
    TR_CHECK_LAUNCH(name);
    prof.end(st, tok);
}

// Fixed exponent for a matrix sliced by columns whose range is learnt from its
// first rows: e_new = max(row exponents of the first block) + margin; later
// blocks must stay below 2^e (else *bad = code).
__global__ void oz_col_exponent(const int *__restrict__ row_e, int p, int first, int margin, int *__restrict__ e_fixed,
                                int *__restrict__ bad, int code)
{
    int mx = -100000;
    for (int i = threadIdx.x; i < p; i += 32) mx = max(mx, row_e[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) {
        if (first) *e_fixed = mx + margin;
        else if (mx > *e_fixed) atomicCAS(bad, 0, code);
    }
}

__global__ void fill_int_from(int *__restrict__ p, long long n, const int *__restrict__ v)
{
    const int x = *v;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        p[t] = x;
}

void oz_col_exponent_update(cudaStream_t st, const int *row_e, int p, bool first, int margin, OzMat &m, int *e_fixed,
                            int *bad, int code)
{
    oz_col_exponent<<<1, 32, 0, st>>>(row_e, p, first ? 1 : 0, margin, e_fixed, bad, code);
    TR_CHECK_LAUNCH("oz_col_exponent");
    if (first) {
        const unsigned blocks = (unsigned)std::min<long long>(cdiv(m.rows, 256), 152LL * 8);
        fill_int_from<<<blocks, 256, 0, st>>>(m.e, m.rows, e_fixed);
        TR_CHECK_LAUNCH("fill_int_from");
    }
}

void oz_set_exponents(cudaStream_t st, OzMat &m, int e)
{
    const unsigned blocks = (unsigned)std::min<long long>(cdiv(m.rows, 256), 152LL * 8);
    fill_int<<<blocks, 256, 0, st>>>(m.e, m.rows, e);
    TR_CHECK_LAUNCH("fill_int");
}

void oz_split_cols_fixed(Prof &prof, cudaStream_t st, const char *name, const double *src, long long ld, OzMat &m,
                         int k0, int p)
{
    TR_REQUIRE(k0 >= 0 && p >= 0 && k0 + p <= m.K, TR_EINVAL, "Ozaki split: column range out of bounds");
    if (p == 0) return;
    const long long tot = m.rows * p;
    const unsigned blocks = (unsigned)std::min<long long>(cdiv(tot, 256), 152LL * 16);
    int tok = prof.begin(st, name, 0, 8.0 * tot + 2.0 * m.SP * tot);
    switch (m.S) {
    case 2: oz_slice_cols<2><<<blocks, 256, 0, st>>>(src, ld, m.rows, k0, p, m.e, m.SP, m.L, m.q); break;
    case 3: oz_slice_cols<3><<<blocks, 256, 0, st>>>(src, ld, m.rows, k0, p, m.e, m.SP, m.L, m.q); break;
    case 4: oz_slice_cols<4><<<blocks, 256, 0, st>>>(src, ld, m.rows, k0, p, m.e, m.SP, m.L, m.q); break;
    case 5: oz_slice_cols<5><<<blocks, 256, 0, st>>>(src, ld, m.rows, k0, p, m.e, m.SP, m.L, m.q); break;
    case 6: oz_slice_cols<6><<<blocks, 256, 0, st>>>(src, ld, m.rows, k0, p, m.e, m.SP, m.L, m.q); break;
    default: oz_slice_cols<7><<<blocks, 256, 0, st>>>(src, ld, m.rows, k0, p, m.e, m.SP, m.L, m.q); break;
    }
    TR_CHECK_LAUNCH("oz_slice_cols");
    prof.end(st, tok);
}

void oz_split_rows(Prof &prof, cudaStream_t st, const char *name, const double *x, long long sr, long long sk,
                   OzMat &m, long long r0, long long nr)
{
    TR_REQUIRE(r0 >= 0 && nr >= 0 && r0 + nr <= m.rows, TR_EINVAL, "Ozaki split: row range out of bounds");
    if (nr == 0) return;
    OzMat v = m;
    v.q = m.q + r0 * m.L;
    v.e = m.e + r0;
    v.rows = nr;
    oz_split(prof, st, name, x, sr, sk, v);
}

void oz_gemm(Prof &prof, cudaStream_t st, const char *name, const OzMat &A, long long a0, long long a1, long long a2,
             int kbA, const OzMat &B, long long c0, long long c1, long long c2, int kbB, int M, int N, int nkb, int n1,
             int n2, const OzOut &out, int *err, int ksplit, double *ws, size_t ws_count, const int *klist,
             const int *kcount, int kld)
{
    if (M <= 0 || N <= 0 || n1 <= 0 || n2 <= 0) return;
    TR_REQUIRE(A.q && B.q && A.S == B.S, TR_EINVAL, "Ozaki GEMM: operands must share the slice count");
    TR_REQUIRE(a0 >= 0 && a1 >= 0 && a2 >= 0 && c0 >= 0 && c1 >= 0 && c2 >= 0, TR_EINVAL,
               "Ozaki GEMM: negative row offset");
    TR_REQUIRE(kbA >= 0 && kbB >= 0 && nkb >= 1 && kbA + nkb <= A.nkb && kbB + nkb <= B.nkb, TR_EINVAL,
               "Ozaki GEMM: K blocks out of range");
    ksplit = std::max(1, std::min(ksplit, nkb));
    TR_REQUIRE(!klist == !kcount && (!klist || (ksplit == 1 && kld >= 1 && kld <= nkb)), TR_EINVAL,
               "Ozaki GEMM: block-sparse K needs both lists and no K split");
    const long long nb = (long long)n1 * n2;
    TR_REQUIRE(cdiv(M, 128) <= (1 << 30), TR_EINVAL, "Ozaki GEMM: too many tiles");
    TR_REQUIRE(ksplit == 1 || (ws && (size_t)ksplit * nb * M * N <= ws_count), TR_EINVAL,
               "Ozaki GEMM: split-K workspace too small");
    const int S = A.S;
    const int BN = 64;
    const long long lastA = a0 + a1 * (n1 - 1) + a2 * (n2 - 1) + (long long)cdiv(M, 128) * 128;
    const long long lastB = c0 + c1 * (n1 - 1) + c2 * (n2 - 1) + (long long)cdiv(N, BN) * BN;
    TR_REQUIRE(lastA < (1LL << 31) && lastB < (1LL << 31), TR_EINVAL, "Ozaki GEMM: row index overflow");
    OzArgs g;
    g.M = M;
    g.N = N;
    g.nkb = nkb;
    g.n2 = n2;
    g.ksplit = ksplit;
    g.kchunk = cdiv(nkb, ksplit);
    g.kbA = kbA;
    g.kbB = kbB;
    g.a0 = a0;
    g.a1 = a1;
    g.a2 = a2;
    g.c0 = c0;
    g.c1 = c1;
    g.c2 = c2;
    g.rowsA = A.rows;
    g.rowsB = B.rows;
    g.eA = A.e;
    g.eB = B.e;
    g.d = ksplit > 1 ? ws : out.d;
    g.s1 = out.s1;
    g.s2 = out.s2;
    g.ldm = out.ldm;
    g.ldn = out.ldn;
    g.alpha = out.alpha;
    g.accumulate = out.accumulate ? 1 : 0;
    g.err = err;
    g.wait = prof.wait_cycles > 0 ? prof.wait_cycles : ptx::WAIT_CYCLES;
    g.stall = prof.wait_stall;
    g.klist = klist;
    g.kcount = kcount;
    g.kld = kld;
    g.ntn = cdiv(N, BN);
    g.ntm = cdiv(M, 128);
    g.ntiles = (long long)g.ntn * g.ntm * nb * ksplit;
    static const int nsm = []() {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
        cudaGetLastError();
        return n > 0 ? n : 148;
    }();
    dim3 grid((unsigned)std::min<long long>(g.ntiles, nsm));
    const double flops = 2.0 * M * N * (double)nkb * 32 * nb;
    const double bytes = 2.0 * A.SP * ((double)M + N) * nkb * 32 * nb + 8.0 * M * N * nb;
    int tok = prof.begin(st, name, flops, bytes);
    switch (S) {
    case 2: oz_launch<2, 64>(st, grid, A, B, g); break;
    case 3: oz_launch<3, 64>(st, grid, A, B, g); break;
    case 4: oz_launch<4, 64>(st, grid, A, B, g); break;
    case 5: oz_launch<5, 64>(st, grid, A, B, g); break;
    case 6: oz_launch<6, 64>(st, grid, A, B, g); break;
    default: oz_launch<7, 64>(st, grid, A, B, g); break;
    }
    TR_CHECK_LAUNCH(name);
    if (ksplit > 1) {
        const long long tot = nb * M * N;
        const unsigned blocks = (unsigned)std::min<long long>(cdiv(tot, 256), 152LL * 8);
        oz_split_reduce<<<blocks, 256, 0, st>>>(ws, ksplit, (int)nb, n2, M, N, out.d, out.s1, out.s2, out.ldm, out.ldn,
                                                out.alpha, out.accumulate ? 1 : 0);
        TR_CHECK_LAUNCH(name);
    }
    prof.end(st, tok);
}

void oz_gemm(Prof &prof, cudaStream_t st, const char *name, const OzMat &A, long long a0, long long a1,
             const OzMat &B, long long c0, long long c1, int M, int N, int nb, double *d, long long s1,
             long long ldm, long long ldn, double alpha, int *err, const int *klist, const int *kcount, int kld)
{
    TR_REQUIRE(A.K == B.K, TR_EINVAL, "Ozaki GEMM: operands must share K");
    OzOut o;
    o.d = d;
    o.s1 = s1;
    o.ldm = ldm;
    o.ldn = ldn;
    o.alpha = alpha;
    oz_gemm(prof, st, name, A, a0, a1, 0, 0, B, c0, c1, 0, 0, M, N, A.nkb, nb, 1, o, err, 1, nullptr, 0, klist, kcount,
            kld);
}

}  // namespace tr
