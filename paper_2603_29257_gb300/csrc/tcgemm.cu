// Tensor-core GEMM C = A B^T on GB300 (sm_103a): tcgen05.mma kind::tf32.
//
// Persistent: one CTA per SM walks the 128 x BN output tiles (N tile fastest,
// then M tile, then batch entry).  Warp 0 (one lane) streams 128 x 32 FP32
// tiles of A and B through a ring of shared-memory stages with TMA
// (cp.async.bulk.tensor, 128-byte swizzle, completion on an mbarrier); warp 1
// (one lane) issues tcgen05.mma into one of two FP32 accumulator sets in
// tensor memory and releases each stage with tcgen05.commit; warps 2..5 drain
// a finished set (tcgen05.ld, 32 TMEM lanes each) and write the tile while the
// products of the next tile go on in the other set.  With three products
// (hi*hi + hi*lo + lo*hi) the result carries close to FP32 accuracy.  Stage
// and accumulator barrier phases run on across tiles.  Every mbarrier wait
// gives up after ~1 s (or the launch's own limit): it records an error code in
// *err and the warp skips to the teardown, where the copies and products still
// in flight are awaited before tensor memory is freed.
#include "tcgemm.cuh"
#include "tcptx.cuh"

#include <cuda.h>

#include <algorithm>
#include <mutex>

namespace tr {
namespace {

constexpr int BM = 128, BKF = 32;             // tile: 128 x BN outputs, 32 FP32 (128 B) of K per stage
constexpr int TILE_BYTES = BM * BKF * 4;      // 16 KB (A tile; a B tile is BN * 128 B)
struct TcArgs {
    int M, N, K, n2;
    int ka0, kb0;                 // K offsets (elements) into the A and B rows
    int ntn, ntm;                 // N and M tiles per batch entry
    long long ntiles;             // ntn x ntm x batch entries
    long long a0, a1, a2, c0, c1, c2;
    TcOut out;
    int *err;
    long long wait;               // pipeline wait limit in SM cycles
    int stall;                    // test of the bounded waits: the producer issues no loads
};

using namespace ptx;

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ float tf32_rest(float v)
{
    return v - __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
}

template <int NSPLIT, int BN>
struct TcCfg {
    static constexpr int BTILE = BN * BKF * 4;
    // stage layout: A value | B value | A remainder | B remainder
    static constexpr uint32_t STAGE = (NSPLIT == 3 ? 2u : 1u) * (uint32_t)(TILE_BYTES + BTILE);
    static constexpr int TBYTES = 4 * 32 * 33 * 4;  // epilogue transpose buffers: 4 warps x 32 x 33 floats
    static constexpr int FIT = (int)((227 * 1024 - TBYTES - 1024 - 256) / STAGE);
    static constexpr int STAGES = FIT > 4 ? 4 : FIT;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE + TBYTES + 1024 + 256;
    static constexpr int TCOLS = 2 * BN;  // two accumulator sets
    static_assert(STAGES >= 2 && SMEM <= 227 * 1024, "shared memory");
};

// output tile t: N tile fastest, then M tile, then batch entry
struct TcTile {
    int m0, n0, b1, b2, arow, brow;
};

__device__ __forceinline__ TcTile tc_tile(const TcArgs &g, long long t, int BN)
{
    TcTile u;
    const int nt = (int)(t % g.ntn);
    const long long r = t / g.ntn;
    const int mt = (int)(r % g.ntm);
    const int b = (int)(r / g.ntm);
    u.b1 = b / g.n2;
    u.b2 = b - u.b1 * g.n2;
    u.m0 = mt * BM;
    u.n0 = nt * BN;
    u.arow = (int)(g.a0 + g.a1 * u.b1 + g.a2 * u.b2) + u.m0;
    u.brow = (int)(g.c0 + g.c1 * u.b1 + g.c2 * u.b2) + u.n0;
    return u;
}

template <int NSPLIT, int MODE, int BN>
__global__ void __launch_bounds__(192, 1)
    tc_kernel(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
              const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl, const TcArgs g)
{
    using C = TcCfg<NSPLIT, BN>;
    constexpr int ST = C::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *tbuf = (float *)(smem + ST * C::STAGE);
    // barriers: full[ST], empty[ST], acc_full[2], acc_empty[2], drain
    uint64_t *bars = (uint64_t *)(smem + ST * C::STAGE + C::TBYTES);
    uint32_t *tslot = (uint32_t *)(bars + 2 * ST + 5);
    const uint32_t FULL = sa(&bars[0]), EMPTY = sa(&bars[ST]);
    const uint32_t ACCF = sa(&bars[2 * ST]), ACCE = sa(&bars[2 * ST + 2]);
    const uint32_t DRAIN = sa(&bars[2 * ST + 4]);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.K + BKF - 1) / BKF;
    const long long ntiles = g.ntiles;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * ST + 2; ++i) bar_init(sa(&bars[i]), 1);
        for (int i = 0; i < 2; ++i) bar_init(ACCE + 8 * i, 4);  // one arrival per epilogue warp
        bar_init(DRAIN, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tslot)),
                     "r"(C::TCOLS)
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
                const TcTile u = tc_tile(g, t, BN);
                for (int kt = 0; kt < nk; ++kt) {
                    const int s = (int)(gk % ST);
                    if (gk >= ST && !bar_wait(EMPTY + 8 * s, (uint32_t)(((gk / ST) - 1) & 1), g.err, 1, g.wait)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = FULL + 8 * s;
                    bar_expect(full, C::STAGE);
                    uint8_t *stg = smem + s * C::STAGE;
                    const int xa = g.ka0 + kt * BKF, xb = g.kb0 + kt * BKF;
                    tma2d(sa(stg), &tAh, xa, u.arow, full);
                    tma2d(sa(stg + TILE_BYTES), &tBh, xb, u.brow, full);
                    if (NSPLIT == 3) {
                        tma2d(sa(stg + TILE_BYTES + C::BTILE), &tAl, xa, u.arow, full);
                        tma2d(sa(stg + 2 * TILE_BYTES + C::BTILE), &tBl, xb, u.brow, full);
                    }
                    ++gk;
                }
            }
            // copies still in flight complete before the CTA ends
            for (long long q = gk > ST ? gk - ST : 0; q < gk; ++q)
                bar_wait(FULL + 8 * (int)(q % ST), (uint32_t)((q / ST) & 1), g.err, 5);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both
            // K-major, N = BN, M = 128
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
            long long gk = 0, tc = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tc) {
                const int buf = (int)(tc & 1);
                if (tc >= 2) {
                    // the epilogue has drained the tile that last used this accumulator set
                    if (!bar_wait(ACCE + 8 * buf, (uint32_t)(((tc / 2) - 1) & 1), g.err, 6, g.wait)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                }
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
                for (int kt = 0; kt < nk; ++kt) {
                    const int s = (int)(gk % ST);
                    if (!bar_wait(FULL + 8 * s, (uint32_t)((gk / ST) & 1), g.err, 2, g.wait)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    uint8_t *stg = smem + s * C::STAGE;
                    const uint64_t dA = smem_desc(sa(stg)), dB = smem_desc(sa(stg + TILE_BYTES));
                    const uint64_t dAl = smem_desc(sa(stg + TILE_BYTES + C::BTILE));
                    const uint64_t dBl = smem_desc(sa(stg + 2 * TILE_BYTES + C::BTILE));
#pragma unroll
                    for (int kk = 0; kk < BKF / 8; ++kk) {
                        mma(acc, dA + 2 * kk, dB + 2 * kk, idesc, (kt | kk) ? 1u : 0u);
                        if (NSPLIT == 3) {
                            mma(acc, dA + 2 * kk, dBl + 2 * kk, idesc, 1u);
                            mma(acc, dAl + 2 * kk, dB + 2 * kk, idesc, 1u);
                        }
                    }
                    commit(EMPTY + 8 * s);
                    ++gk;
                }
                if (!ok) break;
                commit(ACCF + 8 * buf);
            }
            // every product issued has completed before tensor memory is freed, also
            // when a wait gave up and the epilogue no longer consumes them
            commit(DRAIN);
            bar_wait(DRAIN, 0, g.err, 7);
        }
        __syncwarp();
    } else {
        // epilogue warps 2..5; a warp may read TMEM lanes 32 (warp % 4) .. + 31
        const int quarter = warp & 3;
        float *tb = tbuf + (warp - 2) * 32 * 33;
        const TcOut &o = g.out;
        long long tc = 0;
        for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
            const TcTile u = tc_tile(g, t, BN);
            const int buf = (int)(tc & 1);
            if (!bar_wait(ACCF + 8 * buf, (uint32_t)((tc / 2) & 1), g.err, 3, g.wait)) break;
            fence_after();
            const long long base = o.s1 * u.b1 + o.s2 * u.b2;
            const int row = u.m0 + 32 * quarter + lane;
            for (int c0 = 0; c0 < BN && u.n0 + c0 < g.N; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * BN + c0), r);
                if (o.ldm == 1) {
                    // consecutive lanes hold consecutive rows: write directly (coalesced)
                    if (row < g.M) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = u.n0 + c0 + j;
                            if (col >= g.N) break;
                            const long long off = base + (long long)row + (long long)col * o.ldn;
                            const float v = __uint_as_float(r[j]);
                            if (MODE == TC_SPLIT) {
                                o.hi[off] = v;
                                o.lo[off] = tf32_rest(v);
                            } else if (MODE == TC_STORE32) {
                                o.hi[off] = v;
                            } else if (MODE == TC_ACC64) {
                                o.d[off] += o.alpha * (double)v;
                            } else {
                                o.d[off] = o.alpha * (double)v;
                            }
                        }
                    }
                } else {
                    // transpose 32 x 32 through this warp's buffer so that lanes walk columns
#pragma unroll
                    for (int j = 0; j < 32; ++j) tb[lane * 33 + j] = __uint_as_float(r[j]);
                    __syncwarp();
                    const int col = u.n0 + c0 + lane;
                    for (int rr = 0; rr < 32; ++rr) {
                        const int rw = u.m0 + 32 * quarter + rr;
                        if (rw >= g.M || col >= g.N) continue;
                        const long long off = base + (long long)rw * o.ldm + (long long)col * o.ldn;
                        const float v = tb[rr * 33 + lane];
                        if (MODE == TC_SPLIT) {
                            o.hi[off] = v;
                            o.lo[off] = tf32_rest(v);
                        } else if (MODE == TC_STORE32) {
                            o.hi[off] = v;
                        } else if (MODE == TC_ACC64) {
                            o.d[off] += o.alpha * (double)v;
                        } else {
                            o.d[off] = o.alpha * (double)v;
                        }
                    }
                    __syncwarp();
                }
            }
            // the accumulator set is free for the tile after next
            fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(ACCE + 8 * buf);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS) : "memory");
}

__global__ void split_kernel(const double *__restrict__ x, long long rows, long long cols, long long ldi,
                             float *__restrict__ hi, float *__restrict__ lo, long long ldo)
{
    const long long tot = rows * cols;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / cols, c = t - r * cols;
        const float f = (float)x[r * ldi + c];
        hi[r * ldo + c] = f;
        lo[r * ldo + c] = tf32_rest(f);
    }
}

void encode(CUtensorMap &tm, const float *p, long long rows, long long kdim, long long ld, int box_rows)
{
    tma_encode_2d(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, p, rows, kdim, ld * 4, BKF, box_rows);
}

template <int NSPLIT, int MODE, int BN>
void launch(cudaStream_t st, dim3 grid, const TcMat &A, const TcMat &B, const TcArgs &g)
{
    using C = TcCfg<NSPLIT, BN>;
    // set once per kernel instance (thread-safe static initialisation)
    static const cudaError_t attr =
        cudaFuncSetAttribute(tc_kernel<NSPLIT, MODE, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    TR_CUDA(attr);
    const CUtensorMap &bh = BN == 64 ? B.mhi64 : B.mhi;
    const CUtensorMap &bl = BN == 64 ? B.mlo64 : B.mlo;
    tc_kernel<NSPLIT, MODE, BN><<<grid, 192, C::SMEM, st>>>(A.mhi, NSPLIT == 3 ? A.mlo : A.mhi, bh,
                                                             NSPLIT == 3 ? bl : bh, g);
}

template <int NSPLIT, int BN>
void launch_mode(cudaStream_t st, dim3 grid, const TcMat &A, const TcMat &B, const TcArgs &g, int mode)
{
    if (mode == TC_SPLIT) launch<NSPLIT, TC_SPLIT, BN>(st, grid, A, B, g);
    else if (mode == TC_ACC64) launch<NSPLIT, TC_ACC64, BN>(st, grid, A, B, g);
    else if (mode == TC_STORE32) launch<NSPLIT, TC_STORE32, BN>(st, grid, A, B, g);
    else launch<NSPLIT, TC_STORE64, BN>(st, grid, A, B, g);
}

}  // namespace

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        TR_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        TR_REQUIRE(q == cudaDriverEntryPointSuccess && p, TR_ECUDA, "cuTensorMapEncodeTiled unavailable");
        fn = (EncodeTiled)p;
    }
    return fn;
}

void tma_encode_2d(CUtensorMap &tm, CUtensorMapDataType dt, const void *p, long long rows, long long kdim,
                   long long ld_bytes, int box_inner, int box_rows)
{
    cuuint64_t gdim[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
    cuuint64_t gstr[1] = {(cuuint64_t)ld_bytes};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = encoder()(&tm, dt, 2, (void *)p, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    TR_REQUIRE(r == CUDA_SUCCESS, TR_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

void tc_make(TcMat &m, const float *hi, const float *lo, long long rows, long long kdim, long long ld)
{
    TR_REQUIRE((ld * 4) % 16 == 0, TR_EINVAL, "tensor-core operand: row stride must be a multiple of 16 bytes");
    TR_REQUIRE(((uintptr_t)hi % 16) == 0 && (!lo || ((uintptr_t)lo % 16) == 0), TR_EINVAL,
               "tensor-core operand: base must be 16-byte aligned");
    TR_REQUIRE(rows > 0 && kdim > 0 && rows < (1LL << 31) && kdim <= ld, TR_EINVAL, "tensor-core operand: bad shape");
    m.hi = hi;
    m.lo = lo;
    m.rows = rows;
    m.kdim = kdim;
    m.ld = ld;
    encode(m.mhi, hi, rows, kdim, ld, 128);
    encode(m.mhi64, hi, rows, kdim, ld, 64);
    if (lo) {
        encode(m.mlo, lo, rows, kdim, ld, 128);
        encode(m.mlo64, lo, rows, kdim, ld, 64);
    } else {
        m.mlo = m.mhi;
        m.mlo64 = m.mhi64;
    }
}

void tc_gemm(Prof &prof, cudaStream_t st, const char *name, int nsplit, const TcMat &A, long long a0, long long a1,
             long long a2, int ka0, const TcMat &B, long long c0, long long c1, long long c2, int kb0, int M, int N,
             int K, int n1, int n2, const TcOut &out, int *err, double alg_bytes, int bn)
{
    if (M <= 0 || N <= 0 || n1 <= 0 || n2 <= 0) return;
    TR_REQUIRE(bn == 64 || bn == 128, TR_EINVAL, "tc_gemm: tile width must be 64 or 128");
    const int BN = bn;
    TR_REQUIRE(nsplit == 1 || nsplit == 3, TR_EINVAL, "tc_gemm: nsplit must be 1 or 3");
    TR_REQUIRE(nsplit == 1 || (A.lo && B.lo), TR_EINVAL, "tc_gemm: 3-product form needs lo parts");
    TR_REQUIRE(K > 0 && ka0 >= 0 && kb0 >= 0 && ka0 + K <= A.kdim && kb0 + K <= B.kdim, TR_EINVAL, "tc_gemm: bad K");
    TR_REQUIRE(ka0 % 4 == 0 && kb0 % 4 == 0, TR_EINVAL, "tc_gemm: K offsets must be 16-byte aligned");
    TR_REQUIRE(cdiv(M, BM) <= (1 << 30) && (long long)n1 * n2 <= (1LL << 31), TR_EINVAL, "tc_gemm: too many tiles");
    // every row a CTA addresses must exist in the operand views (rows past M may
    // belong to the next batch entry and are discarded)
    const long long lastA = a0 + a1 * (n1 - 1) + a2 * (n2 - 1) + (long long)cdiv(M, BM) * BM;
    const long long lastB = c0 + c1 * (n1 - 1) + c2 * (n2 - 1) + (long long)cdiv(N, BN) * BN;
    TR_REQUIRE(a0 >= 0 && c0 >= 0 && a1 >= 0 && a2 >= 0 && c1 >= 0 && c2 >= 0, TR_EINVAL, "tc_gemm: negative row offset");
    TR_REQUIRE(lastA < (1LL << 31) && lastB < (1LL << 31), TR_EINVAL, "tc_gemm: row index overflow");
    TcArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.n2 = n2;
    g.ka0 = ka0;
    g.kb0 = kb0;
    g.a0 = a0;
    g.c0 = c0;
    g.a1 = a1;
    g.a2 = a2;
    g.c1 = c1;
    g.c2 = c2;
    g.out = out;
    g.err = err;
    g.wait = prof.wait_cycles > 0 ? prof.wait_cycles : ptx::WAIT_CYCLES;
    g.stall = prof.wait_stall;
    g.ntn = cdiv(N, BN);
    g.ntm = cdiv(M, BM);
    g.ntiles = (long long)g.ntn * g.ntm * n1 * n2;
    static const int nsm = []() {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
        cudaGetLastError();
        return n > 0 ? n : 148;
    }();
    dim3 grid((unsigned)std::min<long long>(g.ntiles, nsm));
    const double flops = 2.0 * M * N * (double)K * n1 * n2;
    const double bytes = alg_bytes >= 0 ? alg_bytes : 4.0 * nsplit * ((double)M + N) * K * n1 * n2;
    int tok = prof.begin(st, name, flops, bytes);
    if (nsplit == 3 && bn == 128) launch_mode<3, 128>(st, grid, A, B, g, out.mode);
    else if (nsplit == 3) launch_mode<3, 64>(st, grid, A, B, g, out.mode);
    else if (bn == 128) launch_mode<1, 128>(st, grid, A, B, g, out.mode);
    else launch_mode<1, 64>(st, grid, A, B, g, out.mode);
    TR_CHECK_LAUNCH(name);
    prof.end(st, tok);
}

void tc_split(Prof &prof, cudaStream_t st, const double *x, long long rows, long long cols, long long ld_in, float *hi,
              float *lo, long long ld_out)
{
    const long long tot = rows * cols;
    if (tot <= 0) return;
    const unsigned blocks = (unsigned)std::min<long long>(cdiv(tot, 256), 152 * 16);
    TR_LAUNCH(prof, st, "split_f32", 0, 16.0 * tot, split_kernel<<<blocks, 256, 0, st>>>(x, rows, cols, ld_in, hi, lo, ld_out));
}

}  // namespace tr
