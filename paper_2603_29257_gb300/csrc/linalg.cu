// FP64 dense linear algebra kernels of libtdarisp.
//
// The FP64 pipe of GB300 is narrow (a few DFMA per clock per SM), so these
// kernels are designed to keep it busy rather than to save bandwidth: a
// 64x64x16 shared-memory tiled GEMM with register double-buffering and
// split-K for long reductions, and a column-wise Cholesky with the inverse
// of its factor.  (The Davidson subspace eigensolver lives in eigh.cu.)
#include "linalg.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>

namespace tr {
namespace {

constexpr int BK = 16, NT = 256;

// Thread (tx, ty) of a 16 x 16 block computes TM x TN outputs at rows
// ty + 16 i and columns tx + 16 j; the block tile is (16 TM) x (16 TN).
// Skinny shapes (a dimension of a few dozen) use TM or TN = 1.  With ktl
// (block-sparse B, no K split) the block visits only the K tiles listed for its
// column tile: ktl[blockIdx.x * ktld + t] for t < ktc[blockIdx.x].
template <typename TI, typename TC, bool TA, bool TB, int TM, int TN>
__global__ void __launch_bounds__(NT)
    gemm_kernel(int M, int N, int K, double alpha, const TI *__restrict__ A, long long lda,
                const TI *__restrict__ B, long long ldb, double beta, TC *__restrict__ C,
                long long ldc, Batch bt, int ksplit, int kchunk, double *__restrict__ ws,
                const int *__restrict__ ktl, const int *__restrict__ ktc, int ktld)
{
    constexpr int BM = 16 * TM, BN = 16 * TN;
    __shared__ TI As[BK][BM + 1];
    __shared__ TI Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int z = blockIdx.z;
    const int b = z / ksplit, ks = z - b * ksplit;
    const int b1 = b / bt.n2, b2 = b - b1 * bt.n2;
    A += b1 * bt.sA1 + b2 * bt.sA2;
    B += b1 * bt.sB1 + b2 * bt.sB2;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = ks * kchunk;
    const int ke = min(K, kb + kchunk);

    TI acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = (TI)0;
    TI ra[TM], rb[TN];

    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            const int idx = tid + r * NT;
            const int kk = TA ? idx / BM : (idx & 15);
            const int mm = TA ? idx % BM : (idx >> 4);
            const int m = m0 + mm, k = k0 + kk;
            ra[r] = (m < M && k < ke) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : (TI)0;
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
            const int idx = tid + r * NT;
            const int kk = TB ? (idx & 15) : idx / BN;
            const int nn = TB ? (idx >> 4) : idx % BN;
            const int n = n0 + nn, k = k0 + kk;
            rb[r] = (n < N && k < ke) ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : (TI)0;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
            const int idx = tid + r * NT;
            if (TA)
                As[idx / BM][idx % BM] = ra[r];
            else
                As[idx & 15][idx >> 4] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
            const int idx = tid + r * NT;
            if (TB)
                Bs[idx & 15][idx >> 4] = rb[r];
            else
                Bs[idx / BN][idx % BN] = rb[r];
        }
    };

    // K tiles of this block: [kb, ke) in steps of BK, or the listed ones
    const int nk = ktl ? ktc[blockIdx.x] : (ke > kb ? (ke - kb + BK - 1) / BK : 0);
    const int *kt = ktl ? ktl + (long long)blockIdx.x * ktld : nullptr;
    if (nk > 0) load(kt ? kt[0] * BK : kb);
    for (int t = 0; t < nk; ++t) {
        store();
        __syncthreads();
        if (t + 1 < nk) load(kt ? kt[t + 1] * BK : kb + (t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            TI a[TM], bb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }

    const int nbatch = gridDim.z / ksplit;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            if (ksplit == 1) {
                TC *c = C + b1 * bt.sC1 + b2 * bt.sC2 + (long long)m * ldc + n;
                const double v = (double)acc[i][j];
                *c = (TC)((beta == 0.0) ? alpha * v : fma(alpha, v, beta * (double)*c));
            } else {
                ws[((long long)(ks * nbatch + b) * M + m) * N + n] = (double)acc[i][j];
            }
        }
    }
}

template <typename TC>
__global__ void splitk_reduce(int M, int N, int nbatch, int ksplit, const double *__restrict__ ws,
                              double alpha, double beta, TC *__restrict__ C, long long ldc, Batch bt)
{
    long long tot = (long long)nbatch * M * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int n = (int)(t % N);
        long long r = t / N;
        int m = (int)(r % M);
        int b = (int)(r / M);
        double s = 0.0;
        for (int ks = 0; ks < ksplit; ++ks) s += ws[((long long)(ks * nbatch + b) * M + m) * N + n];
        int b1 = b / bt.n2, b2 = b - b1 * bt.n2;
        TC *c = C + b1 * bt.sC1 + b2 * bt.sC2 + (long long)m * ldc + n;
        *c = (TC)((beta == 0.0) ? alpha * s : fma(alpha, s, beta * (double)*c));
    }
}

// ---------------------------------------------------------------- Cholesky

// Blocked right-looking Cholesky, panels of CB columns: factor the diagonal
// block (chol_diag), solve the rows below it against that block (chol_panel),
// subtract the panel's outer product from the trailing lower triangle
// (chol_update).  Three launches per panel; only the lower triangle and the
// diagonal are read or written.
constexpr int CB = 32;

// the diagonal block G[k0 .. k0+b)^2 in shared memory, one thread per
// element; per column j: the entries below the pivot are scaled (each thread
// takes the pivot's square root itself, the pivot is written afterwards), then
// the block's trailing part is updated; two barriers per column
__global__ void __launch_bounds__(CB * CB) chol_diag(double *G, int n, int k0, int b, int *flag)
{
    __shared__ double A[CB][CB + 1];
    const int m = threadIdx.x, i = threadIdx.y;
    const bool in = i < b && m <= i;
    if (in) A[i][m] = G[(long long)(k0 + i) * n + k0 + m];
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        double ljj = 0.0;
        if (m == j && i >= j && i < b) {
            double d = A[j][j];
            if (!(d > 0.0)) {
                if (i == j) atomicCAS(flag, 0, k0 + j + 1);  // the first non-positive pivot is kept
                d = 1.0;
            }
            ljj = sqrt(d);
            if (i > j) A[i][j] = A[i][j] / ljj;
        }
        __syncthreads();
        if (i == j && m == j) A[j][j] = ljj;
        if (i > j && i < b && m > j && m <= i) A[i][m] = fma(-A[i][j], A[m][j], A[i][m]);
        __syncthreads();
    }
    if (in) G[(long long)(k0 + i) * n + k0 + m] = A[i][m];
}

// rows i >= k0 + b: L[i][k0 .. k0+b) = G[i][k0 .. k0+b) L11^-T, one thread per
// row (the row's entries loaded first; two partial sums per entry)
__global__ void __launch_bounds__(32) chol_panel(double *G, int n, int k0, int b)
{
    __shared__ double L11[CB][CB + 1];
    __shared__ double rdg[CB];
    for (int t = threadIdx.x; t < CB * CB; t += blockDim.x) {
        const int r = t / CB, s = t % CB;
        if (r < b && s <= r) L11[r][s] = G[(long long)(k0 + r) * n + k0 + s];
    }
    __syncthreads();
    if (threadIdx.x < b) rdg[threadIdx.x] = 1.0 / L11[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int i = k0 + b + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *row = G + (long long)i * n + k0;
    double x[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) x[j] = j < b ? row[j] : 0.0;
#pragma unroll
    for (int j = 0; j < CB; ++j) {
        if (j < b) {
            double s0 = x[j], s1 = 0.0;
#pragma unroll
            for (int q = 0; q < j; ++q) {
                if (q & 1)
                    s1 = fma(-x[q], L11[j][q], s1);
                else
                    s0 = fma(-x[q], L11[j][q], s0);
            }
            x[j] = (s0 + s1) * rdg[j];
        }
    }
#pragma unroll
    for (int j = 0; j < CB; ++j)
        if (j < b) row[j] = x[j];
}

// G[i][j] -= sum_q L[i][k0+q] L[j][k0+q] for k1 <= j <= i < n, k1 = k0 + b:
// 32 x 32 tiles of the trailing lower triangle, 2 x 2 elements per thread
__global__ void __launch_bounds__(256) chol_update(double *G, int n, int k0, int b)
{
    const int ti = blockIdx.y, tj = blockIdx.x;
    if (tj > ti) return;
    const int k1 = k0 + b;
    const int i0 = k1 + ti * 32, j0 = k1 + tj * 32;
    __shared__ double Pi[32][CB + 1], Pj[32][CB + 1];
    for (int t = threadIdx.x; t < 32 * CB; t += blockDim.x) {
        const int r = t / CB, q = t % CB;
        Pi[r][q] = (i0 + r < n && q < b) ? G[(long long)(i0 + r) * n + k0 + q] : 0.0;
        Pj[r][q] = (j0 + r < n && q < b) ? G[(long long)(j0 + r) * n + k0 + q] : 0.0;
    }
    __syncthreads();
    const int r0 = (threadIdx.x / 16) * 2, c0 = (threadIdx.x % 16) * 2;
    double s[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll 8
    for (int q = 0; q < CB; ++q)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int e = 0; e < 2; ++e) s[a][e] = fma(Pi[r0 + a][q], Pj[c0 + e][q], s[a][e]);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = i0 + r0 + a, j = j0 + c0 + e;
            if (i < n && j <= i) G[(long long)i * n + j] -= s[a][e];
        }
}

// Linv[i][c] (lower) = column c of L^-1, one warp per column: x_c = 1 / L_cc,
// x_i = -(sum_{c <= j < i} L_ij x_j) / L_ii for i > c, the sums over lanes;
// x and the reciprocal diagonal in shared memory.
__global__ void tri_inverse_warp(const double *__restrict__ L, int n, double *__restrict__ Linv)
{
    extern __shared__ double tsm[];
    double *rd = tsm;  // 1 / L_ii
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *x = tsm + n + (size_t)warp * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rd[i] = 1.0 / L[(long long)i * n + i];
    __syncthreads();
    const int c = blockIdx.x * wpb + warp;
    if (c >= n) return;
    for (int i = lane; i < c; i += 32) Linv[(long long)i * n + c] = 0.0;
    if (lane == 0) x[c] = rd[c];
    __syncwarp();
    for (int i = c + 1; i < n; ++i) {
        const double *Li = L + (long long)i * n;
        double s = 0.0;
        for (int j = c + lane; j < i; j += 32) s = fma(Li[j], x[j], s);
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = -s * rd[i];
        __syncwarp();
    }
    for (int i = c + lane; i < n; i += 32) Linv[(long long)i * n + c] = x[i];
}

// Linv[i][c] (lower) = column c of L^-1 by forward substitution, one thread per
// column: for orders too large for tri_inverse_warp's shared memory.
__global__ void tri_inverse_cols(const double *__restrict__ L, int n, double *__restrict__ Linv)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int i = 0; i < c; ++i) Linv[(long long)i * n + c] = 0.0;
    Linv[(long long)c * n + c] = 1.0 / L[(long long)c * n + c];
    for (int i = c + 1; i < n; ++i) {
        double s = 0.0;
        for (int j = c; j < i; ++j) s = fma(L[(long long)i * n + j], Linv[(long long)j * n + c], s);
        Linv[(long long)i * n + c] = -s / L[(long long)i * n + i];
    }
}

__global__ void sum_rows_kernel(const double *__restrict__ a, int nrows, int n, double *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int r = 0; r < nrows; ++r) s += a[(long long)r * n + i];
    out[i] = s;
}

template <typename TI, typename TC, int TM, int TN>
void launch_gemm(cudaStream_t st, bool ta, bool tb, dim3 grid, int M, int N, int K, double alpha,
                 const TI *A, long long lda, const TI *B, long long ldb, double beta, TC *C,
                 long long ldc, const Batch &bt, int ksplit, int kchunk, double *ws,
                 const int *ktl = nullptr, const int *ktc = nullptr, int ktld = 0)
{
    if (!ta && !tb)
        gemm_kernel<TI, TC, false, false, TM, TN><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws, ktl, ktc, ktld);
    else if (!ta && tb)
        gemm_kernel<TI, TC, false, true, TM, TN><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws, ktl, ktc, ktld);
    else if (ta && !tb)
        gemm_kernel<TI, TC, true, false, TM, TN><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws, ktl, ktc, ktld);
    else
        gemm_kernel<TI, TC, true, true, TM, TN><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws, ktl, ktc, ktld);
}

// resident CTAs per SM of a gemm_kernel instance (queried once) and the SM count
template <typename TI, typename TC, int TM, int TN>
int gemm_occupancy(bool ta, bool tb)
{
    // contexts are created from several host threads (batched builds, the server):
    // the cached values are atomics, and a concurrent first query stores the same value
    static std::atomic<int> occ[2][2];
    std::atomic<int> &o = occ[ta][tb];
    if (o.load(std::memory_order_relaxed) == 0) {
        int v = 0;
        cudaError_t e;
        if (!ta && !tb) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_kernel<TI, TC, false, false, TM, TN>, NT, 0);
        else if (!ta) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_kernel<TI, TC, false, true, TM, TN>, NT, 0);
        else if (!tb) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_kernel<TI, TC, true, false, TM, TN>, NT, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, gemm_kernel<TI, TC, true, true, TM, TN>, NT, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            v = 1;
        }
        o.store(std::max(v, 1), std::memory_order_relaxed);
    }
    return o.load(std::memory_order_relaxed);
}

int sm_count()
{
    static std::atomic<int> n{0};
    if (n.load(std::memory_order_relaxed) == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            v = 152;
        }
        n.store(std::max(v, 1), std::memory_order_relaxed);
    }
    return n.load(std::memory_order_relaxed);
}

template <typename TI, typename TC>
void gemm_any(Prof &prof, cudaStream_t st, const char *name, bool ta, bool tb, int M, int N, int K,
              double alpha, const TI *A, long long lda, const TI *B, long long ldb, double beta,
              TC *C, long long ldc, const Batch &bt, double *ws, size_t ws_elems, double alg_bytes,
              int max_kchunk)
{
    if (M <= 0 || N <= 0 || bt.count() <= 0) return;
    const int nb = bt.count();
    if (K < 0) K = 0;
    // tile shape: 64 x 64, or 16 x 64 / 64 x 16 when one side is skinny
    int TM = 4, TN = 4;
    if (M <= 32 && N > 32) TM = 1;
    else if (N <= 32 && M > 32) TN = 1;
    else if (M <= 32 && N <= 32) TM = TN = 1;
    const int BMx = 16 * TM, BNx = 16 * TN;
    long long tiles = (long long)cdiv(M, BMx) * cdiv(N, BNx) * nb;
    int ksplit = 1;
    const long long target = 4 * 152;
    if (ws && ((tiles < target && K >= 4 * 256) || (max_kchunk > 0 && K > max_kchunk))) {
        long long want = std::min<long long>((target + tiles - 1) / tiles, K / 256);
        if (max_kchunk > 0) want = std::max<long long>(want, (K + max_kchunk - 1) / max_kchunk);
        long long cap = (long long)(ws_elems / ((size_t)nb * M * N));
        ksplit = (int)std::max<long long>(1, std::min(want, cap));
        ksplit = std::min(ksplit, 65535 / nb);
        ksplit = std::max(ksplit, 1);
    }
    // wave quantisation of large FP64 launches: when the output tiles fill the GPU
    // a few times over with a ragged last wave, split K 2..4 ways (at least 1024
    // per part) if that evens out the waves by more than 3 %; partial sums in ws
    if (ksplit == 1 && ws && max_kchunk == 0 && sizeof(TI) == 8 && TM == 4 && TN == 4 && tiles >= target &&
        K >= 2048) {
        const long long wave = (long long)sm_count() * gemm_occupancy<TI, TC, 4, 4>(ta, tb);
        auto eff = [&](int ks) {
            const long long t = tiles * ks;
            return (double)t / (double)(((t + wave - 1) / wave) * wave);
        };
        double best = eff(1) + 0.03;
        for (int ks = 2; ks <= 4; ++ks) {
            if (K / ks < 1024 || (size_t)ks * nb * M * N > ws_elems || (long long)nb * ks > 65535) break;
            if (eff(ks) > best) {
                best = eff(ks);
                ksplit = ks;
            }
        }
    }
    int kchunk = K;
    if (ksplit > 1) {
        kchunk = (int)(((K + ksplit - 1) / ksplit + BK - 1) / BK * BK);
        ksplit = (K + kchunk - 1) / kchunk;
    }
    TR_REQUIRE((long long)nb * ksplit <= 65535, TR_EINVAL, "gemm: batch too large");
    TR_REQUIRE(cdiv(M, BMx) <= 65535, TR_EINVAL, "gemm: M too large");
    dim3 grid(cdiv(N, BNx), cdiv(M, BMx), nb * ksplit);
    double flops = 2.0 * M * N * (double)K * nb;
    double bytes = alg_bytes >= 0 ? alg_bytes
                                  : (double)sizeof(TI) * ((double)M * K + (double)K * N) * nb + 2.0 * sizeof(TC) * M * N * nb;
    int tok = prof.begin(st, name, flops, bytes);
    if (TM == 4 && TN == 4)
        launch_gemm<TI, TC, 4, 4>(st, ta, tb, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    else if (TM == 1 && TN == 4)
        launch_gemm<TI, TC, 1, 4>(st, ta, tb, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    else if (TM == 4 && TN == 1)
        launch_gemm<TI, TC, 4, 1>(st, ta, tb, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    else
        launch_gemm<TI, TC, 1, 1>(st, ta, tb, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    TR_CHECK_LAUNCH(name);
    if (ksplit > 1) {
        prof.launches += 1;
        long long tot = (long long)nb * M * N;
        int blocks = (int)std::min<long long>(cdiv(tot, 256), 4096);
        splitk_reduce<TC><<<blocks, 256, 0, st>>>(M, N, nb, ksplit, ws, alpha, beta, C, ldc, bt);
        TR_CHECK_LAUNCH(name);
    }
    prof.end(st, tok);
}

}  // namespace

void dgemm(Prof &prof, cudaStream_t st, const char *name, bool ta, bool tb, int M, int N, int K,
           double alpha, const double *A, long long lda, const double *B, long long ldb, double beta,
           double *C, long long ldc, const Batch &bt, double *ws, size_t ws_elems, double alg_bytes)
{
    gemm_any<double, double>(prof, st, name, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ws,
                             ws_elems, alg_bytes, 0);
}

void gemm_prepare()
{
    // the occupancy and SM-count queries of the wave-quantisation split, made
    // once outside any stream capture
    sm_count();
    for (int ta = 0; ta < 2; ++ta)
        for (int tb = 0; tb < 2; ++tb) gemm_occupancy<double, double, 4, 4>(ta != 0, tb != 0);
}

void dgemm_ktiles(Prof &prof, cudaStream_t st, const char *name, bool ta, int M, int N, int K, double alpha,
                  const double *A, long long lda, const double *B, long long ldb, double beta, double *C,
                  long long ldc, const Batch &bt, const KTiles &kt)
{
    if (M <= 0 || N <= 0 || bt.count() <= 0) return;
    TR_REQUIRE(kt.list && kt.count && kt.ld >= cdiv(std::max(K, 1), BK), TR_EINVAL, "gemm: bad K-tile list");
    const int nb = bt.count();
    TR_REQUIRE(nb <= 65535 && cdiv(M, 64) <= 65535, TR_EINVAL, "gemm: batch or M too large");
    dim3 grid(cdiv(N, 64), cdiv(M, 64), nb);
    // performed flops (listed tiles only) and every operand byte read once
    const double flops = 2.0 * (double)M * 64.0 * BK * (double)kt.active * nb;
    const double bytes = 8.0 * ((double)M * K + (double)K * N) * nb + 16.0 * M * N * nb;
    int tok = prof.begin(st, name, flops, bytes);
    launch_gemm<double, double, 4, 4>(st, ta, false, grid, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, 1, K,
                                      nullptr, kt.list, kt.count, kt.ld);
    TR_CUDA(cudaGetLastError());
    prof.end(st, tok);
}

void sgemm(Prof &prof, cudaStream_t st, const char *name, bool ta, bool tb, int M, int N, int K,
           double alpha, const float *A, long long lda, const float *B, long long ldb, double beta,
           double *C, long long ldc, const Batch &bt, double *ws, size_t ws_elems, int max_kchunk)
{
    gemm_any<float, double>(prof, st, name, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ws,
                            ws_elems, -1.0, max_kchunk);
}

void cholesky(Prof &prof, cudaStream_t st, double *G, int n, int *flag)
{
    if (n <= 0) return;
    int tok = prof.begin(st, "cholesky", n * (double)n * n / 3.0, 8.0 * n * n);
    for (int k0 = 0; k0 < n; k0 += CB) {
        const int b = std::min(CB, n - k0), rest = n - k0 - b;
        chol_diag<<<1, dim3(CB, CB), 0, st>>>(G, n, k0, b, flag);
        prof.launches += 1;
        if (rest > 0) {
            chol_panel<<<cdiv(rest, 32), 32, 0, st>>>(G, n, k0, b);
            const unsigned nt = cdiv(rest, 32);
            chol_update<<<dim3(nt, nt), 256, 0, st>>>(G, n, k0, b);
            prof.launches += 2;
        }
    }
    TR_CHECK_LAUNCH("cholesky");
    prof.end(st, tok);
}

void chol_inverse(Prof &prof, cudaStream_t st, const double *L, int n, double *Ginv, double *work)
{
    if (n <= 0) return;
    // warps (columns) per block: x of each and 1/L_ii in at most 200 KB of shared memory
    const int wpb = std::min<long long>(8, std::max<long long>(0, 200LL * 1024 / (8LL * n) - 1));
    if (wpb >= 1) {
        static const cudaError_t attr =
            cudaFuncSetAttribute(tri_inverse_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        TR_CUDA(attr);
        const size_t smem = sizeof(double) * (size_t)n * (1 + wpb);
        TR_LAUNCH(prof, st, "tri_inverse", n * (double)n * n / 3.0, 8.0 * n * n,
                  tri_inverse_warp<<<cdiv(n, wpb), 32 * wpb, smem, st>>>(L, n, work));
    } else {
        TR_LAUNCH(prof, st, "tri_inverse", n * (double)n * n / 3.0, 8.0 * n * n,
                  tri_inverse_cols<<<cdiv(n, 64), 64, 0, st>>>(L, n, work));
    }
    // Ginv = Linv^T Linv
    dgemm(prof, st, "metric_inverse", true, false, n, n, n, 1.0, work, n, work, n, 0.0, Ginv, n,
          Batch(), nullptr, 0);
}

void sum_rows(Prof &prof, cudaStream_t st, const double *a, int nrows, int n, double *out)
{
    if (n <= 0) return;
    TR_LAUNCH(prof, st, "sum_rows", 0, 0, sum_rows_kernel<<<cdiv(n, 256), 256, 0, st>>>(a, nrows, n, out));
}

}  // namespace tr
