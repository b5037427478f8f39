// FP64 dense linear algebra kernels of libtdarisp.
//
// The FP64 pipe of GB300 is narrow (a few DFMA per clock per SM), so these
// kernels are designed to keep it busy rather than to save bandwidth: a
// 64x64x16 shared-memory tiled GEMM with register double-buffering and
// split-K for long reductions, a column-wise Cholesky, and a one-block
// parallel cyclic Jacobi eigensolver for the Davidson subspace matrix.
#include "linalg.cuh"

#include <algorithm>
#include <cmath>

namespace tr {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(NT)
    dgemm_kernel(int M, int N, int K, double alpha, const double *__restrict__ A, long long lda,
                 const double *__restrict__ B, long long ldb, double beta, double *__restrict__ C,
                 long long ldc, Batch bt, int ksplit, int kchunk, double *__restrict__ ws)
{
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int z = blockIdx.z;
    const int b = z / ksplit, ks = z - b * ksplit;
    const int b1 = b / bt.n2, b2 = b - b1 * bt.n2;
    A += b1 * bt.sA1 + b2 * bt.sA2;
    B += b1 * bt.sB1 + b2 * bt.sB2;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = ks * kchunk;
    const int ke = min(K, kb + kchunk);

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    double ra[4], rb[4];

    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + r * NT;
            int mm, kk;
            if (!TA) {
                kk = idx & 15;
                mm = idx >> 4;
            } else {
                mm = idx & 63;
                kk = idx >> 6;
            }
            int m = m0 + mm, k = k0 + kk;
            ra[r] = (m < M && k < ke) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.0;
            int nn;
            if (!TB) {
                nn = idx & 63;
                kk = idx >> 6;
            } else {
                kk = idx & 15;
                nn = idx >> 4;
            }
            int n = n0 + nn;
            k = k0 + kk;
            rb[r] = (n < N && k < ke) ? (TB ? B[(long long)n * ldb + k] : B[(long long)k * ldb + n]) : 0.0;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = tid + r * NT;
            if (!TA)
                As[idx & 15][idx >> 4] = ra[r];
            else
                As[idx >> 6][idx & 63] = ra[r];
            if (!TB)
                Bs[idx >> 6][idx & 63] = rb[r];
            else
                Bs[idx & 15][idx >> 4] = rb[r];
        }
    };

    if (kb < ke) load(kb);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        store();
        __syncthreads();
        if (k0 + BK < ke) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }

    const int nbatch = gridDim.z / ksplit;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            if (ksplit == 1) {
                double *c = C + b1 * bt.sC1 + b2 * bt.sC2 + (long long)m * ldc + n;
                *c = (beta == 0.0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
            } else {
                ws[((long long)(ks * nbatch + b) * M + m) * N + n] = acc[i][j];
            }
        }
    }
}

__global__ void splitk_reduce(int M, int N, int nbatch, int ksplit, const double *__restrict__ ws,
                              double alpha, double beta, double *__restrict__ C, long long ldc, Batch bt)
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
        double *c = C + b1 * bt.sC1 + b2 * bt.sC2 + (long long)m * ldc + n;
        *c = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *c);
    }
}

// ---------------------------------------------------------------- Cholesky

// One launch per column k.  Warp w of each block owns row i; lanes split the
// dot product over j < k.  The diagonal of L is kept in dg[] until the end so
// that G[k][k] stays readable by every block of the launch.
__global__ void chol_column(double *G, int n, int k, double *dg, int *flag)
{
    __shared__ double s_lkk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (warp == 0) {
        double s = 0.0;
        for (int j = lane; j < k; j += 32) s = fma(G[(long long)k * n + j], G[(long long)k * n + j], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            double d = G[(long long)k * n + k] - s;
            if (!(d > 0.0)) {
                if (blockIdx.x == 0) atomicCAS(flag, 0, k + 1);
                d = 1.0;
            }
            s_lkk = sqrt(d);
            if (blockIdx.x == 0) dg[k] = s_lkk;
        }
    }
    __syncthreads();
    const double lkk = s_lkk;
    for (int i = k + 1 + blockIdx.x * nw + warp; i < n; i += gridDim.x * nw) {
        double s = 0.0;
        for (int j = lane; j < k; j += 32) s = fma(G[(long long)i * n + j], G[(long long)k * n + j], s);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) G[(long long)i * n + k] = (G[(long long)i * n + k] - s) / lkk;
    }
}

__global__ void chol_finish(double *G, int n, const double *dg)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        G[(long long)i * n + i] = dg[i];
}

// Linv[i][c] (lower) = column c of L^-1 by forward substitution; thread per column.
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

// ---------------------------------------------------------------- Jacobi

__device__ __forceinline__ int rr_pos(int i, int r, int kk)
{
    return i == 0 ? 0 : ((i - 1 + r) % (kk - 1)) + 1;
}

__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

constexpr int JACOBI_MAX_SWEEPS = 60;

__global__ void __launch_bounds__(1024)
    jacobi_kernel(double *H, int k, double *w, double *Yout, double *Y, int *flag)
{
    extern __shared__ double smem[];
    __shared__ double red[33];
    const int kk = k + (k & 1);
    const int np = kk / 2;
    double *cs = smem;
    double *sn = smem + np;
    int *pp = (int *)(sn + np);
    int *qq = pp + np;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int idx = tid; idx < k * k; idx += nt) Y[idx] = (idx / k == idx % k) ? 1.0 : 0.0;
    __syncthreads();

    bool done = (k <= 1);
    for (int sweep = 0; sweep < JACOBI_MAX_SWEEPS && !done; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int idx = tid; idx < k * k; idx += nt) {
            double h = H[idx];
            tot += h * h;
            if (idx / k != idx % k) off += h * h;
        }
        off = block_sum(off, red);
        tot = block_sum(tot, red);
        if (off <= 1e-30 * tot || tot == 0.0) {
            done = true;
            break;
        }
        for (int r = 0; r < kk - 1; ++r) {
            for (int idx = tid; idx < np; idx += nt) {
                int a = rr_pos(idx, r, kk), b = rr_pos(kk - 1 - idx, r, kk);
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                if (q < k) {
                    double hpq = H[p * k + q];
                    if (hpq != 0.0) {
                        double tau = (H[q * k + q] - H[p * k + p]) / (2.0 * hpq);
                        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                pp[idx] = p;
                qq[idx] = q;
                cs[idx] = c;
                sn[idx] = s;
            }
            __syncthreads();
            // rows p, q <- J^T rows
            for (int t = tid; t < np * k; t += nt) {
                int idx = t / k, j = t - idx * k;
                int p = pp[idx], q = qq[idx];
                if (q >= k || sn[idx] == 0.0) continue;
                double c = cs[idx], s = sn[idx];
                double hp = H[p * k + j], hq = H[q * k + j];
                H[p * k + j] = c * hp - s * hq;
                H[q * k + j] = s * hp + c * hq;
            }
            __syncthreads();
            // columns p, q of H and of Y <- cols J
            for (int t = tid; t < np * k; t += nt) {
                int i = t / np, idx = t - i * np;
                int p = pp[idx], q = qq[idx];
                if (q >= k || sn[idx] == 0.0) continue;
                double c = cs[idx], s = sn[idx];
                double hp = H[i * k + p], hq = H[i * k + q];
                H[i * k + p] = c * hp - s * hq;
                H[i * k + q] = s * hp + c * hq;
                double yp = Y[i * k + p], yq = Y[i * k + q];
                Y[i * k + p] = c * yp - s * yq;
                Y[i * k + q] = s * yp + c * yq;
            }
            __syncthreads();
        }
    }
    if (!done && tid == 0) atomicExch(flag, 1);
    __syncthreads();
    // sort ascending by rank (ties by index)
    for (int i = tid; i < k; i += nt) {
        double wi = H[i * k + i];
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            double wj = H[j * k + j];
            rank += (wj < wi || (wj == wi && j < i)) ? 1 : 0;
        }
        w[rank] = wi;
        for (int row = 0; row < k; ++row) Yout[row * k + rank] = Y[row * k + i];
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

}  // namespace

void dgemm(Prof &prof, cudaStream_t st, const char *name, bool ta, bool tb, int M, int N, int K,
           double alpha, const double *A, long long lda, const double *B, long long ldb, double beta,
           double *C, long long ldc, const Batch &bt, double *ws, size_t ws_elems)
{
    if (M <= 0 || N <= 0 || bt.count() <= 0) return;
    const int nb = bt.count();
    if (K <= 0) {
        // C = beta * C: run with zero-length K through the kernel (acc = 0)
        K = 0;
    }
    long long tiles = (long long)cdiv(M, BM) * cdiv(N, BN) * nb;
    int ksplit = 1;
    const long long target = 4 * 152;
    if (ws && tiles < target && K >= 4 * 256) {
        long long want = std::min<long long>((target + tiles - 1) / tiles, K / 256);
        long long cap = (long long)(ws_elems / ((size_t)nb * M * N));
        ksplit = (int)std::max<long long>(1, std::min(want, cap));
        ksplit = std::min(ksplit, 65535 / nb);
        ksplit = std::max(ksplit, 1);
    }
    int kchunk = K;
    if (ksplit > 1) {
        kchunk = (int)(((K + ksplit - 1) / ksplit + BK - 1) / BK * BK);
        ksplit = (K + kchunk - 1) / kchunk;
    }
    TR_REQUIRE((long long)nb * ksplit <= 65535, TR_EINVAL, "dgemm: batch too large");
    TR_REQUIRE(cdiv(M, BM) <= 65535, TR_EINVAL, "dgemm: M too large");
    dim3 grid(cdiv(N, BN), cdiv(M, BM), nb * ksplit);
    double flops = 2.0 * M * N * (double)K * nb;
    double bytes = 8.0 * ((double)M * K + (double)K * N + 2.0 * M * N) * nb;
    int tok = prof.begin(st, name, flops, bytes);
    if (!ta && !tb)
        dgemm_kernel<false, false><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    else if (!ta && tb)
        dgemm_kernel<false, true><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    else if (ta && !tb)
        dgemm_kernel<true, false><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    else
        dgemm_kernel<true, true><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, bt, ksplit, kchunk, ws);
    TR_CUDA(cudaGetLastError());
    if (ksplit > 1) {
        prof.launches += 1;
        long long tot = (long long)nb * M * N;
        int blocks = (int)std::min<long long>(cdiv(tot, 256), 4096);
        splitk_reduce<<<blocks, 256, 0, st>>>(M, N, nb, ksplit, ws, alpha, beta, C, ldc, bt);
        TR_CUDA(cudaGetLastError());
    }
    prof.end(st, tok);
}

void cholesky(Prof &prof, cudaStream_t st, double *G, int n, int *flag)
{
    if (n <= 0) return;
    double *dg = nullptr;
    TR_CUDA(cudaMallocAsync(&dg, sizeof(double) * n, st));
    int tok = prof.begin(st, "cholesky", n * (double)n * n / 3.0, 8.0 * n * n);
    for (int k = 0; k < n; ++k) {
        int rows = n - k - 1;
        int blocks = std::max(1, std::min(1024, (rows + 7) / 8));
        chol_column<<<blocks, 256, 0, st>>>(G, n, k, dg, flag);
        prof.launches += 1;
    }
    chol_finish<<<cdiv(n, 256), 256, 0, st>>>(G, n, dg);
    TR_CUDA(cudaGetLastError());
    prof.end(st, tok);
    TR_CUDA(cudaFreeAsync(dg, st));
}

void chol_inverse(Prof &prof, cudaStream_t st, const double *L, int n, double *Ginv, double *work)
{
    if (n <= 0) return;
    TR_LAUNCH(prof, st, "tri_inverse", n * (double)n * n / 3.0, 8.0 * n * n,
              tri_inverse_cols<<<cdiv(n, 64), 64, 0, st>>>(L, n, work));
    // Ginv = Linv^T Linv
    dgemm(prof, st, "metric_inverse", true, false, n, n, n, 1.0, work, n, work, n, 0.0, Ginv, n,
          Batch(), nullptr, 0);
}

void jacobi_eigh(Prof &prof, cudaStream_t st, double *H, int k, double *w, double *Y, double *work,
                 int *flag)
{
    if (k <= 0) return;
    int kk = k + (k & 1);
    size_t sm = (size_t)(kk / 2) * (2 * sizeof(double) + 2 * sizeof(int));
    TR_REQUIRE(sm <= 48 * 1024, TR_EINVAL, "jacobi: subspace too large");
    TR_LAUNCH(prof, st, "jacobi_eigh", 0, 0,
              jacobi_kernel<<<1, 1024, sm, st>>>(H, k, w, Y, work, flag));
}

void sum_rows(Prof &prof, cudaStream_t st, const double *a, int nrows, int n, double *out)
{
    if (n <= 0) return;
    TR_LAUNCH(prof, st, "sum_rows", 0, 0, sum_rows_kernel<<<cdiv(n, 256), 256, 0, st>>>(a, nrows, n, out));
}

}  // namespace tr
