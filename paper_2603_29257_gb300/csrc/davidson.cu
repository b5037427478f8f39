// Davidson diagonalisation of the TDA-risp matrix (Sec. 3.3).
//
// Standard block Davidson with everything on the GPU in FP64: subspace
// matrix H = 1/2 (V W^T + W V^T) updated by rows, eigen-decomposition by a
// one-block parallel Jacobi, Ritz vectors and residuals by GEMMs, diagonal
// preconditioner, two passes of block classical Gram-Schmidt against V and a
// Cholesky-QR (twice) inside the new block, with vectors whose norm after
// projection falls below 1e-6 dropped.  When the subspace would exceed
// max_space the solver restarts from the current Ritz vectors and recomputes
// A V for them, as the paper's memory-driven restart does (Sec. 3.3).
// Convergence: every one of the nstates residual 2-norms below tol.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>

#include "ctx.cuh"
#include "ozgemm.cuh"

namespace tr {
namespace {

constexpr double DROP_NORM = 1e-6;
// a block kept at least this fraction of its length (1/sqrt 2) in the first
// Gram-Schmidt pass is orthogonal to V to working precision already: the
// second pass is skipped ("twice is enough": Kahan and Parlett's criterion,
// as analysed by Daniel, Gragg, Kaufman and Stewart)
constexpr double REORTH_KEEP = 0.70710678118654752440;
constexpr double PRECOND_FLOOR = 1e-8;


__global__ void set_unit_rows(double *V, const int *idx, int n, long long nov)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) V[(long long)r * nov + idx[r]] = 1.0;
}

// Selection of the initial guess: the b smallest keys (value, index) in
// lexicographic order (equal values: lower index first), the order a stable
// sort of the diagonal gives.  Stage 1: every CTA takes b times the smallest key
// of its segment above the last one taken (values v[t], indices t, or the
// candidates of stage 1 with their indices ix); stage 2 is the same over the
// candidates in one CTA.  Exhausted segments add (+inf, -1).
constexpr int SEL_THREADS = 1024, SEL_MAX_B = 512;

__device__ __forceinline__ bool key_less(double va, double ia, double vb, double ib)
{
    return va < vb || (va == vb && ia < ib);
}

__global__ void __launch_bounds__(SEL_THREADS)
    select_smallest(const double *__restrict__ v, const double *__restrict__ ix, long long n, long long seg, int b,
                    double *__restrict__ out_v, double *__restrict__ out_i)
{
    __shared__ double sv[SEL_THREADS / 32], si[SEL_THREADS / 32];
    __shared__ double last_v, last_i;
    const long long s0 = (long long)blockIdx.x * seg, s1 = min(n, s0 + seg);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        last_v = -INFINITY;
        last_i = -2.0;
    }
    __syncthreads();
    for (int r = 0; r < b; ++r) {
        const double lv = last_v, li = last_i;
        double bv = INFINITY, bi = -1.0;
        for (long long t = s0 + threadIdx.x; t < s1; t += SEL_THREADS) {
            const double x = v[t], xi = ix ? ix[t] : (double)t;
            if (xi >= 0.0 && key_less(lv, li, x, xi) && key_less(x, xi, bv, bi < 0.0 ? INFINITY : bi)) {
                bv = x;
                bi = xi;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o), oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (oi >= 0.0 && (bi < 0.0 || key_less(ov, oi, bv, bi))) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            sv[warp] = bv;
            si[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
            bv = lane < SEL_THREADS / 32 ? sv[lane] : INFINITY;
            bi = lane < SEL_THREADS / 32 ? si[lane] : -1.0;
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, bv, o), oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (oi >= 0.0 && (bi < 0.0 || key_less(ov, oi, bv, bi))) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                out_v[(long long)blockIdx.x * b + r] = bv;
                out_i[(long long)blockIdx.x * b + r] = bi;
                if (bi >= 0.0) {
                    last_v = bv;
                    last_i = bi;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void sel_to_int(const double *__restrict__ ix, int b, int *__restrict__ idx)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < b) idx[r] = (int)ix[r];
}

// H[k0+i][j] = H[j][k0+i] = (A1[i][j] + A2[i][j]) / 2 for i < p, j < k0 + p; each
// unordered pair written once.
__global__ void h_insert(double *H, int ldh, const double *A1, const double *A2, int p, int k, int k0)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j >= k || i >= p) return;
    int row = k0 + i;
    if (j >= k0 && j > row) return;
    double v = 0.5 * (A1[(long long)i * k + j] + A2[(long long)i * k + j]);
    H[(long long)row * ldh + j] = v;
    H[(long long)j * ldh + row] = v;
}

__global__ void copy_sub(const double *H, int ldh, double *Hw, int k)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (j < k) Hw[(long long)i * k + j] = H[(long long)i * ldh + j];
}

// R[r] -= theta[r] X[r]; part[bx][r] = partial sum of R^2
__global__ void ritz_resid(double *R, const double *X, const double *theta, int n, long long nov, double *part)
{
    __shared__ double red[32];
    const int r = blockIdx.y;
    const double th = theta[r];
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nov; t += (long long)gridDim.x * blockDim.x) {
        double v = R[(long long)r * nov + t] - th * X[(long long)r * nov + t];
        R[(long long)r * nov + t] = v;
        s = fma(v, v, s);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * n + r] = s;
    }
}

__global__ void row_sumsq(const double *A, int n, long long nov, double *part)
{
    __shared__ double red[32];
    const int r = blockIdx.y;
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nov; t += (long long)gridDim.x * blockDim.x) {
        double v = A[(long long)r * nov + t];
        s = fma(v, v, s);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * n + r] = s;
    }
}

__global__ void finish_norms(const double *part, int nblk, int n, double *out)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(long long)b * n + r];
    out[r] = sqrt(s);
}

__global__ void precond(double *T, const double *R, const double *D, const double *theta, const int *idx,
                        int p, long long nov, double floor_)
{
    const int q = blockIdx.y;
    const int r = idx[q];
    const double th = theta[r];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nov; t += (long long)gridDim.x * blockDim.x) {
        double den = th - D[t];
        if (fabs(den) < floor_) den = den < 0.0 ? -floor_ : floor_;
        T[(long long)q * nov + t] = R[(long long)r * nov + t] / den;
    }
}

__global__ void row_scale_inv(double *A, int p, long long nov, const double *norms)
{
    const int q = blockIdx.y;
    const double s = norms[q] > 0.0 ? 1.0 / norms[q] : 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nov; t += (long long)gridDim.x * blockDim.x)
        A[(long long)q * nov + t] *= s;
}

// Gram matrix of p <= 64 rows of length n (FP64), the pairs i <= j only: CTA b
// sums k over its chunk for one pair per thread (up to GR_PAIRS per thread),
// 32-value tiles of the rows staged in shared memory as [k][i]; gram_finish adds
// the CTAs' partial sums and fills both triangles.
constexpr int GR_TILE = 32, GR_THREADS = 256, GR_PAIRS = (64 * 65 / 2 + GR_THREADS - 1) / GR_THREADS;

__global__ void __launch_bounds__(GR_THREADS)
    gram_partial(const double *__restrict__ A, int p, long long n, long long chunk, double *__restrict__ part)
{
    __shared__ double As[GR_TILE][65];
    __shared__ unsigned char pi[64 * 65 / 2], pj[64 * 65 / 2];
    const int npair = p * (p + 1) / 2;
    for (int q = threadIdx.x; q < npair; q += GR_THREADS) {
        int i = 0, r = q;
        while (r >= p - i) {
            r -= p - i;
            ++i;
        }
        pi[q] = (unsigned char)i;
        pj[q] = (unsigned char)(i + r);
    }
    double acc[GR_PAIRS];
#pragma unroll
    for (int u = 0; u < GR_PAIRS; ++u) acc[u] = 0.0;
    const long long k0 = (long long)blockIdx.x * chunk, k1 = min(n, k0 + chunk);
    __syncthreads();
    for (long long kt = k0; kt < k1; kt += GR_TILE) {
        for (int e = threadIdx.x; e < p * GR_TILE; e += GR_THREADS) {
            const int i = e / GR_TILE, c = e - i * GR_TILE;
            const long long k = kt + c;
            As[c][i] = k < k1 ? A[(long long)i * n + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < GR_PAIRS; ++u) {
            const int q = threadIdx.x + u * GR_THREADS;
            if (q < npair) {
                const int i = pi[q], j = pj[q];
                double a = acc[u];
#pragma unroll 8
                for (int c = 0; c < GR_TILE; ++c) a = fma(As[c][i], As[c][j], a);
                acc[u] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < GR_PAIRS; ++u) {
        const int q = threadIdx.x + u * GR_THREADS;
        if (q < npair) part[(long long)blockIdx.x * npair + q] = acc[u];
    }
}

__global__ void gram_finish(const double *__restrict__ part, int nb, int p, double *__restrict__ S)
{
    const int npair = p * (p + 1) / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npair; q += gridDim.x * blockDim.x) {
        int i = 0, r = q;
        while (r >= p - i) {
            r -= p - i;
            ++i;
        }
        const int j = i + r;
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[(long long)b * npair + q];
        S[i * p + j] = s;
        S[j * p + i] = s;
    }
}

// dst[l][k] = sum_m C[l][m] src[m][k] for p <= PM (FP64): one column k per thread,
// the p x p coefficients in shared memory
template <int PM>
__global__ void __launch_bounds__(256)
    apply_small(const double *__restrict__ C, int p, const double *__restrict__ src, long long n,
                double *__restrict__ dst)
{
    __shared__ double Cs[PM * PM];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) Cs[e] = C[e];
    __syncthreads();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double x[PM];
#pragma unroll
        for (int m = 0; m < PM; ++m) x[m] = m < p ? src[(long long)m * n + k] : 0.0;
#pragma unroll
        for (int l = 0; l < PM; ++l) {
            if (l >= p) break;
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < PM; ++m)
                if (m < p) s = fma(Cs[l * p + m], x[m], s);
            dst[(long long)l * n + k] = s;
        }
    }
}

// Orthonormal combinations of p vectors from their Gram matrix S (p <= 64):
// Gc[l][:] are the coefficients of the l-th accepted vector; vectors whose
// residual squared norm after projection is below drop2 are skipped.
__global__ void cholqr_coef(const double *S, int p, double drop2, double *Gc, int *nkeep)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double cl[64];
    int nacc = 0;
    for (int j = 0; j < p; ++j) {
        for (int l = 0; l < nacc; ++l) {
            double s = 0.0;
            for (int m = 0; m <= j; ++m) s = fma(Gc[l * p + m], S[m * p + j], s);
            cl[l] = s;
        }
        double r2 = S[j * p + j];
        for (int l = 0; l < nacc; ++l) r2 -= cl[l] * cl[l];
        if (!(r2 > drop2)) continue;
        double inv = 1.0 / sqrt(r2);
        for (int m = 0; m < p; ++m) {
            double g = (m == j) ? 1.0 : 0.0;
            for (int l = 0; l < nacc; ++l) g -= cl[l] * Gc[l * p + m];
            Gc[nacc * p + m] = g * inv;
        }
        ++nacc;
    }
    // rows past the accepted ones produce zero vectors
    for (int l = nacc; l < p; ++l)
        for (int m = 0; m < p; ++m) Gc[l * p + m] = 0.0;
    *nkeep = nacc;
}

// sign convention: largest-magnitude component positive (ties: lowest index)
// the largest-magnitude component of row r of X made positive (ties: lower
// index); row r of X2 (optional) takes the same sign
__global__ void sign_fix(double *X, long long nov, double *X2)
{
    __shared__ double bv[1024];
    __shared__ long long bi[1024];
    const int r = blockIdx.x;
    double best = -1.0;
    long long bidx = 0;
    for (long long t = threadIdx.x; t < nov; t += blockDim.x) {
        double a = fabs(X[(long long)r * nov + t]);
        if (a > best) {
            best = a;
            bidx = t;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int s = blockDim.x / 2; s; s >>= 1) {
        if (threadIdx.x < s) {
            double o = bv[threadIdx.x + s];
            long long oi = bi[threadIdx.x + s];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    __shared__ double s_sg;
    if (threadIdx.x == 0) s_sg = X[(long long)r * nov + bi[0]] < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    const double sg = s_sg;
    for (long long t = threadIdx.x; t < nov; t += blockDim.x) X[(long long)r * nov + t] *= sg;
    if (X2)
        for (long long t = threadIdx.x; t < nov; t += blockDim.x) X2[(long long)r * nov + t] *= sg;
}

// ---- full TDDFT (Sec. 2, Eq. tddft): reduced problem and preconditioner

// zero the strict upper triangle of a k x k matrix (the Cholesky factor keeps its input there)
__global__ void zero_upper(double *L, int k)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j < k && j > i) L[(long long)i * k + j] = 0.0;
}

// After a failed factorisation (flag set) the eigensolver gets the identity, so
// that it runs on finite input; the host reports the failure.
__global__ void guard_identity(double *H, int k, const int *flag)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j < k && *flag) H[(long long)i * k + j] = i == j ? 1.0 : 0.0;
}

// theta_i = Omega_i^2 on entry, Omega_i on exit; Cab[r][i] (a, X+Y) scaled by
// Omega^-1/2 and Cab[r][n + i] (b, X-Y) by Omega^-3/2, so that a.b = 1
__global__ void rpa_coef(double *theta, double *Cab, int k, int n, int *flag)
{
    const int i = blockIdx.x;
    const double w2 = theta[i];
    const bool ok = w2 > 0.0;
    const double om = ok ? sqrt(w2) : 1.0;
    const double sa = 1.0 / sqrt(om), sb = sa / om;
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        Cab[(long long)r * 2 * n + i] *= sa;
        Cab[(long long)r * 2 * n + n + i] *= sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        theta[i] = om;
        if (!ok) atomicCAS(flag, 0, -1);
    }
}

// Diagonal preconditioner of the 2 x 2 response system [[D, -W], [-W, D]] for the
// residual pair (R1, R2) of state r = idx[q] (Omega = theta[r]): row q of T gets
// (D R1 + W R2) / (D^2 - W^2), row p + q gets (W R1 + D R2) / (D^2 - W^2); the
// denominator is floored in magnitude
__global__ void precond_rpa(double *T, const double *R, const double *D, const double *theta, const int *idx,
                            int p, int n, long long nov, double floor_)
{
    const int q = blockIdx.y;
    const int r = idx[q];
    const double w = theta[r];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nov; t += (long long)gridDim.x * blockDim.x) {
        const double d = D[t];
        double den = d * d - w * w;
        if (fabs(den) < floor_) den = den < 0.0 ? -floor_ : floor_;
        const double r1 = R[(long long)r * nov + t], r2 = R[(long long)(n + r) * nov + t];
        T[(long long)q * nov + t] = (d * r1 + w * r2) / den;
        T[(long long)(p + q) * nov + t] = (w * r1 + d * r2) / den;
    }
}

struct Events {
    cudaEvent_t e[6];
    Events()
    {
        for (auto &x : e) TR_CUDA(cudaEventCreate(&x));
    }
    ~Events()
    {
        for (auto &x : e) cudaEventDestroy(x);
    }
};

float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float t = 0.f;
    if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return t;
}

}  // namespace

namespace {

// Rows of the Davidson V or W: [0, kd) in HBM, [kd, cap) in pinned host memory
// (Sec. 3.3: vectors that do not fit on the device are kept in host memory and
// uploaded on demand).
struct RowStore {
    long long nov = 0;
    int cap = 0, kd = 0;
    double *dev = nullptr;
    double *host = nullptr;
};

struct PinnedBuf {
    double *p = nullptr;
    ~PinnedBuf()
    {
        if (p) cudaFreeHost(p);
    }
    void alloc(size_t n, const char *what)
    {
        if (n == 0) return;
        cudaError_t e = cudaHostAlloc((void **)&p, n * sizeof(double), cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            throw Error(TR_ENOMEM, std::string("pinned host allocation failed for ") + what);
        }
    }
};

}  // namespace

// One Davidson solve as a resumable state: the driver alternates
//   eig_async (subspace eigenpairs, Ritz vectors, residual norms; asynchronous)
//   check     (after the stream synchronised: convergence / iteration limit)
//   prepare   (restart or new directions into Tn; may synchronise for counts)
//   [A Tn -> Wn for pend_p rows: one matvec, or one graph for many molecules]
//   absorb    (subspace matrix update, rows stored)
// so that many molecules can be advanced in lockstep.
// error code (tensor-core flag) for a W block beyond the sliced copy's exponent
constexpr int TC_ERR_W_RANGE = 99;

struct Dav {
    tr_ctx *c;
    cudaStream_t st;
    long long nov;
    size_t rowb;
    int n, b0, maxsp, max_iter, pmax, cs, kd;
    double tol;
    static constexpr int nblk = 256;
    PinnedBuf Vh, Wh, Wmh;
    RowStore SV, SW, SWm;  // SWm: (A - B) V rows (full TDDFT)
    long long moved = 0;
    double *ws;
    size_t wsn;
    Events ev;
    double t_mv = 0, t_or = 0, t_eig = 0, t_oth = 0;
    int k = 0, nmv = 0, nrestart = 0, it = 0, converged = 0, reorth_skipped = 0;
    bool done = false, eig_timed = false, or_timed = false;
    std::vector<int> unconv;
    // pinned host copies (asynchronous device-to-host): residual norms, Ritz
    // values and flags [eigensolver, tensor core, first keep count, kept count]
    double *h_rn = nullptr, *h_th = nullptr;
    int *h_fl = nullptr;  // [eigensolver, tensor core, first keep count, kept count, reduced problem]
    int pend_p = 0, pend_k0 = 0, pend_max = 0;
    bool pend_restart = false, pend_counted = true;
    // reduction-type subspace products (V^T W, V^T T) on the tensor cores with
    // 7-slice (FP64-level) Ozaki products: forms that use the tensor cores, when
    // every V/W row is on the device and the sliced copies fit the budget
    bool tcd = false;
    // full TDDFT (Sec. 2, Eq. tddft): one basis V for X+Y and X-Y, W = (A + B) V and
    // Wm = (A - B) V, Xr = [X+Y; X-Y] and R = [R1; R2] with 2 n rows each
    bool rpa = false;
    // one-molecule solves decide after the first Gram-Schmidt pass whether a
    // second is needed (a host round trip); batched and served solves, whose
    // molecules overlap on the device, always run both
    bool adaptive = false;
    double *h_nu = nullptr;  // pinned: norms after the first pass

    explicit Dav(tr_ctx *ctx) : c(ctx), st(ctx->st)
    {
        TR_REQUIRE(c->built, TR_EINVAL, "solve: call tr_build first");
        TR_REQUIRE(c->opt.nstates >= 1, TR_EINVAL, "solve: nstates must be >= 1");
        TR_REQUIRE(c->opt.nstates <= 64, TR_EINVAL, "solve: nstates must be <= 64");
        rpa = c->opt.tddft != 0;
        TR_REQUIRE(!rpa || c->opt.precision != TR_MIXED, TR_EINVAL,
                   "solve: full TDDFT needs precision TR_FP64 or TR_FP64_TC");
        nov = c->nov;
        rowb = (size_t)nov * sizeof(double);
        n = (int)std::min<long long>(c->opt.nstates, nov);
        const int nr = rpa ? 2 * n : n;  // Ritz rows: X (TDA), or X+Y and X-Y
        b0 = c->opt.block > 0 ? c->opt.block : 2 * n;
        b0 = (int)std::min<long long>(std::max(b0, n), nov);
        // new rows per step: up to nr (two directions per state in full TDDFT, or
        // the restart basis); the subspace takes a restart basis plus one step
        pmax = std::max(b0, nr);
        maxsp = c->opt.max_space > 0 ? c->opt.max_space : 20 * n;
        maxsp = std::max(maxsp, rpa ? pmax + nr : b0 + n);
        maxsp = (int)std::min<long long>(maxsp, std::max<long long>(nov, b0));
        TR_REQUIRE(!rpa || maxsp >= pmax + nr, TR_EINVAL,
                   "solve: full TDDFT needs nocc * nvir of at least the initial block plus 2 nstates (" +
                       std::to_string(pmax + nr) + ")");
        max_iter = c->opt.max_iter > 0 ? c->opt.max_iter : 200;
        tol = c->opt.tol;
        // pinned host copies, allocated once per context (64 states at most)
        if (!c->h_pin) TR_CUDA(cudaHostAlloc((void **)&c->h_pin, sizeof(double) * 260, cudaHostAllocDefault));
        h_rn = c->h_pin;
        h_th = c->h_pin + 64;
        h_fl = (int *)(c->h_pin + 128);
        h_nu = c->h_pin + 132;  // up to 128 new directions
        std::memset(h_fl, 0, sizeof(int) * 5);

        reserve_matvec(c, pmax);
        c->Tn.alloc((size_t)pmax * nov, &c->budget, "new vectors");
        c->Wn.alloc((size_t)pmax * nov, &c->budget, "new products");
        if (rpa) c->Wnm.alloc((size_t)pmax * nov, &c->budget, "new products");
        c->T.alloc((size_t)pmax * nov, &c->budget, "new vectors");
        c->Tt.alloc((size_t)pmax * nov, &c->budget, "new vectors");
        c->Xr.alloc((size_t)nr * nov, &c->budget, "Ritz vectors");
        c->R.alloc((size_t)nr * nov, &c->budget, "residuals");
        c->part.alloc((size_t)nblk * pmax, &c->budget, "norms");
        c->rn.alloc(pmax, &c->budget, "norms");
        c->idx_dev.alloc(pmax + 2, &c->budget, "indices");
        c->Ss.alloc((size_t)pmax * pmax, &c->budget, "gram");
        c->Gc.alloc((size_t)pmax * pmax, &c->budget, "gram");
        // rows a product is computed for beyond the pending ones must hold finite values
        TR_CUDA(cudaMemsetAsync(c->Tn.p, 0, sizeof(double) * c->Tn.n, st));

        // how many V/W rows fit in HBM; the rest spill to pinned host memory
        // (the rows of the previous solve count as free: kept when the size is unchanged)
        if (!rpa) c->Wm.release();
        cs = std::max(8, pmax);  // staging rows per chunk
        const int nstore = rpa ? 3 : 2;  // row stores: V, W (and Wm)
        const long long held = (long long)sizeof(double) * (long long)(c->V.n + c->W.n + c->Wm.n);
        const long long avail = (long long)c->budget.limit - (long long)c->budget.used + held;
        const long long small = (rpa ? 11LL : 5LL) * maxsp * maxsp * 8 + 2LL * maxsp * pmax * 8 + (64LL << 20);
        kd = (int)std::max<long long>(0, (avail - small) / (long long)(nstore * rowb));
        if (kd < maxsp) kd = (int)std::max<long long>(0, (avail - small - 2LL * cs * rowb) / (long long)(nstore * rowb));
        if (c->opt.dav_dev_rows > 0) kd = std::min(kd, c->opt.dav_dev_rows);
        kd = std::min(kd, maxsp);
        if (kd < maxsp && c->opt.host_budget > 0) {
            const long long hrows = (long long)(c->opt.host_budget / (nstore * rowb));
            maxsp = (int)std::min<long long>(maxsp, kd + hrows);
        }
        TR_REQUIRE(maxsp >= b0 + 1 && maxsp >= n + 1 && (!rpa || maxsp >= pmax + nr), TR_ENOMEM,
                   "solve: device and host budgets leave no room for the Davidson subspace");
        c->V.alloc((size_t)kd * nov, &c->budget, "Davidson V");
        c->W.alloc((size_t)kd * nov, &c->budget, "Davidson W");
        if (rpa) {
            c->Wm.alloc((size_t)kd * nov, &c->budget, "Davidson (A - B) V");
            c->Hsm.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
            c->Lr.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
            c->Mr.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
            c->Qr.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
            c->Ca.alloc((size_t)maxsp * 2 * n, &c->budget, "subspace");
        }
        c->Hs.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
        c->Hw.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
        c->Yev.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
        c->Yw.alloc(eigh_lowest_scratch(maxsp, n) / sizeof(double), &c->budget, "subspace eigensolver scratch");
        c->theta.alloc(maxsp, &c->budget, "subspace");
        c->Cs.alloc((size_t)2 * maxsp * pmax, &c->budget, "projections");
        SV.nov = SW.nov = SWm.nov = nov;
        SV.cap = SW.cap = SWm.cap = maxsp;
        SV.kd = SW.kd = SWm.kd = kd;
        SV.dev = c->V.p;
        SW.dev = c->W.p;
        SWm.dev = c->Wm.p;
        if (kd < maxsp) {
            Vh.alloc((size_t)(maxsp - kd) * nov, "Davidson V");
            Wh.alloc((size_t)(maxsp - kd) * nov, "Davidson W");
            SV.host = Vh.p;
            SW.host = Wh.p;
            if (rpa) {
                Wmh.alloc((size_t)(maxsp - kd) * nov, "Davidson (A - B) V");
                SWm.host = Wmh.p;
            }
            c->stage.reserve((size_t)2 * cs * nov, &c->budget, "spill staging");
            if (!c->cst) TR_CUDA(cudaStreamCreateWithFlags(&c->cst, cudaStreamNonBlocking));
            for (auto &e : c->sev)
                if (!e) TR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        ws = c->ws_split.p;
        wsn = c->ws_split.n;
        if ((c->opt.precision == TR_MIXED || c->opt.precision == TR_FP64_TC) && kd == maxsp) {
            const size_t sv = oz_bytes(maxsp, (int)nov, dav_slices(c)), stn = oz_bytes(pmax, (int)nov, dav_slices(c));
            const size_t svt = oz_bytes(nov, maxsp, dav_slices(c));
            const size_t ssm = oz_bytes(std::max(n, pmax), maxsp, dav_slices(c));
            const size_t nsl = rpa ? 3 : 2;  // sliced row stores: V, W (and Wm), each by rows and by columns
            if (c->budget.used + nsl * sv + nsl * svt + stn + 2 * ssm + (64u << 20) <= c->budget.limit) {
                c->dvs_V.alloc(cdiv(sv, 8), &c->budget, "sliced Davidson V");
                c->dvs_W.alloc(cdiv(sv, 8), &c->budget, "sliced Davidson W");
                c->dvs_T.alloc(cdiv(stn, 8), &c->budget, "sliced new directions");
                c->dvs_Vt.alloc(cdiv(svt, 8), &c->budget, "sliced Davidson V by columns");
                c->dvs_Y.alloc(cdiv(ssm, 8), &c->budget, "sliced subspace vectors");
                c->dvs_C.alloc(cdiv(ssm, 8), &c->budget, "sliced projections");
                TR_CUDA(cudaMemsetAsync(c->dvs_Vt.p, 0, c->dvs_Vt.n * sizeof(double), st));
                oz_bind(c->dz_Vt, c->dvs_Vt.p, nov, maxsp, dav_slices(c));
                oz_set_exponents(st, c->dz_Vt, 1);  // orthonormal rows: every |v| < 2
                c->dvs_Wt.alloc(cdiv(svt, 8), &c->budget, "sliced Davidson W by columns");
                c->dz_eW.alloc(1, &c->budget, "exponent");
                TR_CUDA(cudaMemsetAsync(c->dvs_Wt.p, 0, c->dvs_Wt.n * sizeof(double), st));
                oz_bind(c->dz_Wt, c->dvs_Wt.p, nov, maxsp, dav_slices(c));
                // rows not yet sliced read as zero (tiles extend past the live rows)
                TR_CUDA(cudaMemsetAsync(c->dvs_V.p, 0, c->dvs_V.n * sizeof(double), st));
                TR_CUDA(cudaMemsetAsync(c->dvs_W.p, 0, c->dvs_W.n * sizeof(double), st));
                TR_CUDA(cudaMemsetAsync(c->dvs_T.p, 0, c->dvs_T.n * sizeof(double), st));
                oz_bind(c->dz_V, c->dvs_V.p, maxsp, (int)nov, dav_slices(c));
                oz_bind(c->dz_W, c->dvs_W.p, maxsp, (int)nov, dav_slices(c));
                if (rpa) {
                    c->dvs_Wm.alloc(cdiv(sv, 8), &c->budget, "sliced Davidson (A - B) V");
                    c->dvs_Wmt.alloc(cdiv(svt, 8), &c->budget, "sliced Davidson (A - B) V by columns");
                    c->dz_eWm.alloc(1, &c->budget, "exponent");
                    TR_CUDA(cudaMemsetAsync(c->dvs_Wm.p, 0, c->dvs_Wm.n * sizeof(double), st));
                    TR_CUDA(cudaMemsetAsync(c->dvs_Wmt.p, 0, c->dvs_Wmt.n * sizeof(double), st));
                    oz_bind(c->dz_Wm, c->dvs_Wm.p, maxsp, (int)nov, dav_slices(c));
                    oz_bind(c->dz_Wmt, c->dvs_Wmt.p, nov, maxsp, dav_slices(c));
                }
                tcd = true;
            }
        }
        TR_CUDA(cudaMemsetAsync(c->flag.p, 0, 2 * sizeof(int), st));
        if (rpa) TR_CUDA(cudaMemsetAsync(c->flag.p + 3, 0, sizeof(int), st));
    }
    // C(row r, col i) = sum_k A[ra0 + r][k] B[rb0 + i][k] for r < M, i < N into
    // d[r ldm + i ldn], FP64-level products on the tensor cores, K split over CTAs
    void tc_reduce(const char *name, const OzMat &A, long long ra0, const OzMat &B, long long rb0, int M, int N,
                   double *d, long long ldm, long long ldn)
    {
        OzOut o;
        o.d = d;
        o.ldm = ldm;
        o.ldn = ldn;
        const int tiles = cdiv(M, 128) * cdiv(N, 64);
        int ks = std::max(1, 2 * 152 / tiles);
        ks = (int)std::max<long long>(1, std::min<long long>(ks, (long long)wsn / ((long long)M * N)));
        oz_gemm(c->prof, st, name, A, ra0, 0, 0, 0, B, rb0, 0, 0, 0, M, N, A.nkb, 1, 1, o, c->flag.p + 1, ks, ws, wsn);
    }

    ~Dav()
    {
        // queued copies into the pinned buffers (error paths) finish first
        cudaStreamSynchronize(st);
        if (c->cst) cudaStreamSynchronize(c->cst);
    }
    Dav(const Dav &) = delete;
    Dav &operator=(const Dav &) = delete;

    // f(device pointer, first row, rows) for rows [r0, r1) of S; host rows are
    // staged through two device slots on the copy stream
    template <typename F>
    void for_rows(RowStore &S, int r0, int r1, F &&f)
    {
        int a = r0, b = std::min(r1, S.kd);
        if (a < b) f(S.dev + (long long)a * nov, a, b - a);
        a = std::max(r0, S.kd);
        if (a >= r1) return;
        TR_CUDA(cudaEventRecord(c->sev[4], st));
        TR_CUDA(cudaStreamWaitEvent(c->cst, c->sev[4], 0));
        int i = 0;
        for (int s0 = a; s0 < r1; s0 += cs, ++i) {
            const int nr = std::min(cs, r1 - s0), slot = i & 1;
            double *buf = c->stage.p + (size_t)slot * cs * nov;
            TR_CUDA(cudaStreamWaitEvent(c->cst, c->sev[2 + slot], 0));
            TR_CUDA(cudaMemcpyAsync(buf, S.host + (size_t)(s0 - S.kd) * nov, nr * rowb, cudaMemcpyHostToDevice, c->cst));
            TR_CUDA(cudaEventRecord(c->sev[slot], c->cst));
            TR_CUDA(cudaStreamWaitEvent(st, c->sev[slot], 0));
            f(buf, s0, nr);
            TR_CUDA(cudaEventRecord(c->sev[2 + slot], st));
            moved += (long long)nr * rowb;
        }
    }
    void store_rows(RowStore &S, int r0, int nr, const double *src)
    {
        int a = r0, b = std::min(r0 + nr, S.kd);
        if (a < b)
            TR_CUDA(cudaMemcpyAsync(S.dev + (long long)a * nov, src, (b - a) * rowb, cudaMemcpyDeviceToDevice, st));
        a = std::max(r0, S.kd);
        if (a < r0 + nr) {
            TR_CUDA(cudaMemcpyAsync(S.host + (size_t)(a - S.kd) * nov, src + (long long)(a - r0) * nov,
                                    (r0 + nr - a) * rowb, cudaMemcpyDeviceToHost, st));
            moved += (long long)(r0 + nr - a) * rowb;
        }
    }
    void norms_of(const double *A, int p, double *out)
    {
        TR_LAUNCH(c->prof, st, "row_norms", 0, 8.0 * p * nov,
                  row_sumsq<<<dim3(nblk, p), 256, 0, st>>>(A, p, nov, c->part.p));
        TR_LAUNCH(c->prof, st, "row_norms", 0, 0, finish_norms<<<cdiv(p, 64), 64, 0, st>>>(c->part.p, nblk, p, out));
    }
    // rows/cols k0..k0+p of H for the new vectors Vn (products Wn)
    void h_update(int k0, int p, const double *Vn, const double *Wn)
    {
        Prof &pf = c->prof;
        const int kk = k0 + p;
        double *A1 = c->Cs.p, *A2 = c->Cs.p + (size_t)maxsp * pmax;
        if (tcd) {
            // the new rows join the sliced copies first, then one product over rows 0..kk
            oz_split_rows(pf, st, "oz_split_V", Vn, nov, 1, c->dz_V, k0, p);
            oz_split_rows(pf, st, "oz_split_W", Wn, nov, 1, c->dz_W, k0, p);
            oz_split_cols_fixed(pf, st, "oz_split_Vt", Vn, nov, c->dz_Vt, k0, p);
            // W by columns with one exponent: the first block's largest row exponent
            // plus 8 bits (|A v| for unit v stays far below 256 times the first
            // block's largest entry); a later block beyond it is reported
            oz_col_exponent_update(st, c->dz_W.e + k0, p, k0 == 0, 8, c->dz_Wt, c->dz_eW.p, c->flag.p + 1,
                                   TC_ERR_W_RANGE);
            oz_split_cols_fixed(pf, st, "oz_split_Wt", Wn, nov, c->dz_Wt, k0, p);
            tc_reduce("subspace_H_tc", c->dz_W, 0, c->dz_V, k0, kk, p, A1, 1, kk);  // A1[i][r] = Vn_i . W_r
            tc_reduce("subspace_H_tc", c->dz_V, 0, c->dz_W, k0, kk, p, A2, 1, kk);  // A2[i][r] = Wn_i . V_r
            TR_LAUNCH(pf, st, "subspace_insert", 0, 0,
                      h_insert<<<dim3(cdiv(kk, 128), p), 128, 0, st>>>(c->Hs.p, maxsp, A1, A2, p, kk, k0));
            return;
        }
        h_update_rows(k0, p, Vn, Wn, SW, c->Hs.p);
    }
    // full TDDFT: rows/cols k0..k0+p of M- = V^T (A - B) V for the new vectors Vn
    // (products Wnm); h_update has already sliced Vn
    void h_update_minus(int k0, int p, const double *Vn, const double *Wnm)
    {
        if (!tcd) {
            h_update_rows(k0, p, Vn, Wnm, SWm, c->Hsm.p);
            return;
        }
        Prof &pf = c->prof;
        const int kk = k0 + p;
        double *A1 = c->Cs.p, *A2 = c->Cs.p + (size_t)maxsp * pmax;
        oz_split_rows(pf, st, "oz_split_Wm", Wnm, nov, 1, c->dz_Wm, k0, p);
        oz_col_exponent_update(st, c->dz_Wm.e + k0, p, k0 == 0, 8, c->dz_Wmt, c->dz_eWm.p, c->flag.p + 1,
                               TC_ERR_W_RANGE);
        oz_split_cols_fixed(pf, st, "oz_split_Wmt", Wnm, nov, c->dz_Wmt, k0, p);
        tc_reduce("subspace_H_tc", c->dz_Wm, 0, c->dz_V, k0, kk, p, A1, 1, kk);  // A1[i][r] = Vn_i . Wm_r
        tc_reduce("subspace_H_tc", c->dz_V, 0, c->dz_Wm, k0, kk, p, A2, 1, kk);  // A2[i][r] = Wmn_i . V_r
        TR_LAUNCH(pf, st, "subspace_insert", 0, 0,
                  h_insert<<<dim3(cdiv(kk, 128), p), 128, 0, st>>>(c->Hsm.p, maxsp, A1, A2, p, kk, k0));
    }
    // rows/cols k0..k0+p of the subspace matrix H (ld maxsp) of the products in S, FP64
    void h_update_rows(int k0, int p, const double *Vn, const double *Wn, RowStore &S, double *H)
    {
        Prof &pf = c->prof;
        const int kk = k0 + p;
        double *A1 = c->Cs.p, *A2 = c->Cs.p + (size_t)maxsp * pmax;
        for_rows(S, 0, k0, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "subspace_H", false, true, p, nr, (int)nov, 1.0, Vn, nov, rows, nov, 0.0, A1 + r0, kk,
                  Batch(), ws, wsn);
        });
        dgemm(pf, st, "subspace_H", false, true, p, p, (int)nov, 1.0, Vn, nov, Wn, nov, 0.0, A1 + k0, kk, Batch(), ws, wsn);
        for_rows(SV, 0, k0, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "subspace_H", false, true, p, nr, (int)nov, 1.0, Wn, nov, rows, nov, 0.0, A2 + r0, kk,
                  Batch(), ws, wsn);
        });
        dgemm(pf, st, "subspace_H", false, true, p, p, (int)nov, 1.0, Wn, nov, Vn, nov, 0.0, A2 + k0, kk, Batch(), ws, wsn);
        TR_LAUNCH(pf, st, "subspace_insert", 0, 0,
                  h_insert<<<dim3(cdiv(kk, 128), p), 128, 0, st>>>(H, maxsp, A1, A2, p, kk, k0));
    }
    // Orthonormalise rows src[0:p] into dst[0:p] without waiting on the host:
    // Cholesky-QR with dropping (first pass), then again without dropping; rows
    // past the kept count come out zero.  The kept count lands in h_fl[3] once
    // the stream reaches the end of this work.
    void orthonormal_block_async(double *src, int p, double *dst, double *tmp)
    {
        Prof &pf = c->prof;
        int *cnt = c->idx_dev.p + pmax;
        gram(src, p);
        TR_LAUNCH(pf, st, "cholqr_coef", 0, 0,
                  cholqr_coef<<<1, 1, 0, st>>>(c->Ss.p, p, DROP_NORM * DROP_NORM, c->Gc.p, cnt));
        apply(c->Gc.p, p, src, tmp);
        gram(tmp, p);
        TR_LAUNCH(pf, st, "cholqr_coef", 0, 0, cholqr_coef<<<1, 1, 0, st>>>(c->Ss.p, p, 0.0, c->Gc.p, cnt + 1));
        apply(c->Gc.p, p, tmp, dst);
        TR_CUDA(cudaMemcpyAsync(h_fl + 2, cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    // Ss = A A^T for p rows of A (FP64)
    void gram(const double *A, int p)
    {
        Prof &pf = c->prof;
        const int npair = p * (p + 1) / 2;
        const long long nb = std::min<long long>(std::max<long long>(1, nov / 2048), 4LL * 152);
        if (p > 64 || (size_t)nb * npair > wsn) {
            dgemm(pf, st, "gram", false, true, p, p, (int)nov, 1.0, A, nov, A, nov, 0.0, c->Ss.p, p, Batch(), ws, wsn);
            return;
        }
        const long long chunk = (nov + nb - 1) / nb;
        TR_LAUNCH(pf, st, "gram", (double)npair * 2.0 * nov, 8.0 * p * (double)nov,
                  gram_partial<<<(unsigned)nb, GR_THREADS, 0, st>>>(A, p, nov, chunk, ws));
        TR_LAUNCH(pf, st, "gram", 0, 0, gram_finish<<<cdiv(npair, 128), 128, 0, st>>>(ws, (int)nb, p, c->Ss.p));
    }
    // out = C src for the p x p coefficients C (FP64)
    void apply(const double *C, int p, const double *src, double *out)
    {
        Prof &pf = c->prof;
        const double fl = 2.0 * p * p * (double)nov, by = 16.0 * p * (double)nov;
        const unsigned blocks = (unsigned)std::min<long long>(cdiv(nov, 256), 152LL * 8);
        if (p <= 16)
            TR_LAUNCH(pf, st, "orth_apply", fl, by, apply_small<16><<<blocks, 256, 0, st>>>(C, p, src, nov, out));
        else if (p <= 32)
            TR_LAUNCH(pf, st, "orth_apply", fl, by, apply_small<32><<<blocks, 256, 0, st>>>(C, p, src, nov, out));
        else
            dgemm(pf, st, "orth_apply", false, false, p, (int)nov, p, 1.0, C, p, src, nov, 0.0, out, nov, Batch(),
                  nullptr, 0);
    }

    // initial guess: unit vectors on the b0 smallest e_a - e_i (ties: lower index)
    void guess()
    {
        if (b0 <= SEL_MAX_B) {
            // on the device, no host round trip: segments of >= 4096 entries, at most 1024 of them
            const long long seg = std::max<long long>(4096, (nov + 1023) / 1024);
            const int nseg = (int)((nov + seg - 1) / seg);
            c->gsel.reserve((size_t)2 * nseg * b0 + 2 * (size_t)b0, &c->budget, "guess selection");
            double *cv = c->gsel.p, *ci = cv + (size_t)nseg * b0;
            double *fv = ci + (size_t)nseg * b0, *fi = fv + b0;
            TR_LAUNCH(c->prof, st, "guess_select", 8.0 * nov, 0,
                      select_smallest<<<nseg, SEL_THREADS, 0, st>>>(c->D.p, nullptr, nov, seg, b0, cv, ci));
            TR_LAUNCH(c->prof, st, "guess_select", 0, 0,
                      select_smallest<<<1, SEL_THREADS, 0, st>>>(cv, ci, (long long)nseg * b0, (long long)nseg * b0,
                                                                 b0, fv, fi));
            TR_LAUNCH(c->prof, st, "guess_select", 0, 0, sel_to_int<<<cdiv(b0, 64), 64, 0, st>>>(fi, b0, c->idx_dev.p));
        } else {
            std::vector<double> Dh(nov);
            TR_CUDA(cudaMemcpyAsync(Dh.data(), c->D.p, sizeof(double) * nov, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaStreamSynchronize(st));
            std::vector<int> order(nov);
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Dh[a] < Dh[b]; });
            TR_CUDA(cudaMemcpyAsync(c->idx_dev.p, order.data(), sizeof(int) * b0, cudaMemcpyHostToDevice, st));
            TR_CUDA(cudaStreamSynchronize(st));
        }
        TR_CUDA(cudaMemsetAsync(c->Tn.p, 0, sizeof(double) * (size_t)b0 * nov, st));
        TR_LAUNCH(c->prof, st, "set_unit", 0, 0, set_unit_rows<<<cdiv(b0, 64), 64, 0, st>>>(c->Tn.p, c->idx_dev.p, b0, nov));
        pend_k0 = 0;
        pend_p = pend_max = b0;
        pend_restart = false;
        pend_counted = true;
    }
    // products of the pending rows by this context's own matvec
    void apply_pending()
    {
        TR_CUDA(cudaEventRecord(ev.e[4], st));
        if (rpa) matvec_pm(c, pend_max, c->Tn.p, c->Wn.p, c->Wnm.p);
        else matvec(c, pend_max, c->Tn.p, c->Wn.p);
        TR_CUDA(cudaEventRecord(ev.e[5], st));
    }
    // the kept count of prepare() must be on the host: call after the stream
    // passed that point (any later synchronisation of st)
    void absorb()
    {
        if (!pend_counted) {
            TR_CUDA(cudaStreamSynchronize(st));
            pend_p = h_fl[3];
            pend_counted = true;
            if (pend_p == 0) {
                TR_REQUIRE(!pend_restart, TR_ECUDA, "solve: restart produced an empty subspace");
                done = true;  // no new directions: stagnation
                return;
            }
        }
        h_update(pend_k0, pend_p, c->Tn.p, c->Wn.p);
        if (rpa) h_update_minus(pend_k0, pend_p, c->Tn.p, c->Wnm.p);
        store_rows(SV, pend_k0, pend_p, c->Tn.p);
        store_rows(SW, pend_k0, pend_p, c->Wn.p);
        if (rpa) store_rows(SWm, pend_k0, pend_p, c->Wnm.p);
        k = pend_k0 + pend_p;
        nmv += pend_p;
        pend_p = 0;
    }
    void eig_async()
    {
        if (rpa) {
            eig_rpa_async();
            return;
        }
        Prof &pf = c->prof;
        ++it;
        TR_CUDA(cudaEventRecord(ev.e[0], st));
        TR_LAUNCH(pf, st, "copy_sub", 0, 0, copy_sub<<<dim3(cdiv(k, 128), k), 128, 0, st>>>(c->Hs.p, maxsp, c->Hw.p, k));
        TR_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int), st));
        eigh_lowest(pf, st, c->Hw.p, k, n, c->theta.p, c->Yev.p, k, c->Yw.p, c->flag.p);
        TR_CUDA(cudaEventRecord(ev.e[1], st));
        // Ritz vectors X = Y^T V and residuals R = Y^T W - theta X
        if (tcd) {
            // X[i][col] = sum_r V[r][col] Y[r][i]: rows col of V by columns, columns i
            OzMat Ys;
            oz_bind(Ys, c->dvs_Y.p, n, k, dav_slices(c));
            oz_split(pf, st, "oz_split_Yev", c->Yev.p, 1, k, Ys);
            OzOut o;
            o.d = c->Xr.p;
            o.ldm = 1;
            o.ldn = nov;
            oz_gemm(pf, st, "ritz_tc", c->dz_Vt, 0, 0, 0, 0, Ys, 0, 0, 0, 0, (int)nov, n, Ys.nkb, 1, 1, o, c->flag.p + 1);
            o.d = c->R.p;
            oz_gemm(pf, st, "ritz_tc", c->dz_Wt, 0, 0, 0, 0, Ys, 0, 0, 0, 0, (int)nov, n, Ys.nkb, 1, 1, o, c->flag.p + 1);
        } else {
            for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
                dgemm(pf, st, "ritz", true, false, n, (int)nov, nr, 1.0, c->Yev.p + (long long)r0 * k, k, rows, nov,
                      r0 == 0 ? 0.0 : 1.0, c->Xr.p, nov, Batch(), nullptr, 0);
            });
        }
        if (!tcd) {
            for_rows(SW, 0, k, [&](const double *rows, int r0, int nr) {
                dgemm(pf, st, "ritz", true, false, n, (int)nov, nr, 1.0, c->Yev.p + (long long)r0 * k, k, rows, nov,
                      r0 == 0 ? 0.0 : 1.0, c->R.p, nov, Batch(), nullptr, 0);
            });
        }
        TR_LAUNCH(pf, st, "residual", 0, 24.0 * n * nov,
                  ritz_resid<<<dim3(nblk, n), 256, 0, st>>>(c->R.p, c->Xr.p, c->theta.p, n, nov, c->part.p));
        TR_LAUNCH(pf, st, "residual", 0, 0, finish_norms<<<cdiv(n, 64), 64, 0, st>>>(c->part.p, nblk, n, c->rn.p));
        TR_CUDA(cudaMemcpyAsync(h_rn, c->rn.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaMemcpyAsync(h_th, c->theta.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaMemcpyAsync(h_fl, c->flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaEventRecord(ev.e[2], st));
        eig_timed = true;
    }
    // Full TDDFT (Sec. 2, Eq. tddft; Sec. 3.3): with M+ = V^T (A+B) V and
    // M- = V^T (A-B) V = L L^T, the reduced problem M- M+ a = Omega^2 a is the
    // symmetric L^T M+ L w = Omega^2 w with a = L w; b = M+ a / Omega (so that
    // M- b = Omega a), scaled to a.b = 1.  X+Y = V^T a, X-Y = V^T b and the
    // residuals R1 = (A+B)(X+Y) - Omega (X-Y), R2 = (A-B)(X-Y) - Omega (X+Y).
    void eig_rpa_async()
    {
        Prof &pf = c->prof;
        ++it;
        const int n2 = 2 * n;
        double *Lr = c->Lr.p, *Mr = c->Mr.p, *Qr = c->Qr.p, *Cab = c->Ca.p;
        int *rflag = c->flag.p + 3;
        TR_CUDA(cudaEventRecord(ev.e[0], st));
        TR_LAUNCH(pf, st, "copy_sub", 0, 0, copy_sub<<<dim3(cdiv(k, 128), k), 128, 0, st>>>(c->Hsm.p, maxsp, Lr, k));
        TR_LAUNCH(pf, st, "copy_sub", 0, 0, copy_sub<<<dim3(cdiv(k, 128), k), 128, 0, st>>>(c->Hs.p, maxsp, Mr, k));
        TR_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int), st));
        TR_CUDA(cudaMemsetAsync(rflag, 0, sizeof(int), st));
        cholesky(pf, st, Lr, k, rflag);
        TR_LAUNCH(pf, st, "zero_upper", 0, 0, zero_upper<<<dim3(cdiv(k, 128), k), 128, 0, st>>>(Lr, k));
        dgemm(pf, st, "rpa_reduce", false, false, k, k, k, 1.0, Mr, k, Lr, k, 0.0, Qr, k, Batch(), nullptr, 0);
        dgemm(pf, st, "rpa_reduce", true, false, k, k, k, 1.0, Lr, k, Qr, k, 0.0, c->Hw.p, k, Batch(), nullptr, 0);
        TR_LAUNCH(pf, st, "guard", 0, 0, guard_identity<<<dim3(cdiv(k, 128), k), 128, 0, st>>>(c->Hw.p, k, rflag));
        eigh_lowest(pf, st, c->Hw.p, k, n, c->theta.p, c->Yev.p, k, c->Yw.p, c->flag.p);
        // a = L w into columns 0..n-1 of Cab (ld 2n), b = M+ a into columns n..2n-1
        dgemm(pf, st, "rpa_coef", false, false, k, n, k, 1.0, Lr, k, c->Yev.p, k, 0.0, Cab, n2, Batch(), nullptr, 0);
        dgemm(pf, st, "rpa_coef", false, false, k, n, k, 1.0, Mr, k, Cab, n2, 0.0, Cab + n, n2, Batch(), nullptr, 0);
        TR_LAUNCH(pf, st, "rpa_coef", 0, 0, rpa_coef<<<n, 128, 0, st>>>(c->theta.p, Cab, k, n, rflag));
        TR_CUDA(cudaEventRecord(ev.e[1], st));
        // [X+Y; X-Y] = [a b]^T V in one pass over V; R1 = a^T W, R2 = b^T Wm
        if (tcd) {
            // Cs rows i < 2n with K = r: element (i, r) = Cab[r][i]
            OzMat Ys;
            oz_bind(Ys, c->dvs_Y.p, n2, k, dav_slices(c));
            oz_split(pf, st, "oz_split_Yev", Cab, 1, n2, Ys);
            OzOut o;
            o.d = c->Xr.p;
            o.ldm = 1;
            o.ldn = nov;
            oz_gemm(pf, st, "ritz_tc", c->dz_Vt, 0, 0, 0, 0, Ys, 0, 0, 0, 0, (int)nov, n2, Ys.nkb, 1, 1, o, c->flag.p + 1);
            o.d = c->R.p;
            oz_gemm(pf, st, "ritz_tc", c->dz_Wt, 0, 0, 0, 0, Ys, 0, 0, 0, 0, (int)nov, n, Ys.nkb, 1, 1, o, c->flag.p + 1);
            o.d = c->R.p + (long long)n * nov;
            oz_gemm(pf, st, "ritz_tc", c->dz_Wmt, 0, 0, 0, 0, Ys, n, 0, 0, 0, (int)nov, n, Ys.nkb, 1, 1, o,
                    c->flag.p + 1);
        } else {
        for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "ritz", true, false, n2, (int)nov, nr, 1.0, Cab + (long long)r0 * n2, n2, rows, nov,
                  r0 == 0 ? 0.0 : 1.0, c->Xr.p, nov, Batch(), nullptr, 0);
        });
        for_rows(SW, 0, k, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "ritz", true, false, n, (int)nov, nr, 1.0, Cab + (long long)r0 * n2, n2, rows, nov,
                  r0 == 0 ? 0.0 : 1.0, c->R.p, nov, Batch(), nullptr, 0);
        });
        for_rows(SWm, 0, k, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "ritz", true, false, n, (int)nov, nr, 1.0, Cab + (long long)r0 * n2 + n, n2, rows, nov,
                  r0 == 0 ? 0.0 : 1.0, c->R.p + (long long)n * nov, nov, Batch(), nullptr, 0);
        });
        }
        TR_LAUNCH(pf, st, "residual", 0, 24.0 * n * nov,
                  ritz_resid<<<dim3(nblk, n), 256, 0, st>>>(c->R.p, c->Xr.p + (long long)n * nov, c->theta.p, n, nov,
                                                            c->part.p));
        TR_LAUNCH(pf, st, "residual", 0, 24.0 * n * nov,
                  ritz_resid<<<dim3(nblk, n), 256, 0, st>>>(c->R.p + (long long)n * nov, c->Xr.p, c->theta.p, n, nov,
                                                            c->part.p + (long long)nblk * n));
        TR_LAUNCH(pf, st, "residual", 0, 0, finish_norms<<<cdiv(n, 64), 64, 0, st>>>(c->part.p, 2 * nblk, n, c->rn.p));
        TR_CUDA(cudaMemcpyAsync(h_rn, c->rn.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaMemcpyAsync(h_th, c->theta.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaMemcpyAsync(h_fl, c->flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaMemcpyAsync(h_fl + 4, rflag, sizeof(int), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaEventRecord(ev.e[2], st));
        eig_timed = true;
    }
    // after st synchronised
    void check()
    {
        if (eig_timed) {
            t_eig += elapsed(ev.e[0], ev.e[1]);
            t_oth += elapsed(ev.e[1], ev.e[2]);
            eig_timed = false;
        }
        // a product whose pipeline wait ran out left invalid data behind: report that
        // first, before what the invalid data may have tripped downstream
        TR_REQUIRE(!h_fl[1] || h_fl[1] == TC_ERR_W_RANGE, TR_ETIMEOUT,
                   "solve: a tensor-core pipeline wait ran out (code " + std::to_string(h_fl[1]) + ")");
        TR_REQUIRE(!rpa || h_fl[4] == 0, TR_ECUDA,
                   h_fl[4] < 0 ? "solve: non-positive Omega^2 in the projected full TDDFT problem"
                               : "solve: A - B projected on the subspace is not positive definite");
        TR_REQUIRE(!h_fl[0], TR_ECUDA, "solve: subspace eigensolver did not converge");
        TR_REQUIRE(h_fl[1] != TC_ERR_W_RANGE, TR_ECUDA,
                   "solve: a product block exceeded the exponent range fixed for the sliced W");
        unconv.clear();
        for (int r = 0; r < n; ++r)
            if (!(h_rn[r] < tol)) unconv.push_back(r);
        if (unconv.empty()) {
            converged = 1;
            done = true;
        } else if (it >= max_iter) {
            done = true;
        }
    }
    // asynchronous: the new directions (or the restart basis) go to Tn; their
    // count is read in absorb()
    void prepare()
    {
        Prof &pf = c->prof;
        const int p = (int)unconv.size();
        const int pp = rpa ? 2 * p : p;  // new directions
        const int nr = rpa ? 2 * n : n;  // restart basis: the Ritz vectors (X+Y and X-Y)
        pend_counted = false;
        if (k + pp > maxsp) {
            // restart from the Ritz vectors; A V is recomputed for them (Sec. 3.3)
            orthonormal_block_async(c->Xr.p, nr, c->Tn.p, c->Tt.p);
            pend_k0 = 0;
            pend_max = nr;
            pend_restart = true;
            nrestart += 1;
            return;
        }
        TR_CUDA(cudaMemcpyAsync(c->idx_dev.p, unconv.data(), sizeof(int) * p, cudaMemcpyHostToDevice, st));
        if (rpa)
            TR_LAUNCH(pf, st, "precondition", 0, 48.0 * p * nov,
                      precond_rpa<<<dim3(nblk, p), 256, 0, st>>>(c->T.p, c->R.p, c->D.p, c->theta.p, c->idx_dev.p, p, n,
                                                                  nov, PRECOND_FLOOR));
        else
            TR_LAUNCH(pf, st, "precondition", 0, 32.0 * p * nov,
                      precond<<<dim3(nblk, p), 256, 0, st>>>(c->T.p, c->R.p, c->D.p, c->theta.p, c->idx_dev.p, p, nov,
                                                              PRECOND_FLOOR));
        norms_of(c->T.p, pp, c->rn.p);
        TR_LAUNCH(pf, st, "normalise", 0, 16.0 * pp * nov,
                  row_scale_inv<<<dim3(nblk, pp), 256, 0, st>>>(c->T.p, pp, nov, c->rn.p));
        // two passes of block classical Gram-Schmidt against V[0:k] (the second
        // skipped in one-molecule solves when the first kept every vector long)
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1 && adaptive && pp <= 128) {
                norms_of(c->T.p, pp, c->rn.p);
                TR_CUDA(cudaMemcpyAsync(h_nu, c->rn.p, sizeof(double) * pp, cudaMemcpyDeviceToHost, st));
                TR_CUDA(cudaStreamSynchronize(st));
                if (*std::min_element(h_nu, h_nu + pp) >= REORTH_KEEP) {
                    ++reorth_skipped;
                    break;
                }
            }
            if (tcd) {
                OzMat Ts;
                oz_bind(Ts, c->dvs_T.p, pp, (int)nov, dav_slices(c));
                oz_split(pf, st, "oz_split_T", c->T.p, nov, 1, Ts);
                tc_reduce("orth_project_tc", c->dz_V, 0, Ts, 0, k, pp, c->Cs.p, pp, 1);  // Cs[r][i] = V_r . T_i
            } else {
                for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
                    dgemm(pf, st, "orth_project", false, true, nr, pp, (int)nov, 1.0, rows, nov, c->T.p, nov, 0.0,
                          c->Cs.p + (long long)r0 * pp, pp, Batch(), ws, wsn);
                });
            }
            if (tcd) {
                // T[i][col] -= sum_r V[r][col] Cs[r][i]
                OzMat Css;
                oz_bind(Css, c->dvs_C.p, pp, k, dav_slices(c));
                oz_split(pf, st, "oz_split_Cs", c->Cs.p, 1, pp, Css);
                OzOut o;
                o.d = c->T.p;
                o.ldm = 1;
                o.ldn = nov;
                o.alpha = -1.0;
                o.accumulate = true;
                oz_gemm(pf, st, "orth_update_tc", c->dz_Vt, 0, 0, 0, 0, Css, 0, 0, 0, 0, (int)nov, pp, Css.nkb, 1, 1, o,
                        c->flag.p + 1);
            } else {
                for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
                    dgemm(pf, st, "orth_update", true, false, pp, (int)nov, nr, -1.0, c->Cs.p + (long long)r0 * pp, pp, rows,
                          nov, 1.0, c->T.p, nov, Batch(), nullptr, 0);
                });
            }
        }
        orthonormal_block_async(c->T.p, pp, c->Tn.p, c->Tt.p);
        pend_k0 = k;
        pend_max = pp;
        pend_restart = false;
    }
    // outputs: omega, unit-norm sign-fixed X, residual norms
    // (full TDDFT: X+Y into Xout and X-Y into Xmout, (X+Y).(X-Y) = 1 from the
    // reduced problem, the sign fixed on X+Y)
    int output(double *omega, double *Xout, double *Xmout, double *resid, int on_device, tr_solve_info *info)
    {
        Prof &pf = c->prof;
        if (rpa) {
            TR_LAUNCH(pf, st, "sign_fix", 0, 0, sign_fix<<<n, 1024, 0, st>>>(c->Xr.p, nov, c->Xr.p + (long long)n * nov));
        } else {
            norms_of(c->Xr.p, n, c->rn.p);
            TR_LAUNCH(pf, st, "normalise", 0, 16.0 * n * nov,
                      row_scale_inv<<<dim3(nblk, n), 256, 0, st>>>(c->Xr.p, n, nov, c->rn.p));
            TR_LAUNCH(pf, st, "sign_fix", 0, 0, sign_fix<<<n, 1024, 0, st>>>(c->Xr.p, nov, nullptr));
        }
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        TR_CUDA(cudaMemcpyAsync(omega, c->theta.p, sizeof(double) * n, kind, st));
        if (Xout) TR_CUDA(cudaMemcpyAsync(Xout, c->Xr.p, sizeof(double) * (size_t)n * nov, kind, st));
        if (Xmout && rpa)
            TR_CUDA(cudaMemcpyAsync(Xmout, c->Xr.p + (size_t)n * nov, sizeof(double) * (size_t)n * nov, kind, st));
        if (resid) {
            if (on_device)
                TR_CUDA(cudaMemcpyAsync(resid, h_rn, sizeof(double) * n, cudaMemcpyHostToDevice, st));
            else
                std::copy(h_rn, h_rn + n, resid);
        }
        TR_CUDA(cudaStreamSynchronize(st));
        if (c->cst) TR_CUDA(cudaStreamSynchronize(c->cst));
        if (info) {
            info->niter = it;
            info->nmatvec = nmv;
            info->nrestart = nrestart;
            info->converged = converged;
            info->t_matvec_ms = t_mv;
            info->t_ortho_ms = t_or;
            info->t_eigh_ms = t_eig;
            info->t_other_ms = t_oth;
            info->max_space = maxsp;
            info->dev_rows = kd;
            info->host_bytes_moved = moved;
        }
        return converged ? TR_OK : TR_ENOCONV;
    }
};

int solve(tr_ctx *c, double *omega, double *Xout, double *Xmout, double *resid, int on_device, tr_solve_info *info)
{
    TR_REQUIRE(omega, TR_EINVAL, "solve: omega must not be NULL");
    TR_REQUIRE(!Xmout || c->opt.tddft, TR_EINVAL, "solve: X-Y is returned for tddft = 1 only");
    Dav d(c);
    d.adaptive = true;
    d.guess();
    d.apply_pending();
    d.absorb();
    TR_CUDA(cudaStreamSynchronize(d.st));
    d.t_mv += elapsed(d.ev.e[4], d.ev.e[5]);
    while (!d.done) {
        d.eig_async();
        TR_CUDA(cudaStreamSynchronize(d.st));
        d.check();
        if (d.done) break;
        TR_CUDA(cudaEventRecord(d.ev.e[3], d.st));
        d.prepare();
        d.apply_pending();
        TR_CUDA(cudaStreamSynchronize(d.st));
        d.t_or += elapsed(d.ev.e[3], d.ev.e[4]);
        d.t_mv += elapsed(d.ev.e[4], d.ev.e[5]);
        d.absorb();
    }
    return d.output(omega, Xout, Xmout, resid, on_device, info);
}

// ---------------------------------------------------------------- many molecules

namespace {

// The products of one Davidson step of all molecules as one CUDA graph: each
// molecule's matvec on its own stream, forked from and joined to the batch
// stream, recorded once for a fixed row count and replayed every step (rows
// beyond a molecule's pending count are computed and ignored).
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<int> members;
    int rows_key = -1;
    ~StepGraph()
    {
        if (exec) cudaGraphExecDestroy(exec);
    }
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        members.clear();
    }
};

void capture(StepGraph &g, cudaStream_t s0, std::vector<tr_ctx *> &cs, const std::vector<int> &members,
             const std::vector<int> &rows, cudaEvent_t fork, std::vector<cudaEvent_t> &joins)
{
    TR_CUDA(cudaStreamSynchronize(s0));  // the previous graph has finished before it is replaced
    g.reset();
    // profiling events cannot live inside the graph
    std::vector<bool> prof_on(cs.size());
    for (size_t i = 0; i < cs.size(); ++i) {
        prof_on[i] = cs[i]->prof.enabled;
        cs[i]->prof.flush();
        cs[i]->prof.enabled = false;
    }
    cudaGraph_t graph = nullptr;
    TR_CUDA(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    try {
        TR_CUDA(cudaEventRecord(fork, s0));
        for (int i : members) {
            tr_ctx *c = cs[i];
            TR_CUDA(cudaStreamWaitEvent(c->st, fork, 0));
            matvec(c, rows[i], c->Tn.p, c->Wn.p);
            TR_CUDA(cudaEventRecord(joins[i], c->st));
            TR_CUDA(cudaStreamWaitEvent(s0, joins[i], 0));
        }
    } catch (...) {
        cudaStreamEndCapture(s0, &graph);
        if (graph) cudaGraphDestroy(graph);
        for (size_t i = 0; i < cs.size(); ++i) cs[i]->prof.enabled = prof_on[i];
        throw;
    }
    err = cudaStreamEndCapture(s0, &graph);
    for (size_t i = 0; i < cs.size(); ++i) cs[i]->prof.enabled = prof_on[i];
    TR_CUDA(err);
    err = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    TR_CUDA(err);
    g.members = members;
}

// Pick the tensor-core tile width of each reduced-precision context by timing
// one product of `rows` vectors with 64- and 128-wide tiles.
void autotune(std::vector<tr_ctx *> &cs, const std::vector<int> &rows)
{
    cudaEvent_t a, b;
    TR_CUDA(cudaEventCreate(&a));
    TR_CUDA(cudaEventCreate(&b));
    for (size_t i = 0; i < cs.size(); ++i) {
        tr_ctx *c = cs[i];
        if (c->opt.precision != TR_MIXED || !c->k_active) continue;
        float best = 1e30f;
        int pick = 128;
        for (int bn : {128, 64}) {
            c->tc_bn = bn;
            matvec(c, rows[i], c->Tn.p, c->Wn.p);  // warm
            TR_CUDA(cudaEventRecord(a, c->st));
            matvec(c, rows[i], c->Tn.p, c->Wn.p);
            TR_CUDA(cudaEventRecord(b, c->st));
            TR_CUDA(cudaEventSynchronize(b));
            float ms = elapsed(a, b);
            if (ms < best) {
                best = ms;
                pick = bn;
            }
        }
        c->tc_bn = pick;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
}

}  // namespace

int solve_batch(tr_ctx **ctxs, int nb, double **omega, double **X, double **resid, int on_device,
                tr_solve_info *infos, int autotune_tiles)
{
    TR_REQUIRE(ctxs && nb > 0 && omega, TR_EINVAL, "solve_batch: empty batch");
    std::vector<tr_ctx *> cs(ctxs, ctxs + nb);
    for (int i = 0; i < nb; ++i) {
        TR_REQUIRE(cs[i] && cs[i]->built, TR_EINVAL, "solve_batch: every context must be built");
        TR_REQUIRE(!cs[i]->opt.tddft, TR_EINVAL, "solve_batch: full TDDFT (tddft = 1) runs through tr_solve only");
        TR_REQUIRE(omega[i], TR_EINVAL, "solve_batch: omega must not be NULL");
        for (int j = 0; j < i; ++j) TR_REQUIRE(cs[i] != cs[j], TR_EINVAL, "solve_batch: a context appears twice");
        TR_REQUIRE(cs[i]->device == cs[0]->device, TR_EINVAL, "solve_batch: contexts on different devices");
    }
    // every molecule works on a stream of its own for the duration of the call
    struct Streams {
        std::vector<tr_ctx *> &cs;
        std::vector<cudaStream_t> orig, own;
        cudaStream_t s0 = nullptr;
        cudaEvent_t fork = nullptr, done = nullptr;
        std::vector<cudaEvent_t> joins;
        explicit Streams(std::vector<tr_ctx *> &c) : cs(c) {}
        ~Streams()
        {
            for (size_t i = 0; i < own.size(); ++i) {
                cudaStreamSynchronize(own[i]);
                cs[i]->st = orig[i];
                cudaStreamDestroy(own[i]);
            }
            for (auto e : joins) cudaEventDestroy(e);
            if (fork) cudaEventDestroy(fork);
            if (done) cudaEventDestroy(done);
            if (s0) {
                cudaStreamSynchronize(s0);
                cudaStreamDestroy(s0);
            }
        }
    } S(cs);
    for (int i = 0; i < nb; ++i) TR_CUDA(cudaStreamSynchronize(cs[i]->st));
    TR_CUDA(cudaStreamCreateWithFlags(&S.s0, cudaStreamNonBlocking));
    TR_CUDA(cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming));
    TR_CUDA(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
    for (int i = 0; i < nb; ++i) {
        cudaStream_t s;
        TR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        S.orig.push_back(cs[i]->st);
        S.own.push_back(s);
        cs[i]->st = s;
        cudaEvent_t e;
        TR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        S.joins.push_back(e);
    }
    std::vector<std::unique_ptr<Dav>> ds;
    for (int i = 0; i < nb; ++i) ds.emplace_back(new Dav(cs[i]));
    std::vector<int> init_rows(nb), step_rows(nb);
    for (int i = 0; i < nb; ++i) {
        init_rows[i] = ds[i]->b0;
        step_rows[i] = ds[i]->n;
    }
    if (autotune_tiles)
        autotune(cs, step_rows);
    else
        for (int i = 0; i < nb; ++i) matvec(cs[i], step_rows[i], cs[i]->Tn.p, cs[i]->Wn.p);  // loads kernels before capture

    cudaEvent_t g0, g1;
    TR_CUDA(cudaEventCreate(&g0));
    TR_CUDA(cudaEventCreate(&g1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard()
        {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } eg{g0, g1};
    double graph_ms = 0.0;
    long graph_launches = 0;
    StepGraph gi, gs;
    auto run_graph = [&](StepGraph &g, const std::vector<int> &members) {
        for (int i : members) {
            TR_CUDA(cudaEventRecord(S.joins[i], cs[i]->st));
            TR_CUDA(cudaStreamWaitEvent(S.s0, S.joins[i], 0));
        }
        TR_CUDA(cudaEventRecord(g0, S.s0));
        TR_CUDA(cudaGraphLaunch(g.exec, S.s0));
        TR_CUDA(cudaEventRecord(g1, S.s0));
        TR_CUDA(cudaEventRecord(S.done, S.s0));
        for (int i : members) TR_CUDA(cudaStreamWaitEvent(cs[i]->st, S.done, 0));
        graph_launches += 1;
    };

    std::vector<int> all(nb);
    std::iota(all.begin(), all.end(), 0);
    for (int i = 0; i < nb; ++i) ds[i]->guess();
    capture(gi, S.s0, cs, all, init_rows, S.fork, S.joins);
    run_graph(gi, all);
    for (int i = 0; i < nb; ++i) ds[i]->absorb();
    TR_CUDA(cudaEventSynchronize(g1));
    graph_ms += elapsed(g0, g1);
    gi.reset();

    while (true) {
        std::vector<int> act;
        for (int i = 0; i < nb; ++i)
            if (!ds[i]->done) act.push_back(i);
        if (act.empty()) break;
        for (int i : act) ds[i]->eig_async();
        for (int i : act) {
            TR_CUDA(cudaStreamSynchronize(ds[i]->st));
            ds[i]->check();
        }
        std::vector<int> pend;
        for (int i : act) {
            if (ds[i]->done) continue;
            ds[i]->prepare();
            if (!ds[i]->done) pend.push_back(i);
        }
        if (pend.empty()) continue;
        if (gs.exec == nullptr || gs.members != pend) capture(gs, S.s0, cs, pend, step_rows, S.fork, S.joins);
        run_graph(gs, pend);
        for (int i : pend) ds[i]->absorb();
        TR_CUDA(cudaEventSynchronize(g1));
        graph_ms += elapsed(g0, g1);
    }
    int rc = TR_OK;
    for (int i = 0; i < nb; ++i) {
        ds[i]->t_mv = graph_ms;
        int r = ds[i]->output(omega[i], X ? X[i] : nullptr, nullptr, resid ? resid[i] : nullptr, on_device,
                              infos ? &infos[i] : nullptr);
        if (r != TR_OK) rc = r;
    }
    (void)graph_launches;
    return rc;
}

}  // namespace tr

// ---------------------------------------------------------------- serving runtime
//
// Continuous batching of TDA-risp solves as requests arrive: builder threads
// admit requests strictly in arrival order when their estimated device footprint
// fits in what the server's budget has left (requests larger than the whole
// budget are rejected), create each context on a stream of its own and run
// tr_build, several builds at once; a
// solver thread keeps every built molecule's tensors and Davidson state resident
// and advances all of them in lockstep, the products of one step of all of them
// being one CUDA-graph launch.  Molecules join at the next step after their build
// and leave when converged, returning their memory to the budget; builds overlap
// on the device with the solver's steps.

struct tr_server {
    tr_server_options opt{};
    int device = 0;
    size_t budget = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_submit, cv_ready, cv_mem, cv_result;
    struct Req {
        long long id = 0;
        std::vector<int> Z;
        std::vector<double> xyz, aux, C, eps;
        std::vector<tr_shell> shells;
        std::vector<std::vector<double>> sexp, scoef;
        int nao = 0, nmo = 0, nocc = 0, want_x = 0;
        tr_options o{};
        double t_submit = 0, t_admit = 0, t_built = 0;
        size_t foot = 0;
        tr_ctx *ctx = nullptr;
        cudaStream_t stream = nullptr;
    };
    std::deque<std::unique_ptr<Req>> submitted, ready;
    std::deque<tr_result> results;
    long long next_id = 1;
    long long pop_seq = 0, admit_seq = 0;  // admission turns in arrival order
    int outstanding = 0;
    bool stop = false;
    std::vector<std::thread> builders;
    std::thread solver;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace tr {
namespace {

void release_request(tr_server *S, tr_server::Req *r)
{
    if (r->ctx) {
        cudaStreamSynchronize(r->stream);
        tr_destroy(r->ctx);
        r->ctx = nullptr;
    }
    if (r->stream) {
        cudaStreamDestroy(r->stream);
        r->stream = nullptr;
    }
}

void post_result(tr_server *S, tr_result &res)
{
    std::lock_guard<std::mutex> lk(S->mu);
    S->results.push_back(res);
    S->cv_result.notify_all();
}

void fail(tr_server *S, tr_server::Req *r, int code, const std::string &msg)
{
    tr_result res;
    std::memset(&res, 0, sizeof res);
    res.id = r->id;
    res.status = code;
    res.t_submit = r->t_submit;
    res.t_admit = r->t_admit;
    res.t_built = r->t_built;
    res.t_done = S->now();
    std::strncpy(res.error, msg.c_str(), sizeof(res.error) - 1);
    post_result(S, res);
}

void builder_loop(tr_server *S)
{
    cudaSetDevice(S->device);
    while (true) {
        std::unique_ptr<tr_server::Req> r;
        long long seq = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_submit.wait(lk, [&] { return S->stop || !S->submitted.empty(); });
            if (S->stop) return;
            r = std::move(S->submitted.front());
            S->submitted.pop_front();
            seq = S->pop_seq++;
        }
        int rc = TR_OK;
        std::string msg;
        bool turn_taken = false;
        // waits for this request's admission turn; fits: whether it may take memory
        auto take_turn = [&](bool fits) -> bool {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_mem.wait(lk, [&] {
                return S->stop || (S->admit_seq == seq && (!fits || S->in_use + r->foot <= S->budget));
            });
            if (S->stop) return false;
            S->admit_seq += 1;
            if (fits) S->in_use += r->foot;
            S->cv_mem.notify_all();
            turn_taken = true;
            return true;
        };
        try {
            TR_CUDA(cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking));
            tr_options o = r->o;
            o.hbm_budget = S->budget;
            rc = tr_create(&r->ctx, &o, r->stream);
            if (rc != TR_OK) throw Error(rc, "server: context creation failed");
            rc = tr_set_molecule(r->ctx, (int)r->Z.size(), r->Z.data(), r->xyz.data(), r->aux.data(),
                                 (int)r->shells.size(), r->shells.data());
            if (rc != TR_OK) throw Error(rc, r->ctx->err);
            rc = tr_set_orbitals(r->ctx, r->nao, r->nmo, r->nocc, r->C.data(), r->eps.data(), 0);
            if (rc != TR_OK) throw Error(rc, r->ctx->err);
            r->foot = footprint(r->ctx);
            if (r->foot > S->budget && !r->ctx->opt.j_ao && r->ctx->nJ > 0) {
                // (P|ia) does not fit: the Coulomb term on the fly in the AO basis
                // (Sec. 3.1), with integral chunks halved until the request fits
                tr_options o2 = r->ctx->opt;
                o2.j_ao = 1;
                const size_t least = (size_t)(8.0 * r->ctx->nao * r->ctx->nao * 4);
                for (size_t cb = o2.aux_chunk_bytes; cb >= least; cb /= 2) {
                    o2.aux_chunk_bytes = cb;
                    rc = tr_set_options(r->ctx, &o2);
                    if (rc != TR_OK) throw Error(rc, r->ctx->err);
                    r->foot = footprint(r->ctx);
                    if (r->foot <= S->budget) break;
                }
            }
            if (r->foot > S->budget)
                throw Error(TR_ENOMEM, "server: request needs " + std::to_string(r->foot >> 20) +
                                           " MiB of device memory, the server budget is " +
                                           std::to_string(S->budget >> 20) + " MiB");
            if (!take_turn(true)) {
                release_request(S, r.get());
                return;
            }
            r->t_admit = S->now();
            r->ctx->budget.limit = r->foot;
            rc = tr_build(r->ctx);
            if (rc != TR_OK) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->in_use -= r->foot;
                S->cv_mem.notify_all();
                throw Error(rc, r->ctx->err);
            }
            r->t_built = S->now();
            std::lock_guard<std::mutex> lk(S->mu);
            S->ready.push_back(std::move(r));
            S->cv_ready.notify_all();
            continue;
        } catch (const Error &e) {
            rc = e.code;
            msg = e.what();
        } catch (const std::exception &e) {
            rc = TR_ECUDA;
            msg = e.what();
        }
        if (!turn_taken && !take_turn(false)) {
            release_request(S, r.get());
            return;
        }
        fail(S, r.get(), rc, msg);
        release_request(S, r.get());
    }
}

void solver_loop(tr_server *S)
{
    cudaSetDevice(S->device);
    struct Member {
        std::unique_ptr<tr_server::Req> r;
        std::unique_ptr<Dav> d;
        bool fresh = true;
        cudaEvent_t join = nullptr;
    };
    std::vector<std::unique_ptr<Member>> act;
    cudaStream_t s0 = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    StepGraph g;
    // the graph is keyed by request ids, never by context addresses: a finished
    // request's context is freed and a later one may be allocated at the same address
    std::vector<std::pair<long long, int>> sig;
    bool warmed = false;

    auto finish = [&](Member &m, int rc_in, const std::string &msg) {
        tr_result res;
        std::memset(&res, 0, sizeof res);
        res.id = m.r->id;
        res.t_submit = m.r->t_submit;
        res.t_admit = m.r->t_admit;
        res.t_built = m.r->t_built;
        int rc = rc_in;
        if (rc == TR_OK && m.d) {
            try {
                const int n = m.d->n;
                res.nstates = n;
                double *X = nullptr;
                if (m.r->want_x) {
                    X = (double *)std::malloc(sizeof(double) * (size_t)n * m.d->nov);
                    if (!X) throw Error(TR_ENOMEM, "server: host allocation of X failed");
                }
                tr_solve_info info;
                rc = m.d->output(res.omega, X, nullptr, res.resid, 0, &info);
                res.X = X;
                res.niter = info.niter;
                res.nmatvec = info.nmatvec;
            } catch (const Error &e) {
                rc = e.code;
                std::strncpy(res.error, e.what(), sizeof(res.error) - 1);
            } catch (const std::exception &e) {
                rc = TR_ECUDA;
                std::strncpy(res.error, e.what(), sizeof(res.error) - 1);
            }
        } else {
            std::strncpy(res.error, msg.c_str(), sizeof(res.error) - 1);
        }
        res.status = rc;
        res.j_ao = m.r->ctx ? m.r->ctx->opt.j_ao : 0;
        // nothing of this request may still be queued when its pinned and device
        // buffers are freed (the error paths get here without a synchronisation)
        if (m.r->stream) cudaStreamSynchronize(m.r->stream);
        if (m.r->ctx && m.r->ctx->cst) cudaStreamSynchronize(m.r->ctx->cst);
        m.d.reset();
        release_request(S, m.r.get());
        if (m.join) cudaEventDestroy(m.join);
        m.join = nullptr;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->in_use -= m.r->foot;
            S->cv_mem.notify_all();
        }
        res.t_done = S->now();
        post_result(S, res);
    };

    while (true) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_ready.wait(lk, [&] { return S->stop || !S->ready.empty() || !act.empty(); });
            if (S->stop && act.empty()) break;
            while (!S->ready.empty() && (int)act.size() < S->opt.max_active) {
                std::unique_ptr<Member> m(new Member);
                m->r = std::move(S->ready.front());
                S->ready.pop_front();
                act.push_back(std::move(m));
            }
        }
        if (S->stop) break;
        // newcomers: Davidson state, guess, kernels loaded before any capture
        for (auto &mp : act) {
            Member &m = *mp;
            if (!m.fresh || m.d) continue;
            try {
                m.d.reset(new Dav(m.r->ctx));
                cudaEventCreateWithFlags(&m.join, cudaEventDisableTiming);
                std::vector<tr_ctx *> one{m.r->ctx};
                std::vector<int> rows{m.d->n};
                if (S->opt.autotune_tiles) autotune(one, rows);
                if (!warmed || !S->opt.autotune_tiles) matvec(m.r->ctx, m.d->n, m.r->ctx->Tn.p, m.r->ctx->Wn.p);
                warmed = true;
                m.d->guess();
            } catch (const Error &e) {
                finish(m, e.code, e.what());
            } catch (const std::exception &e) {
                finish(m, TR_ECUDA, e.what());
            }
        }
        act.erase(std::remove_if(act.begin(), act.end(), [](const std::unique_ptr<Member> &m) { return !m->r->ctx; }),
                  act.end());
        // one step for the members already in flight
        std::vector<Member *> pend;
        for (auto &mp : act) {
            Member &m = *mp;
            if (m.fresh) {
                pend.push_back(&m);
                continue;
            }
            try {
                if (m.d->done)
                    finish(m, TR_OK, "");  // stagnated in the last absorb
                else
                    m.d->eig_async();
            } catch (const Error &e) {
                finish(m, e.code, e.what());
            }
        }
        for (auto &mp : act) {
            Member &m = *mp;
            if (m.fresh || !m.r->ctx) continue;
            if (std::find(pend.begin(), pend.end(), &m) != pend.end()) continue;
            try {
                TR_CUDA(cudaStreamSynchronize(m.d->st));
                m.d->check();
                if (!m.d->done) m.d->prepare();
                if (m.d->done)
                    finish(m, TR_OK, "");
                else
                    pend.push_back(&m);
            } catch (const Error &e) {
                finish(m, e.code, e.what());
            } catch (const std::exception &e) {
                finish(m, TR_ECUDA, e.what());
            }
        }
        act.erase(std::remove_if(act.begin(), act.end(), [](const std::unique_ptr<Member> &m) { return !m->r->ctx; }),
                  act.end());
        pend.erase(std::remove_if(pend.begin(), pend.end(), [](Member *m) { return !m->r->ctx; }), pend.end());
        if (pend.empty()) continue;
        // the products of this step: one graph launch (recorded again when the membership changes)
        try {
            std::vector<std::pair<long long, int>> key;
            std::vector<tr_ctx *> cs;
            std::vector<int> rows, members;
            std::vector<cudaEvent_t> joins;
            for (Member *m : pend) {
                const int rws = m->fresh ? m->d->b0 : m->d->n;
                key.push_back({m->r->id, rws});
                members.push_back((int)cs.size());
                cs.push_back(m->r->ctx);
                rows.push_back(rws);
                joins.push_back(m->join);
            }
            if (!g.exec || key != sig) {
                capture(g, s0, cs, members, rows, fork, joins);
                sig = key;
            }
            for (Member *m : pend) {
                TR_CUDA(cudaEventRecord(m->join, m->d->st));
                TR_CUDA(cudaStreamWaitEvent(s0, m->join, 0));
            }
            TR_CUDA(cudaGraphLaunch(g.exec, s0));
            TR_CUDA(cudaEventRecord(done, s0));
            for (Member *m : pend) {
                TR_CUDA(cudaStreamWaitEvent(m->d->st, done, 0));
                m->d->absorb();
                m->fresh = false;
            }
        } catch (const Error &e) {
            // a launched graph may still use the members' buffers
            cudaStreamSynchronize(s0);
            for (Member *m : pend) finish(*m, e.code, e.what());
            act.erase(std::remove_if(act.begin(), act.end(), [](const std::unique_ptr<Member> &m) { return !m->r->ctx; }),
                      act.end());
            g.reset();
            sig.clear();
        }
    }
    for (auto &mp : act) finish(*mp, TR_ECUDA, "server: stopped before completion");
    cudaStreamSynchronize(s0);
    g.reset();
    cudaStreamDestroy(s0);
    cudaEventDestroy(fork);
    cudaEventDestroy(done);
}

}  // namespace
}  // namespace tr

extern "C" {

int tr_server_create(tr_server **out, const tr_server_options *opt)
{
    if (!out) return TR_EINVAL;
    *out = nullptr;
    tr_server *S = new (std::nothrow) tr_server();
    if (!S) return TR_ENOMEM;
    if (opt) S->opt = *opt;
    if (S->opt.max_active <= 0) S->opt.max_active = 64;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return TR_ECUDA;
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete S;
        return TR_ECUDA;
    }
    S->budget = S->opt.hbm_budget ? S->opt.hbm_budget : (size_t)(0.9 * (double)fr);
    if (S->opt.build_threads <= 0) S->opt.build_threads = 4;
    for (int t = 0; t < S->opt.build_threads; ++t) S->builders.emplace_back(tr::builder_loop, S);
    S->solver = std::thread(tr::solver_loop, S);
    *out = S;
    return TR_OK;
}

int tr_server_submit(tr_server *S, const tr_request *q, long long *id)
{
    if (!S || !q || !q->Z || !q->xyz || !q->aux_exp || !q->shells || !q->C || !q->eps) return TR_EINVAL;
    if (q->natm <= 0 || q->nshell <= 0 || q->nao <= 0 || q->nmo <= 0 || q->nocc <= 0) return TR_EINVAL;
    std::unique_ptr<tr_server::Req> r(new tr_server::Req);
    r->Z.assign(q->Z, q->Z + q->natm);
    r->xyz.assign(q->xyz, q->xyz + 3 * q->natm);
    r->aux.assign(q->aux_exp, q->aux_exp + q->natm);
    r->sexp.resize(q->nshell);
    r->scoef.resize(q->nshell);
    for (int s = 0; s < q->nshell; ++s) {
        const tr_shell &sh = q->shells[s];
        if (sh.nprim < 1 || sh.nprim > 16 || !sh.exp || !sh.coef) return TR_EINVAL;
        r->sexp[s].assign(sh.exp, sh.exp + sh.nprim);
        r->scoef[s].assign(sh.coef, sh.coef + sh.nprim);
        tr_shell c = sh;
        c.exp = r->sexp[s].data();
        c.coef = r->scoef[s].data();
        r->shells.push_back(c);
    }
    r->nao = q->nao;
    r->nmo = q->nmo;
    r->nocc = q->nocc;
    r->C.assign(q->C, q->C + (size_t)q->nao * q->nmo);
    r->eps.assign(q->eps, q->eps + q->nmo);
    if (q->opt.tddft) return TR_EINVAL;  // full TDDFT runs through tr_solve only
    r->o = q->opt;
    r->want_x = q->want_x;
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = S->now();
    if (id) *id = r->id;
    S->outstanding += 1;
    S->submitted.push_back(std::move(r));
    S->cv_submit.notify_all();
    return TR_OK;
}

int tr_server_poll(tr_server *S, tr_result *out, int max, int timeout_ms)
{
    if (!S || (!out && max > 0)) return TR_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->results.empty() && timeout_ms != 0) {
        if (timeout_ms < 0)
            S->cv_result.wait(lk, [&] { return !S->results.empty() || S->outstanding == 0; });
        else
            S->cv_result.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !S->results.empty(); });
    }
    int n = 0;
    while (n < max && !S->results.empty()) {
        out[n++] = S->results.front();
        S->results.pop_front();
        S->outstanding -= 1;
    }
    return n;
}

int tr_server_outstanding(tr_server *S)
{
    if (!S) return TR_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    return S->outstanding;
}

double tr_server_clock(tr_server *S) { return S ? S->now() : 0.0; }

void tr_server_destroy(tr_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_submit.notify_all();
        S->cv_ready.notify_all();
        S->cv_mem.notify_all();
    }
    for (auto &t : S->builders)
        if (t.joinable()) t.join();
    if (S->solver.joinable()) S->solver.join();
    for (auto &r : S->submitted) tr::release_request(S, r.get());
    for (auto &r : S->ready) tr::release_request(S, r.get());
    for (auto &res : S->results) std::free(res.X);
    delete S;
}

void tr_free(void *p) { std::free(p); }

}  // extern "C"
