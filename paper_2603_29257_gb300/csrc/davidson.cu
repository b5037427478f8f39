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
#include <cmath>
#include <numeric>

#include "ctx.cuh"

namespace tr {
namespace {

constexpr double DROP_NORM = 1e-6;
constexpr double PRECOND_FLOOR = 1e-8;


__global__ void set_unit_rows(double *V, const int *idx, int n, long long nov)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) V[(long long)r * nov + idx[r]] = 1.0;
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
    *nkeep = nacc;
}

// sign convention: largest-magnitude component positive (ties: lowest index)
__global__ void sign_fix(double *X, long long nov)
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

int solve(tr_ctx *c, double *omega, double *Xout, double *resid, int on_device, tr_solve_info *info)
{
    TR_REQUIRE(c->built, TR_EINVAL, "solve: call tr_build first");
    TR_REQUIRE(omega, TR_EINVAL, "solve: omega must not be NULL");
    TR_REQUIRE(c->opt.nstates >= 1, TR_EINVAL, "solve: nstates must be >= 1");
    TR_REQUIRE(c->opt.nstates <= 64, TR_EINVAL, "solve: nstates must be <= 64");
    const long long nov = c->nov;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int n = (int)std::min<long long>(c->opt.nstates, nov);
    int b0 = c->opt.block > 0 ? c->opt.block : 2 * n;
    b0 = (int)std::min<long long>(std::max(b0, n), nov);
    int maxsp = c->opt.max_space > 0 ? c->opt.max_space : 20 * n;
    maxsp = std::max(maxsp, b0 + n);
    maxsp = (int)std::min<long long>(maxsp, std::max<long long>(nov, b0));
    const int max_iter = c->opt.max_iter > 0 ? c->opt.max_iter : 200;
    const double tol = c->opt.tol;
    const int pmax = std::max(b0, n);
    const size_t rowb = (size_t)nov * sizeof(double);

    // fixed buffers
    reserve_matvec(c, pmax);
    c->Tn.alloc((size_t)pmax * nov, &c->budget, "new vectors");
    c->Wn.alloc((size_t)pmax * nov, &c->budget, "new products");
    c->T.alloc((size_t)pmax * nov, &c->budget, "new vectors");
    c->Tt.alloc((size_t)pmax * nov, &c->budget, "new vectors");
    c->Xr.alloc((size_t)n * nov, &c->budget, "Ritz vectors");
    c->R.alloc((size_t)n * nov, &c->budget, "residuals");
    const int nblk = 256;
    c->part.alloc((size_t)nblk * pmax, &c->budget, "norms");
    c->rn.alloc(pmax, &c->budget, "norms");
    c->idx_dev.alloc(pmax + 2, &c->budget, "indices");
    c->Ss.alloc((size_t)pmax * pmax, &c->budget, "gram");
    c->Gc.alloc((size_t)pmax * pmax, &c->budget, "gram");

    // how many V/W rows fit in HBM; the rest spill to pinned host memory
    c->V.release();
    c->W.release();
    const int cs = std::max(8, pmax);  // staging rows per chunk
    long long avail = (long long)c->budget.limit - (long long)c->budget.used;
    const long long small = 5LL * maxsp * maxsp * 8 + 2LL * maxsp * pmax * 8 + (64LL << 20);
    int kd = (int)std::max<long long>(0, (avail - small) / (long long)(2 * rowb));
    if (kd < maxsp) kd = (int)std::max<long long>(0, (avail - small - 2LL * cs * rowb) / (long long)(2 * rowb));
    if (c->opt.dav_dev_rows > 0) kd = std::min(kd, c->opt.dav_dev_rows);
    kd = std::min(kd, maxsp);
    if (kd < maxsp && c->opt.host_budget > 0) {
        const long long hrows = (long long)(c->opt.host_budget / (2 * rowb));
        maxsp = (int)std::min<long long>(maxsp, kd + hrows);
    }
    TR_REQUIRE(maxsp >= b0 + 1 && maxsp >= n + 1, TR_ENOMEM,
               "solve: device and host budgets leave no room for the Davidson subspace");
    c->V.alloc((size_t)kd * nov, &c->budget, "Davidson V");
    c->W.alloc((size_t)kd * nov, &c->budget, "Davidson W");
    c->Hs.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
    c->Hw.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
    c->Yev.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
    c->Yw.alloc((size_t)maxsp * maxsp, &c->budget, "subspace");
    c->theta.alloc(maxsp, &c->budget, "subspace");
    c->Cs.alloc((size_t)2 * maxsp * pmax, &c->budget, "projections");
    PinnedBuf Vh, Wh;
    RowStore SV, SW;
    SV.nov = SW.nov = nov;
    SV.cap = SW.cap = maxsp;
    SV.kd = SW.kd = kd;
    SV.dev = c->V.p;
    SW.dev = c->W.p;
    if (kd < maxsp) {
        Vh.alloc((size_t)(maxsp - kd) * nov, "Davidson V");
        Wh.alloc((size_t)(maxsp - kd) * nov, "Davidson W");
        SV.host = Vh.p;
        SW.host = Wh.p;
        c->stage.reserve((size_t)2 * cs * nov, &c->budget, "spill staging");
        if (!c->cst) TR_CUDA(cudaStreamCreateWithFlags(&c->cst, cudaStreamNonBlocking));
        for (auto &e : c->sev)
            if (!e) TR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    long long moved = 0;

    double *ws = c->ws_split.p;
    const size_t wsn = c->ws_split.n;
    Events ev;
    double t_mv = 0, t_or = 0, t_eig = 0, t_oth = 0;

    // f(device pointer, first row, rows) for rows [r0, r1) of S; host rows are
    // staged through two device slots on the copy stream
    auto for_rows = [&](RowStore &S, int r0, int r1, auto &&f) {
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
            TR_CUDA(cudaMemcpyAsync(buf, S.host + (size_t)(s0 - S.kd) * nov, nr * rowb,
                                    cudaMemcpyHostToDevice, c->cst));
            TR_CUDA(cudaEventRecord(c->sev[slot], c->cst));
            TR_CUDA(cudaStreamWaitEvent(st, c->sev[slot], 0));
            f(buf, s0, nr);
            TR_CUDA(cudaEventRecord(c->sev[2 + slot], st));
            moved += (long long)nr * rowb;
        }
    };
    auto store_rows = [&](RowStore &S, int r0, int nr, const double *src) {
        int a = r0, b = std::min(r0 + nr, S.kd);
        if (a < b)
            TR_CUDA(cudaMemcpyAsync(S.dev + (long long)a * nov, src, (b - a) * rowb, cudaMemcpyDeviceToDevice, st));
        a = std::max(r0, S.kd);
        if (a < r0 + nr) {
            TR_CUDA(cudaMemcpyAsync(S.host + (size_t)(a - S.kd) * nov, src + (long long)(a - r0) * nov,
                                    (r0 + nr - a) * rowb, cudaMemcpyDeviceToHost, st));
            moved += (long long)(r0 + nr - a) * rowb;
        }
    };
    auto norms_of = [&](const double *A, int p, double *out) {
        TR_LAUNCH(pf, st, "row_norms", 0, 8.0 * p * nov,
                  row_sumsq<<<dim3(nblk, p), 256, 0, st>>>(A, p, nov, c->part.p));
        TR_LAUNCH(pf, st, "row_norms", 0, 0, finish_norms<<<cdiv(p, 64), 64, 0, st>>>(c->part.p, nblk, p, out));
    };
    // rows/cols k0..k0+p of H for the new vectors Vn (products Wn)
    auto h_update = [&](int k0, int p, const double *Vn, const double *Wn) {
        const int k = k0 + p;
        double *A1 = c->Cs.p, *A2 = c->Cs.p + (size_t)maxsp * pmax;
        for_rows(SW, 0, k0, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "subspace_H", false, true, p, nr, (int)nov, 1.0, Vn, nov, rows, nov, 0.0, A1 + r0, k,
                  Batch(), ws, wsn);
        });
        dgemm(pf, st, "subspace_H", false, true, p, p, (int)nov, 1.0, Vn, nov, Wn, nov, 0.0, A1 + k0, k, Batch(), ws, wsn);
        for_rows(SV, 0, k0, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "subspace_H", false, true, p, nr, (int)nov, 1.0, Wn, nov, rows, nov, 0.0, A2 + r0, k,
                  Batch(), ws, wsn);
        });
        dgemm(pf, st, "subspace_H", false, true, p, p, (int)nov, 1.0, Wn, nov, Vn, nov, 0.0, A2 + k0, k, Batch(), ws, wsn);
        TR_LAUNCH(pf, st, "subspace_insert", 0, 0,
                  h_insert<<<dim3(cdiv(k, 128), p), 128, 0, st>>>(c->Hs.p, maxsp, A1, A2, p, k, k0));
    };
    // orthonormalise rows src[0:p] into dst; returns the count kept
    auto cholqr = [&](double *src, int p, double *dst, double drop2) -> int {
        dgemm(pf, st, "gram", false, true, p, p, (int)nov, 1.0, src, nov, src, nov, 0.0, c->Ss.p, p, Batch(), ws, wsn);
        TR_LAUNCH(pf, st, "cholqr_coef", 0, 0, cholqr_coef<<<1, 1, 0, st>>>(c->Ss.p, p, drop2, c->Gc.p, c->idx_dev.p + pmax));
        int keep = 0;
        TR_CUDA(cudaMemcpyAsync(&keep, c->idx_dev.p + pmax, sizeof(int), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaStreamSynchronize(st));
        if (keep > 0)
            dgemm(pf, st, "orth_apply", false, false, keep, (int)nov, p, 1.0, c->Gc.p, p, src, nov, 0.0, dst,
                  nov, Batch(), nullptr, 0);
        return keep;
    };
    auto orthonormal_block = [&](double *src, int p, double *dst, double *tmp) -> int {
        int k1 = cholqr(src, p, tmp, DROP_NORM * DROP_NORM);
        if (k1 == 0) return 0;
        return cholqr(tmp, k1, dst, 0.0);
    };
    auto apply_A = [&](const double *Vn, double *Wn, int p) {
        TR_CUDA(cudaEventRecord(ev.e[4], st));
        matvec(c, p, Vn, Wn);
        TR_CUDA(cudaEventRecord(ev.e[5], st));
    };

    TR_CUDA(cudaMemsetAsync(c->flag.p, 0, 2 * sizeof(int), st));
    // initial guess: unit vectors on the b0 smallest e_a - e_i (ties: lower index)
    std::vector<double> Dh(nov);
    TR_CUDA(cudaMemcpyAsync(Dh.data(), c->D.p, sizeof(double) * nov, cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    std::vector<int> order(nov);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Dh[a] < Dh[b]; });
    TR_CUDA(cudaMemcpyAsync(c->idx_dev.p, order.data(), sizeof(int) * b0, cudaMemcpyHostToDevice, st));
    TR_CUDA(cudaMemsetAsync(c->Tn.p, 0, sizeof(double) * (size_t)b0 * nov, st));
    TR_LAUNCH(pf, st, "set_unit", 0, 0, set_unit_rows<<<cdiv(b0, 64), 64, 0, st>>>(c->Tn.p, c->idx_dev.p, b0, nov));
    int k = b0;
    apply_A(c->Tn.p, c->Wn.p, k);
    h_update(0, k, c->Tn.p, c->Wn.p);
    store_rows(SV, 0, k, c->Tn.p);
    store_rows(SW, 0, k, c->Wn.p);
    TR_CUDA(cudaStreamSynchronize(st));
    t_mv += elapsed(ev.e[4], ev.e[5]);

    int nmv = b0, nrestart = 0, it = 0, converged = 0;
    std::vector<double> rn_h(n), th_h(n);
    std::vector<int> unconv;
    for (it = 1; it <= max_iter; ++it) {
        TR_CUDA(cudaEventRecord(ev.e[0], st));
        TR_LAUNCH(pf, st, "copy_sub", 0, 0, copy_sub<<<dim3(cdiv(k, 128), k), 128, 0, st>>>(c->Hs.p, maxsp, c->Hw.p, k));
        TR_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int), st));
        jacobi_eigh(pf, st, c->Hw.p, k, c->theta.p, c->Yev.p, c->Yw.p, c->flag.p);
        TR_CUDA(cudaEventRecord(ev.e[1], st));
        // Ritz vectors X = Y^T V and residuals R = Y^T W - theta X
        for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "ritz", true, false, n, (int)nov, nr, 1.0, c->Yev.p + (long long)r0 * k, k, rows, nov,
                  r0 == 0 ? 0.0 : 1.0, c->Xr.p, nov, Batch(), nullptr, 0);
        });
        for_rows(SW, 0, k, [&](const double *rows, int r0, int nr) {
            dgemm(pf, st, "ritz", true, false, n, (int)nov, nr, 1.0, c->Yev.p + (long long)r0 * k, k, rows, nov,
                  r0 == 0 ? 0.0 : 1.0, c->R.p, nov, Batch(), nullptr, 0);
        });
        TR_LAUNCH(pf, st, "residual", 0, 24.0 * n * nov,
                  ritz_resid<<<dim3(nblk, n), 256, 0, st>>>(c->R.p, c->Xr.p, c->theta.p, n, nov, c->part.p));
        TR_LAUNCH(pf, st, "residual", 0, 0, finish_norms<<<cdiv(n, 64), 64, 0, st>>>(c->part.p, nblk, n, c->rn.p));
        TR_CUDA(cudaMemcpyAsync(rn_h.data(), c->rn.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaMemcpyAsync(th_h.data(), c->theta.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        int jflag[2] = {0, 0};
        TR_CUDA(cudaMemcpyAsync(jflag, c->flag.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaEventRecord(ev.e[2], st));
        TR_CUDA(cudaStreamSynchronize(st));
        t_eig += elapsed(ev.e[0], ev.e[1]);
        t_oth += elapsed(ev.e[1], ev.e[2]);
        TR_REQUIRE(!jflag[0], TR_ECUDA, "solve: subspace eigensolver did not converge");
        TR_REQUIRE(!jflag[1], TR_ECUDA, "solve: a tensor-core pipeline wait timed out");
        unconv.clear();
        for (int r = 0; r < n; ++r)
            if (!(rn_h[r] < tol)) unconv.push_back(r);
        if (unconv.empty()) {
            converged = 1;
            break;
        }
        if (it == max_iter) break;
        const int p = (int)unconv.size();
        if (k + p > maxsp) {
            // restart from the Ritz vectors; A V is recomputed for them (Sec. 3.3)
            TR_CUDA(cudaEventRecord(ev.e[0], st));
            int kk = orthonormal_block(c->Xr.p, n, c->Tn.p, c->Tt.p);
            TR_CUDA(cudaEventRecord(ev.e[1], st));
            TR_REQUIRE(kk > 0, TR_ECUDA, "solve: restart produced an empty subspace");
            apply_A(c->Tn.p, c->Wn.p, kk);
            nmv += kk;
            h_update(0, kk, c->Tn.p, c->Wn.p);
            store_rows(SV, 0, kk, c->Tn.p);
            store_rows(SW, 0, kk, c->Wn.p);
            TR_CUDA(cudaStreamSynchronize(st));
            t_or += elapsed(ev.e[0], ev.e[1]);
            t_mv += elapsed(ev.e[4], ev.e[5]);
            k = kk;
            nrestart += 1;
            continue;
        }
        TR_CUDA(cudaEventRecord(ev.e[0], st));
        TR_CUDA(cudaMemcpyAsync(c->idx_dev.p, unconv.data(), sizeof(int) * p, cudaMemcpyHostToDevice, st));
        TR_LAUNCH(pf, st, "precondition", 0, 32.0 * p * nov,
                  precond<<<dim3(nblk, p), 256, 0, st>>>(c->T.p, c->R.p, c->D.p, c->theta.p, c->idx_dev.p, p, nov,
                                                          PRECOND_FLOOR));
        norms_of(c->T.p, p, c->rn.p);
        TR_LAUNCH(pf, st, "normalise", 0, 16.0 * p * nov,
                  row_scale_inv<<<dim3(nblk, p), 256, 0, st>>>(c->T.p, p, nov, c->rn.p));
        // two passes of block classical Gram-Schmidt against V[0:k]
        for (int pass = 0; pass < 2; ++pass) {
            for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
                dgemm(pf, st, "orth_project", false, true, nr, p, (int)nov, 1.0, rows, nov, c->T.p, nov, 0.0,
                      c->Cs.p + (long long)r0 * p, p, Batch(), ws, wsn);
            });
            for_rows(SV, 0, k, [&](const double *rows, int r0, int nr) {
                dgemm(pf, st, "orth_update", true, false, p, (int)nov, nr, -1.0, c->Cs.p + (long long)r0 * p, p,
                      rows, nov, 1.0, c->T.p, nov, Batch(), nullptr, 0);
            });
        }
        int pk = orthonormal_block(c->T.p, p, c->Tn.p, c->Tt.p);
        TR_CUDA(cudaEventRecord(ev.e[1], st));
        if (pk == 0) break;  // no new directions: stagnation
        apply_A(c->Tn.p, c->Wn.p, pk);
        nmv += pk;
        h_update(k, pk, c->Tn.p, c->Wn.p);
        store_rows(SV, k, pk, c->Tn.p);
        store_rows(SW, k, pk, c->Wn.p);
        TR_CUDA(cudaStreamSynchronize(st));
        t_or += elapsed(ev.e[0], ev.e[1]);
        t_mv += elapsed(ev.e[4], ev.e[5]);
        k += pk;
    }
    if (it > max_iter) it = max_iter;

    // outputs: omega, unit-norm sign-fixed X, residual norms
    norms_of(c->Xr.p, n, c->rn.p);
    TR_LAUNCH(pf, st, "normalise", 0, 16.0 * n * nov, row_scale_inv<<<dim3(nblk, n), 256, 0, st>>>(c->Xr.p, n, nov, c->rn.p));
    TR_LAUNCH(pf, st, "sign_fix", 0, 0, sign_fix<<<n, 1024, 0, st>>>(c->Xr.p, nov));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TR_CUDA(cudaMemcpyAsync(omega, c->theta.p, sizeof(double) * n, kind, st));
    if (Xout) TR_CUDA(cudaMemcpyAsync(Xout, c->Xr.p, sizeof(double) * (size_t)n * nov, kind, st));
    if (resid) {
        if (on_device)
            TR_CUDA(cudaMemcpyAsync(resid, rn_h.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
        else
            std::copy(rn_h.begin(), rn_h.end(), resid);
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

}  // namespace tr
