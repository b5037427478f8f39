// tr_matvec_noalloc: the TDA-risp matrix-vector product with every piece of
// scratch taken from one file-scope device array instead of cudaMalloc.
//
// Who needs it: code that records the product into a CUDA graph (cudaMalloc
// and cudaFree are not allowed while a stream is being captured), code that
// runs under another framework's memory allocator with a hard cap, and
// latency-critical loops that cannot afford cudaMalloc's implicit device
// synchronisation.  tr_matvec grows its workspaces on first use; this variant
// never allocates.
//
// The array is TR_NOALLOC_SCRATCH_BYTES (32 MiB) of device memory that every
// GPU which loads the library holds until the process exits.  Its device
// address is looked up once per device (cudaGetSymbolAddress) by the first call
// on that device, with that device current; that first call must therefore not
// be made while a stream is being captured.  All calls share the array: two
// calls whose work overlaps on the GPU (different streams or contexts at the
// same time) race on it.  Every region is fully written before it is read
// within a call, so nothing has to start at zero and the contents left by the
// previous call are never used.
#include <algorithm>
#include <mutex>

#include "ctx.cuh"

namespace {

constexpr size_t SCRATCH_DOUBLES = (size_t)TR_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr size_t SPLITK_DOUBLES = 65536;  // split-K partial sums of the J contraction
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

std::mutex g_mu;
double *g_addr[MAX_DEVICES] = {nullptr};

double *scratch_address(int dev)
{
    TR_REQUIRE(dev >= 0 && dev < MAX_DEVICES, TR_EINVAL, "matvec_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw tr::Error(TR_ECUDA, std::string("matvec_noalloc: cudaGetSymbolAddress failed: ") +
                                          cudaGetErrorString(e));
        }
        g_addr[dev] = (double *)p;
    }
    return g_addr[dev];
}

__global__ void na_diag(const double *__restrict__ D, const double *__restrict__ X, double *__restrict__ AX,
                        long long nov, int m)
{
    // one pass over the index ia: D read once, then the m vectors (no division per element)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nov; i += (long long)gridDim.x * blockDim.x) {
        const double d = D[i];
#pragma unroll 4
        for (int j = 0; j < m; ++j) AX[(long long)j * nov + i] = d * X[(long long)j * nov + i];
    }
}

__global__ void na_gather(const double *__restrict__ X, double *__restrict__ Xw, int m, int nocc, int nvir,
                          int o0, int oK, int vK)
{
    const long long tot = (long long)m * oK * vK;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t % vK);
        const long long r = t / vK;
        const int j = (int)(r % oK);
        const int mm = (int)(r / oK);
        Xw[t] = X[((long long)mm * nocc + o0 + j) * nvir + b];
    }
}

unsigned na_grid(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>(tr::cdiv(n, 256), 152 * 16)); }

}  // namespace

namespace tr {

void matvec_noalloc(tr_ctx *c, int m, const double *X, double *AX)
{
    TR_REQUIRE(c->built, TR_EINVAL, "matvec_noalloc: call tr_build first");
    TR_REQUIRE(c->opt.precision == TR_FP64, TR_EINVAL, "matvec_noalloc: only the FP64 form is available");
    if (m <= 0) return;
    int dev = -1;
    TR_CUDA(cudaGetDevice(&dev));
    TR_REQUIRE(dev == c->device, TR_EINVAL, "matvec_noalloc: the context's device must be current");
    double *scr = scratch_address(dev);

    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ, nK = c->nK;
    const int oK = c->oK, vK = c->vK, o0 = c->o0;
    const long long nov = c->nov;
    const bool kact = c->k_active;
    // per vector: Z and Zt (2 nJ), and for K the window copy plus at least one
    // aux function of M (2 oK vK)
    const size_t avail = SCRATCH_DOUBLES - SPLITK_DOUBLES;
    const size_t per_vec = 2 * (size_t)nJ + (kact ? 2 * (size_t)oK * vK : 0);
    TR_REQUIRE(per_vec <= avail, TR_EINVAL,
               "matvec_noalloc: problem too large for the 32 MiB static scratch (needs 2 N_auxJ + "
               "2 nocc_k nvir_k doubles per vector plus 65536 split-K doubles)");
    // per_vec is 0 when there is neither a Coulomb nor an exchange term (no
    // auxiliary functions and no active window): then only the diagonal runs
    const int mb = (int)std::min<size_t>({(size_t)m, (size_t)32, per_vec ? avail / per_vec : (size_t)32});
    int npk = 0;
    if (kact) {
        const size_t used = (size_t)mb * (2 * (size_t)nJ + (size_t)oK * vK);
        npk = (int)std::min<size_t>(nK, (avail - used) / ((size_t)mb * oK * vK));
        npk = std::min(npk, 65535 / mb);
    }
    double *ws = scr;
    double *Z = scr + SPLITK_DOUBLES;
    double *Z2 = Z + (size_t)nJ * mb;
    double *Xw = Z2 + (size_t)nJ * mb;
    double *M = Xw + (size_t)mb * oK * vK;

    // a profiler that records nothing: no event objects are created here
    Prof lp;
    cudaStream_t st = c->st;
    for (int m0 = 0; m0 < m; m0 += mb) {
        const int mm = std::min(mb, m - m0);
        const double *x = X + (long long)m0 * nov;
        double *ax = AX + (long long)m0 * nov;
        TR_LAUNCH(lp, st, "diag", 0, 0, na_diag<<<na_grid(nov), 256, 0, st>>>(c->D.p, x, ax, nov, mm));
        if (nJ) {
            dgemm(lp, st, "J_contract", false, true, nJ, mm, (int)nov, 1.0, c->Y.p, nov, x, nov, 0.0, Z, mm,
                  Batch(), ws, SPLITK_DOUBLES);
            dgemm(lp, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, Z, mm, 0.0, Z2, mm, Batch(),
                  nullptr, 0);
            dgemm(lp, st, "J_expand", true, false, mm, (int)nov, nJ, 2.0, Z2, mm, c->Y.p, nov, 1.0, ax, nov,
                  Batch(), nullptr, 0);
        }
        if (kact) {
            const long long tot = (long long)mm * oK * vK;
            TR_LAUNCH(lp, st, "gather_window", 0, 0,
                      na_gather<<<na_grid(tot), 256, 0, st>>>(x, Xw, mm, nocc, nvir, o0, oK, vK));
            for (int P0 = 0; P0 < nK; P0 += npk) {
                const int np = std::min(npk, nK - P0);
                Batch b1;
                b1.n1 = mm;
                b1.n2 = np;
                b1.sA1 = (long long)oK * vK;
                b1.sC1 = (long long)np * oK * vK;
                b1.sB2 = (long long)vK * vK;
                b1.sC2 = (long long)oK * vK;
                dgemm(lp, st, "K_stage1", false, false, oK, vK, vK, 1.0, Xw, vK, c->Tab.p + (long long)P0 * vK * vK,
                      vK, 0.0, M, vK, b1, nullptr, 0);
                Batch b2;
                b2.n1 = mm;
                b2.sB1 = (long long)np * oK * vK;
                b2.sC1 = nov;
                dgemm(lp, st, "K_stage2", false, false, oK, vK, np * oK, -c->opt.cx, c->T2.p + (long long)P0 * oK,
                      (long long)nK * oK, M, vK, 1.0, ax + (long long)o0 * nvir, nvir, b2, nullptr, 0);
            }
        }
    }
    c->prof.launches += lp.launches;
}

}  // namespace tr

extern "C" int tr_matvec_noalloc(tr_ctx *ctx, int m, const double *X, double *AX)
{
    if (!ctx) return TR_EINVAL;
    try {
        ctx->err.clear();
        TR_REQUIRE(m >= 0, TR_EINVAL, "matvec_noalloc: m must be >= 0");
        if (m == 0) return TR_OK;
        TR_REQUIRE(X && AX, TR_EINVAL, "matvec_noalloc: null pointer");
        TR_REQUIRE(!ctx->opt.j_ao, TR_EINVAL, "matvec_noalloc: the AO form of J (j_ao) allocates its workspaces");
        const size_t n = (size_t)m * ctx->nov;
        TR_REQUIRE(X + n <= AX || AX + n <= X, TR_EINVAL, "matvec_noalloc: X and AX overlap");
        tr::matvec_noalloc(ctx, m, X, AX);
        return TR_OK;
    } catch (const tr::Error &e) {
        ctx->err = e.what();
        return e.code;
    } catch (const std::exception &e) {
        ctx->err = e.what();
        return TR_ECUDA;
    }
}
