// Reduced-precision form of the TDA-risp matrix-vector product.
//
// Same operator as the FP64 form (Sec. 2 Eq. TDA-risp; Sec. 3.2 for K):
//   - the three-centre integrals, metrics and MO transforms are built in FP64
//     and the MO tensors are then rounded to FP32 (the paper builds its
//     integrals in FP64 and runs everything after them in FP32, Sec. 3.3);
//     see build_mixed for why the transforms themselves stay FP64;
//   - J (Sec. 3.1): Z = (Q|jb) X and J = (P|ia) Zt as FP32 products on the CUDA
//     cores at the FFMA rate (Z summed in FP32 over chunks of at most 4096
//     terms and in FP64 across chunks); (P|Q)^-1 is applied in FP64;
//   - K: both stages on the tensor cores (tcgen05 kind::tf32) with split
//     operands, hi*hi + hi*lo + lo*hi, FP32 accumulation; stage 1 writes M^P
//     already split and laid out K-major for stage 2, stage 2 accumulates
//     -c_x K into the FP64 output;
//   - the diagonal and everything in the Davidson driver stay FP64.
#include <algorithm>
#include <cmath>

#include "ctx.cuh"

namespace tr {
namespace {

__global__ void mixed_prepare(const double *__restrict__ X, float *__restrict__ X32, float *__restrict__ Xh,
                              float *__restrict__ Xl, int m, int nocc, int nvir, int o0, int oK, int vK, int vKp)
{
    const long long nov = (long long)nocc * nvir;
    const long long tot = nov * m;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const float f = (float)X[t];
        X32[t] = f;
        const long long mm = t / nov, r = t - mm * nov;
        const int i = (int)(r / nvir), a = (int)(r - (long long)i * nvir);
        if (i >= o0 && a < vK) {
            const long long w = (mm * oK + (i - o0)) * vKp + a;
            Xh[w] = f;
            Xl[w] = f - __uint_as_float(__float_as_uint(f) & 0xFFFFE000u);
        }
    }
}

// ---------------------------------------------------------------- J on the CUDA cores
//
// The Coulomb contractions stream (P|ia) in FP32 with the block of MB <= 32
// trial vectors: 2 MB flops per 4-byte element, above the FP32 CUDA-core
// ridge (73 TFLOP/s over 6.8 TB/s is 10.7 flop/B) for MB = 32, so both kernels
// are built for the FFMA rate: every thread keeps 4 x MB accumulators, and the
// operand shared by a whole warp (the MB trial values) is read from shared
// memory as broadcast float4 loads.

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES), "r"(valid ? BYTES : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// CTA tile: 256 aux functions x MB trial vectors, 64 threads (thread t: P = P0 +
// t + 64 q, q < 4); stages of 16 ia: Y rows padded to 20 floats (80 bytes: the
// float4 reads of 8 consecutive rows by a quarter warp hit 32 distinct banks),
// X stored [ia][m] for broadcast float4 reads
constexpr int JC_THREADS = 64, JC_TP = 256, JC_KK = 16, JC_LD = 20, JC_CHUNK = 4096;
constexpr int JC_STAGE = JC_TP * JC_LD + JC_KK * 32;  // floats

// Z partials: part[s][P][m] = sum over the ia of split s of Y[P][ia] X[m][ia],
// FP32 sums over chunks of at most 4096 ia added into the FP64 partial after
// each chunk.  VEC: rows of Y start on 16-byte boundaries (nov a multiple of
// 4) and are copied 16 bytes at a time.
template <int MB, bool VEC>
__global__ void __launch_bounds__(JC_THREADS)
    jc_kernel(const float *__restrict__ Y, const float *__restrict__ X, int nJ, int mm, long long nov, long long per,
              double *__restrict__ part)
{
    extern __shared__ __align__(16) float jsm[];
    const int t = threadIdx.x;
    const int P0 = blockIdx.x * JC_TP;
    const long long i0 = (long long)blockIdx.y * per, i1 = min(nov, i0 + per);
    double *out = part + ((long long)blockIdx.y * nJ) * mm;
    const int nst = (int)((i1 - i0 + JC_KK - 1) / JC_KK);
    auto load = [&](int s, float *buf) {
        const long long c0 = i0 + (long long)s * JC_KK;
        if (VEC) {
            for (int e = t; e < JC_TP * (JC_KK / 4); e += JC_THREADS) {
                const int r = e >> 2, k = 4 * (e & 3);
                const long long col = c0 + k;
                const bool ok = P0 + r < nJ && col < i1;  // i1 and col are multiples of 4 here
                cp_async<16>(buf + r * JC_LD + k, Y + (ok ? (long long)(P0 + r) * nov + col : 0), ok);
            }
        } else {
            for (int e = t; e < JC_TP * JC_KK; e += JC_THREADS) {
                const int r = e / JC_KK, k = e - r * JC_KK;
                const long long col = c0 + k;
                const bool ok = P0 + r < nJ && col < i1;
                cp_async<4>(buf + r * JC_LD + k, Y + (ok ? (long long)(P0 + r) * nov + col : 0), ok);
            }
        }
        float *xs = buf + JC_TP * JC_LD;
        for (int e = t; e < JC_KK * MB; e += JC_THREADS) {
            const int m = e / JC_KK, k = e - m * JC_KK;
            const long long col = c0 + k;
            const bool ok = m < mm && col < i1;
            cp_async<4>(xs + k * 32 + m, X + (ok ? (long long)m * nov + col : 0), ok);
        }
        cp_async_commit();
    };
    float acc[4][MB];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int m = 0; m < MB; ++m) acc[q][m] = 0.f;
    int chunk_left = JC_CHUNK / JC_KK;
    bool first = true;
    load(0, jsm);
    for (int s = 0; s < nst; ++s) {
        const float *cur = jsm + (s & 1) * JC_STAGE;
        if (s + 1 < nst) {
            load(s + 1, jsm + ((s + 1) & 1) * JC_STAGE);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *xs = cur + JC_TP * JC_LD;
#pragma unroll
        for (int k4 = 0; k4 < JC_KK / 4; ++k4) {
            float4 y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) y[q] = *(const float4 *)(cur + (t + 64 * q) * JC_LD + 4 * k4);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int k = 4 * k4 + kk;
#pragma unroll
                for (int m4 = 0; m4 < MB / 4; ++m4) {
                    const float4 x = *(const float4 *)(xs + k * 32 + 4 * m4);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float yv = kk == 0 ? y[q].x : kk == 1 ? y[q].y : kk == 2 ? y[q].z : y[q].w;
                        acc[q][4 * m4 + 0] = fmaf(yv, x.x, acc[q][4 * m4 + 0]);
                        acc[q][4 * m4 + 1] = fmaf(yv, x.y, acc[q][4 * m4 + 1]);
                        acc[q][4 * m4 + 2] = fmaf(yv, x.z, acc[q][4 * m4 + 2]);
                        acc[q][4 * m4 + 3] = fmaf(yv, x.w, acc[q][4 * m4 + 3]);
                    }
                }
            }
        }
        __syncthreads();
        if (--chunk_left == 0 || s == nst - 1) {
            // end of a chunk of 4096 ia: the FP32 sums into the FP64 partial
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int P = P0 + t + 64 * q;
#pragma unroll
                for (int m = 0; m < MB; ++m) {
                    if (P < nJ && m < mm) {
                        double *o = out + (long long)P * mm + m;
                        *o = first ? (double)acc[q][m] : *o + (double)acc[q][m];
                    }
                    acc[q][m] = 0.f;
                }
            }
            first = false;
            chunk_left = JC_CHUNK / JC_KK;
        }
    }
}

// J expansion: AX[m][ia] += alpha sum_P Z[P][m] Y[P][ia] for Q consecutive ia
// per thread (Q MB = 64 accumulators: Q = 4 for MB = 16, 2 for MB = 32) and
// m < MB, FP32 sums over P.  Y is read once, straight from global memory (the
// lanes of a warp cover 32 Q consecutive ia); Z sits in shared memory in tiles
// of 256 aux functions, read as broadcast float4 loads.  VEC: the rows of Y
// start on (4 Q)-byte boundaries, so that each thread loads its Q values as one
// vector.
constexpr int JE_THREADS = 128, JE_PT = 256;

template <int MB, int Q, bool VEC>
__global__ void __launch_bounds__(JE_THREADS)
    je2_kernel(const float *__restrict__ Y, const float *__restrict__ Z, int nJ, int mm, long long nov, double alpha,
               double *__restrict__ AX)
{
    __shared__ __align__(16) float zs[JE_PT * MB];
    const long long ia = ((long long)blockIdx.x * JE_THREADS + threadIdx.x) * Q;
    float acc[Q][MB];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int m = 0; m < MB; ++m) acc[q][m] = 0.f;
    for (int P0 = 0; P0 < nJ; P0 += JE_PT) {
        const int np = min(JE_PT, nJ - P0);
        __syncthreads();
        for (int e = threadIdx.x; e < np * MB; e += JE_THREADS) {
            const int p = e / MB, m = e - p * MB;
            zs[e] = m < mm ? Z[(long long)(P0 + p) * mm + m] : 0.f;
        }
        __syncthreads();
        const float *yp = Y + (long long)P0 * nov + ia;
        // the Y values of 8 aux functions are loaded before any is used: 8 loads in
        // flight per thread hide the HBM latency
        for (int pb = 0; pb < np; pb += 8) {
            float y[8][Q];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float *yu = yp + (long long)(pb + u) * nov;
                if (pb + u < np && VEC && ia + Q - 1 < nov) {
                    if constexpr (Q == 4) {
                        const float4 v = __ldg((const float4 *)yu);
                        y[u][0] = v.x, y[u][1] = v.y, y[u][2] = v.z, y[u][3] = v.w;
                    } else {
                        const float2 v = __ldg((const float2 *)yu);
                        y[u][0] = v.x, y[u][1] = v.y;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < Q; ++q) y[u][q] = (pb + u < np && ia + q < nov) ? __ldg(yu + q) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (pb + u >= np) break;
#pragma unroll
                for (int m4 = 0; m4 < MB / 4; ++m4) {
                    const float4 z = *(const float4 *)(zs + (pb + u) * MB + 4 * m4);
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        acc[q][4 * m4 + 0] = fmaf(z.x, y[u][q], acc[q][4 * m4 + 0]);
                        acc[q][4 * m4 + 1] = fmaf(z.y, y[u][q], acc[q][4 * m4 + 1]);
                        acc[q][4 * m4 + 2] = fmaf(z.z, y[u][q], acc[q][4 * m4 + 2]);
                        acc[q][4 * m4 + 3] = fmaf(z.w, y[u][q], acc[q][4 * m4 + 3]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        if (m >= mm) break;
        double *o = AX + (long long)m * nov + ia;
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (ia + q < nov) o[q] += alpha * (double)acc[q][m];
    }
}

// Z[P][m] = sum_s part[s][P][m] (FP64, fixed order)
__global__ void jc_reduce(const double *__restrict__ part, int nsplit, long long n, double *__restrict__ Z)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double z = 0.0;
        for (int s = 0; s < nsplit; ++s) z += part[(long long)s * n + e];
        Z[e] = z;
    }
}

__global__ void to_f32(const double *__restrict__ x, float *__restrict__ y, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        y[t] = (float)x[t];
}

__global__ void mixed_diag(const double *__restrict__ D, const double *__restrict__ X, double *__restrict__ AX,
                           long long nov, int m)
{
    // one pass over the index ia: D read once, then the m vectors (no division per element)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nov; i += (long long)gridDim.x * blockDim.x) {
        const double d = D[i];
#pragma unroll 4
        for (int j = 0; j < m; ++j) AX[(long long)j * nov + i] = d * X[(long long)j * nov + i];
    }
}

unsigned gfor(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>(cdiv(n, 256), 152 * 16)); }

// Z[P][m] = sum_ia Y32[P][ia] X32[m][ia] into Z (FP64 [nJ][mm]): split over ia
// so that about ten CTAs of two warps per SM stream (P|ia); partials in the
// split-K workspace, reduced in a fixed order
void j_contract(tr_ctx *c, int mm, double *Z)
{
    const int nJ = c->nJ;
    const long long nov = c->nov;
    const int nPt = (int)cdiv(nJ, JC_TP);
    const long long target = std::max<long long>(1, (152LL * 10) / nPt);
    long long per = std::max<long long>(JC_KK, (nov + target - 1) / target);
    per = (per + JC_KK - 1) / JC_KK * JC_KK;
    const long long cap = std::max<long long>(1, (long long)c->ws_split.n / ((long long)nJ * mm));
    if ((nov + per - 1) / per > cap) per = ((nov + cap - 1) / cap + JC_KK - 1) / JC_KK * JC_KK;
    const int nsplit = (int)std::max<long long>(1, (nov + per - 1) / per);
    TR_REQUIRE(nsplit <= 65535, TR_EINVAL, "J contraction: too many ia splits");
    const size_t smem = 2 * JC_STAGE * sizeof(float);
    const dim3 grid(nPt, nsplit);
    const bool vec = nov % 4 == 0;
    const double flops = 2.0 * nJ * mm * (double)nov, bytes = 4.0 * nJ * (double)nov + 4.0 * nPt * mm * (double)nov;
#define TR_JC(MB, V) \
    TR_LAUNCH(c->prof, c->st, "J_contract", flops, bytes, \
              (jc_kernel<MB, V><<<grid, JC_THREADS, smem, c->st>>>(c->Y32.p, c->X32.p, nJ, mm, nov, per, c->ws_split.p)))
    if (mm <= 16) {
        if (vec) TR_JC(16, true);
        else TR_JC(16, false);
    } else {
        if (vec) TR_JC(32, true);
        else TR_JC(32, false);
    }
#undef TR_JC
    const long long n = (long long)nJ * mm;
    TR_LAUNCH(c->prof, c->st, "J_contract", 0, 8.0 * n * (nsplit + 1),
              jc_reduce<<<gfor(n), 256, 0, c->st>>>(c->ws_split.p, nsplit, n, Z));
}

// AX[m][ia] += 2 sum_P Z32[P][m] Y32[P][ia]
void j_expand(tr_ctx *c, int mm, double *ax)
{
    const int nJ = c->nJ;
    const long long nov = c->nov;
    const double flops = 2.0 * nJ * mm * (double)nov, bytes = 4.0 * nJ * (double)nov + 16.0 * mm * (double)nov;
#define TR_JE(MB, Q, V) \
    TR_LAUNCH(c->prof, c->st, "J_expand", flops, bytes, \
              (je2_kernel<MB, Q, V><<<(unsigned)cdiv(nov, (long long)Q * JE_THREADS), JE_THREADS, 0, c->st>>>( \
                  c->Y32.p, c->Z32.p, nJ, mm, nov, 2.0, ax)))
    if (mm <= 16) {
        if (nov % 4 == 0) TR_JE(16, 4, true);
        else TR_JE(16, 4, false);
    } else {
        if (nov % 2 == 0) TR_JE(32, 2, true);
        else TR_JE(32, 2, false);
    }
#undef TR_JE
}

int pad32(int x) { return (x + 31) / 32 * 32; }

}  // namespace

namespace {

__global__ void unpad_f32(const float *__restrict__ x, long long rows, int cols, int ld, double *__restrict__ y)
{
    const long long tot = rows * cols;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / cols;
        y[t] = (double)x[r * ld + (t - r * cols)];
    }
}

}  // namespace

void get_tensor_mixed(tr_ctx *c, int which, double *out, int on_device)
{
    DevBuf<double> tmp;
    size_t n = 0;
    TR_REQUIRE(which != 0 || !c->opt.j_ao, TR_EINVAL, "get_tensor: (P|ia) is not built with j_ao = 1");
    if (which == 0) {
        n = (size_t)c->nJ * c->nov;
        if (!n) return;
        tmp.alloc(n, &c->budget, "tensor copy");
        TR_LAUNCH(c->prof, c->st, "unpad", 0, 0,
                  unpad_f32<<<gfor(n), 256, 0, c->st>>>(c->Y32.p, (long long)c->nJ * c->nocc, c->nvir, c->nvir, tmp.p));
    } else {
        n = c->k_active ? (size_t)c->nK * c->vK * c->vK : 0;
        if (!n) return;
        tmp.alloc(n, &c->budget, "tensor copy");
        TR_LAUNCH(c->prof, c->st, "unpad", 0, 0,
                  unpad_f32<<<gfor(n), 256, 0, c->st>>>(c->Tab_h.p, (long long)c->nK * c->vK, c->vK, c->vKp, tmp.p));
    }
    TR_CUDA(cudaMemcpyAsync(out, tmp.p, sizeof(double) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->st));
    TR_CUDA(cudaStreamSynchronize(c->st));
}

// After the FP64 transforms: (P|ia) rounded to FP32 for the J contractions;
// T_ab^P and T_ij^P (metric applied) split into value and tf32 remainder with
// padded rows for the tensor-core K contraction; tensor maps of the K operands.
// The MO transforms themselves stay FP64: with C = S^-1/2 Q the sums over AO
// indices cancel terms tens of times larger than their result, and FP32
// accumulation on the tensor cores then leaves ~1e-4 relative errors in
// (P|ia), too close to the 1e-5 Ha target of this form.
void build_mixed(tr_ctx *c)
{
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const long long nov = c->nov;
    if (c->opt.j_ao) {
        c->Y32.release();  // the Coulomb term is formed in the AO basis
    } else {
        c->Y32.alloc((size_t)std::max(c->nJ, 1) * nov, &c->budget, "(P|ia) FP32");
        if (c->nJ)
            TR_LAUNCH(pf, st, "to_f32", 0, 12.0 * c->nJ * nov,
                      to_f32<<<gfor(c->nJ * nov), 256, 0, st>>>(c->Y.p, c->Y32.p, c->nJ * nov));
    }
    c->oKp = pad32(std::max(c->oK, 1));
    c->vKp = pad32(std::max(c->vK, 1));
    if (c->k_active) {
        const int nK = c->nK, oK = c->oK, vK = c->vK, oKp = c->oKp, vKp = c->vKp;
        c->Tab_h.alloc((size_t)nK * vK * vKp, &c->budget, "T_ab FP32");
        c->Tab_l.alloc((size_t)nK * vK * vKp, &c->budget, "T_ab FP32");
        tc_split(pf, st, c->Tab.p, (long long)nK * vK, vK, vK, c->Tab_h.p, c->Tab_l.p, vKp);
        c->T2_h.alloc((size_t)oK * nK * oKp, &c->budget, "T_ij FP32");
        c->T2_l.alloc((size_t)oK * nK * oKp, &c->budget, "T_ij FP32");
        TR_CUDA(cudaMemsetAsync(c->T2_h.p, 0, sizeof(float) * c->T2_h.n, st));
        TR_CUDA(cudaMemsetAsync(c->T2_l.p, 0, sizeof(float) * c->T2_l.n, st));
        tc_split(pf, st, c->T2.p, (long long)oK * nK, oK, oK, c->T2_h.p, c->T2_l.p, oKp);
        tc_make(c->tm_tab, c->Tab_h.p, c->Tab_l.p, (long long)nK * vK, vK, vKp);
        tc_make(c->tm_t2, c->T2_h.p, c->T2_l.p, oK, (long long)nK * oKp, (long long)nK * oKp);
    }
    // the FP32 copies are what the products use; the FP64 (P|ia) and T_ab are freed
    TR_CUDA(cudaStreamSynchronize(st));
    c->Y.release();
    c->Tab.release();
    c->mixed_mb = 0;  // workspaces are sized at the first product
}

void reserve_mixed(tr_ctx *c, int mb)
{
    if (mb <= c->mixed_mb) return;
    const long long nov = c->nov;
    c->X32.alloc((size_t)mb * nov, &c->budget, "X FP32");
    c->Z32.alloc((size_t)std::max(c->nJ, 1) * mb, &c->budget, "J workspace");
    if (c->k_active) {
        const int nK = c->nK, oK = c->oK, vK = c->vK, oKp = c->oKp, vKp = c->vKp;
        c->Xw_h.alloc((size_t)mb * oK * vKp, &c->budget, "K workspace");
        c->Xw_l.alloc((size_t)mb * oK * vKp, &c->budget, "K workspace");
        const size_t perP = (size_t)mb * vK * oKp * 2 * sizeof(float);
        int npk = (int)std::max<size_t>(1, c->opt.matvec_ws_bytes / perP);
        npk = std::min(npk, nK);
        npk = std::min(npk, 65535 / mb);
        c->mixed_npk = npk;
        c->Mt_h.alloc((size_t)mb * vK * npk * oKp, &c->budget, "K workspace");
        c->Mt_l.alloc((size_t)mb * vK * npk * oKp, &c->budget, "K workspace");
        // the padding columns j >= oK of every aux block stay zero for good
        TR_CUDA(cudaMemsetAsync(c->Mt_h.p, 0, sizeof(float) * c->Mt_h.n, c->st));
        TR_CUDA(cudaMemsetAsync(c->Mt_l.p, 0, sizeof(float) * c->Mt_l.n, c->st));
        tc_make(c->tm_xw, c->Xw_h.p, c->Xw_l.p, (long long)mb * oK, vK, vKp);
        tc_make(c->tm_mt, c->Mt_h.p, c->Mt_l.p, (long long)mb * vK, (long long)npk * oKp, (long long)npk * oKp);
    }
    c->mixed_mb = mb;
}

void matvec_mixed(tr_ctx *c, int m, const double *X, double *AX)
{
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ, nK = c->nK;
    const int oK = c->oK, vK = c->vK, o0 = c->o0, oKp = c->oKp, vKp = c->vKp;
    const long long nov = c->nov;
    const int mb = std::min(m, c->mblk);
    reserve_matvec(c, mb);
    int *tc_err = c->flag.p + 1;
    for (int m0 = 0; m0 < m; m0 += mb) {
        const int mm = std::min(mb, m - m0);
        const double *x = X + (long long)m0 * nov;
        double *ax = AX + (long long)m0 * nov;
        TR_LAUNCH(pf, st, "diag", 0, 8.0 * nov * (2.0 * mm + 1.0), mixed_diag<<<gfor(nov), 256, 0, st>>>(c->D.p, x, ax, nov, mm));
        TR_LAUNCH(pf, st, "prepare_f32", 0, 12.0 * nov * mm,
                  mixed_prepare<<<gfor(nov * mm), 256, 0, st>>>(x, c->X32.p, c->k_active ? c->Xw_h.p : nullptr,
                                                                 c->k_active ? c->Xw_l.p : nullptr, mm, nocc, nvir,
                                                                 c->k_active ? o0 : nocc, oK, vK, vKp));
        if (nJ && c->opt.j_ao) {
            j_ao_block(c, mm, x, ax);  // Coulomb term in FP64 from the AO transition densities
        } else if (nJ) {
            j_contract(c, mm, c->ws_Z.p);
            dgemm(pf, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, c->ws_Z.p, mm, 0.0, c->ws_Z2.p,
                  mm, Batch(), nullptr, 0);
            TR_LAUNCH(pf, st, "to_f32", 0, 0, to_f32<<<gfor((long long)nJ * mm), 256, 0, st>>>(c->ws_Z2.p, c->Z32.p, (long long)nJ * mm));
            j_expand(c, mm, ax);
        }
        if (c->k_active) {
            const int npk = c->mixed_npk;
            for (int P0 = 0; P0 < nK; P0 += npk) {
                const int np = std::min(npk, nK - P0);
                // stage 1: M^P_mja = sum_b X_mjb T_ab^P, written split as Mt[m][a][P][j]
                TcOut o1;
                o1.mode = TC_SPLIT;
                o1.hi = c->Mt_h.p;
                o1.lo = c->Mt_l.p;
                o1.ldm = 1;
                o1.ldn = (long long)npk * oKp;
                o1.s1 = (long long)vK * npk * oKp;
                o1.s2 = oKp;
                const double b1 = 4.0 * 2 * ((double)mm * np * vK * oK + (double)mm * oK * vK + (double)np * vK * vK);
                tc_gemm(pf, st, "K_stage1_tc", 3, c->tm_xw, 0, oK, 0, 0, c->tm_tab, (long long)P0 * vK, 0, vK, 0, oK,
                        vK, vK, mm, np, o1, tc_err, b1, c->tc_bn);
                // stage 2: AX_mia -= c_x sum_(P,j) T_ij^P M^P_mja
                TcOut o2;
                o2.mode = TC_ACC64;
                o2.d = ax + (long long)o0 * nvir;
                o2.alpha = -c->opt.cx;
                o2.ldm = nvir;
                o2.ldn = 1;
                o2.s1 = nov;
                const double b2 = 4.0 * 2 * ((double)mm * np * vK * oKp + (double)oK * np * oKp) + 16.0 * mm * oK * vK;
                tc_gemm(pf, st, "K_stage2_tc", 3, c->tm_t2, 0, 0, 0, P0 * oKp, c->tm_mt, 0, vK, 0, 0, oK, vK, np * oKp,
                        mm, 1, o2, tc_err, b2, c->tc_bn);
            }
        }
    }
}

}  // namespace tr
