// Reduced-precision form of the TDA-risp matrix-vector product.
//
// Same operator as the FP64 form (Sec. 2 Eq. TDA-risp; Sec. 3.2 for K):
//   - the three-centre integrals, metrics and MO transforms are built in FP64
//     and the MO tensors are then rounded to FP32 (the paper builds its
//     integrals in FP64 and runs everything after them in FP32, Sec. 3.3);
//     see build_mixed for why the transforms themselves stay FP64;
//   - J: Z = (Q|jb) X and J = (P|ia) Zt as FP32 products on the CUDA cores (Z
//     summed in FP32 over chunks of at most 4096 terms and in FP64 across
//     chunks; the expansion by a kernel for blocks of at most 32 vectors);
//     (P|Q)^-1 is applied in FP64;
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

// J expansion for a block of at most 32 vectors (Sec. 3.1):
//   AX[m][ia] += alpha sum_P Z32[P][m] Y32[P][ia]
// in FP32 over P, added to the FP64 output.  A CTA covers 128 ia x 32 m (4 x 4 per
// thread); 32-row tiles of Y (coalesced along ia) and Z staged in shared memory.
__global__ void __launch_bounds__(256)
    je_kernel(const float *__restrict__ Y, const float *__restrict__ Z, int nJ, int mm, long long nov, double alpha,
              double *__restrict__ AX)
{
    __shared__ float4 Ys[32][32];
    __shared__ float4 Zs[32][8];
    float *ys = (float *)Ys, *zs = (float *)Zs;
    const int tid = threadIdx.x, ti = tid & 31, tm = tid >> 5;
    const long long i0 = (long long)blockIdx.x * 128;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    for (int P0 = 0; P0 < nJ; P0 += 32) {
        for (int e = tid; e < 32 * 128; e += 256) {
            const int p = e >> 7, c = e & 127;
            const long long ia = i0 + c;
            ys[p * 128 + c] = (P0 + p < nJ && ia < nov) ? Y[(long long)(P0 + p) * nov + ia] : 0.f;
        }
        for (int e = tid; e < 32 * 32; e += 256) {
            const int p = e >> 5, m = e & 31;
            zs[p * 32 + m] = (P0 + p < nJ && m < mm) ? Z[(long long)(P0 + p) * mm + m] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < 32; ++p) {
            const float4 y = Ys[p][ti];
            const float4 z = Zs[p][tm];
            const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[j][0] = fmaf(zz[j], y.x, acc[j][0]);
                acc[j][1] = fmaf(zz[j], y.y, acc[j][1]);
                acc[j][2] = fmaf(zz[j], y.z, acc[j][2]);
                acc[j][3] = fmaf(zz[j], y.w, acc[j][3]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = 4 * tm + j;
        if (m >= mm) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long ia = i0 + 4 * ti + q;
            if (ia < nov) AX[(long long)m * nov + ia] += alpha * (double)acc[j][q];
        }
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
            sgemm(pf, st, "J_contract", false, true, nJ, mm, (int)nov, 1.0, c->Y32.p, nov, c->X32.p, nov, 0.0,
                  c->ws_Z.p, mm, Batch(), c->ws_split.p, c->ws_split.n, 4096);
            dgemm(pf, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, c->ws_Z.p, mm, 0.0, c->ws_Z2.p,
                  mm, Batch(), nullptr, 0);
            TR_LAUNCH(pf, st, "to_f32", 0, 0, to_f32<<<gfor((long long)nJ * mm), 256, 0, st>>>(c->ws_Z2.p, c->Z32.p, (long long)nJ * mm));
            TR_LAUNCH(pf, st, "J_expand", 2.0 * nJ * mm * (double)nov, 4.0 * (double)nJ * nov + 16.0 * mm * (double)nov,
                      je_kernel<<<(unsigned)cdiv(nov, 128), 256, 0, st>>>(c->Y32.p, c->Z32.p, nJ, mm, nov, 2.0, ax));
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
