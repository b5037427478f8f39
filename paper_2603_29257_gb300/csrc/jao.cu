// Coulomb term on the fly in the AO basis (Sec. 3.1, Eq. J_mia and the four
// contractions that follow it): no (P|ia) tensor is stored.  For a block of
// m trial vectors
//   D^m_kl  = sum_jb C_kj C_lb X_mjb                (AO transition densities)
//   R_mQ    = sum_kl (Q|kl) D^m_kl                  (integrals per auxiliary chunk)
//   R~_mP   = sum_Q (P|Q)^-1 R_mQ
//   U^m_mn  = sum_P (mn|P) R~_mP                    (the chunks generated again)
//   J_mia   = sum_mn C_mi C_na U^m_mn,              AX += 2 J
// all in FP64.  The three-centre integrals of a chunk are generated as full
// symmetric nao x nao matrices, so D need not be symmetrised.  Both integral
// contractions run over the function pairs (k, l) of the screened shell pairs
// only (Sec. 3.1: the sparsity of the AO pairs): the chunk and the densities
// are gathered to those pairs, the potentials come out packed and are scattered
// back (zero elsewhere, where every integral is zero).  When every auxiliary
// function fits in one chunk the integrals are generated once per pass and
// serve both contractions.  The integral chunk and the vectors' AO densities
// and potentials are each held within the chunk budget (aux_chunk_bytes): a
// large molecule runs a few vectors per pass, over many chunks, but never
// stores an N_aux x nov tensor.
#include <algorithm>

#include "ctx.cuh"

namespace tr {

namespace {

// auxiliary functions per integral chunk: whole J atoms (multiples of 4) within
// the chunk budget (the dense chunk and its packed copy)
int jao_chunk(const tr_ctx *c)
{
    const double per = 8.0 * (double)c->nao * c->nao * 1.5;
    int npc = (int)std::max(1.0, std::floor((double)c->opt.aux_chunk_bytes / per));
    npc = std::min(npc, std::max(c->nJ, 1));
    if (npc >= 4) npc = npc / 4 * 4;
    return npc;
}

// vectors per pass: their AO densities and potentials (2 nao^2 doubles each, plus
// the packed copies) within the same budget, so that large molecules run a few
// vectors at a time
int jao_vectors(const tr_ctx *c, int mb)
{
    const double per = 24.0 * (double)c->nao * c->nao;
    return std::max(1, std::min(mb, (int)std::floor((double)c->opt.aux_chunk_bytes / per)));
}

// flat indices k nao + l of the function pairs of the kept shell pairs (both
// orders), ascending; built once per molecule
void list_pairs(tr_ctx *c)
{
    if (c->nkl >= 0) return;
    const long long nao = c->nao;
    std::vector<int> idx;
    for (const int2 &ab : c->pl.pairs) {
        const ShellDev &A = c->shells_h[ab.x], &B = c->shells_h[ab.y];
        const int na = 2 * A.l + 1, nb = 2 * B.l + 1;
        for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j) {
                idx.push_back((int)((A.ao + i) * nao + B.ao + j));
                if (ab.x != ab.y) idx.push_back((int)((B.ao + j) * nao + A.ao + i));
            }
    }
    std::sort(idx.begin(), idx.end());
    idx.erase(std::unique(idx.begin(), idx.end()), idx.end());
    c->nkl = (long long)idx.size();
    c->kl_idx.alloc(std::max<size_t>(idx.size(), 1), &c->budget, "AO pair list");
    if (!idx.empty())
        TR_CUDA(cudaMemcpy(c->kl_idx.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
}

// dst[r][t] = src[r * ld + idx[t]] for r < rows, t < n
__global__ void gather_pairs(const double *__restrict__ src, long long ld, int rows, const int *__restrict__ idx,
                             long long n, double *__restrict__ dst)
{
    const long long tot = (long long)rows * n;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
        const long long r = u / n, t = u - r * n;
        dst[u] = src[r * ld + idx[t]];
    }
}

// dst[r * ld + idx[t]] = src[r][t] (the rest of dst zeroed beforehand)
__global__ void scatter_pairs(const double *__restrict__ src, long long ld, int rows, const int *__restrict__ idx,
                              long long n, double *__restrict__ dst)
{
    const long long tot = (long long)rows * n;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < tot; u += (long long)gridDim.x * blockDim.x) {
        const long long r = u / n, t = u - r * n;
        dst[r * ld + idx[t]] = src[u];
    }
}

unsigned pair_grid(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>(cdiv(n, 256), 152 * 16)); }

}  // namespace

void reserve_jao(tr_ctx *c, int mb)
{
    const long long nao = c->nao, nao2 = nao * nao;
    const int mv = jao_vectors(c, mb);
    list_pairs(c);
    const size_t nkl = (size_t)std::max<long long>(c->nkl, 1);
    c->ws_jT.reserve((size_t)mv * c->nocc * nao, &c->budget, "AO J half-transformed densities");
    c->ws_jD.reserve((size_t)mv * nao2, &c->budget, "AO transition densities");
    c->ws_jU.reserve((size_t)mv * nao2, &c->budget, "AO J potential");
    c->ws_jDp.reserve((size_t)mv * nkl, &c->budget, "AO transition densities on the kept pairs");
    c->ws_jUp.reserve((size_t)mv * nkl, &c->budget, "AO J potential on the kept pairs");
    c->ws_jR.reserve((size_t)2 * std::max(c->nJ, 1) * mv, &c->budget, "AO J fit coefficients");
    if (c->nJ > 0) {
        c->ws_jI.reserve((size_t)jao_chunk(c) * nao2, &c->budget, "AO J integral chunk");
        c->ws_jIp.reserve((size_t)jao_chunk(c) * nkl, &c->budget, "AO J integral chunk on the kept pairs");
    }
}

int jao_chunk_size(const tr_ctx *c) { return jao_chunk(c); }

size_t jao_bytes(const tr_ctx *c, int mb)
{
    const double nao = c->nao, nao2 = nao * nao;
    const double mv = jao_vectors(c, mb);
    // the pair list is not known before the molecule's pairs are; bound it by nao^2
    const double nkl = c->nkl >= 0 ? (double)c->nkl : nao2;
    const double chunk = c->nJ > 0 ? (double)jao_chunk(c) * (nao2 + nkl) : 0.0;
    return (size_t)(8.0 * (mv * c->nocc * nao + 2.0 * mv * (nao2 + nkl) + 2.0 * std::max(c->nJ, 1) * mv + chunk) +
                    4.0 * nkl);
}

namespace {
void j_ao_pass(tr_ctx *c, int mm, const double *X, double *AX);
}

void j_ao_block(tr_ctx *c, int mm, const double *X, double *AX)
{
    if (c->nJ == 0 || mm <= 0) return;
    const int mv = jao_vectors(c, mm);
    for (int m0 = 0; m0 < mm; m0 += mv)
        j_ao_pass(c, std::min(mv, mm - m0), X + (long long)m0 * c->nov, AX + (long long)m0 * c->nov);
}

namespace {

void j_ao_pass(tr_ctx *c, int mm, const double *X, double *AX)
{
    const int nJ = c->nJ;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nao = c->nao, nmo = c->nmo, nocc = c->nocc, nvir = c->nvir;
    const long long nov = c->nov, nao2 = (long long)nao * nao;
    TR_REQUIRE(nao2 < (1LL << 31), TR_EINVAL, "AO J: nao^2 must fit in 32 bits");
    reserve_jao(c, mm);
    const long long nkl = c->nkl;
    double *T = c->ws_jT.p, *D = c->ws_jD.p, *U = c->ws_jU.p, *R = c->ws_jR.p, *Rt = c->ws_jR.p + (size_t)nJ * mm;
    double *I = c->ws_jI.p, *Ip = c->ws_jIp.p, *Dp = c->ws_jDp.p, *Up = c->ws_jUp.p;
    const int *kl = c->kl_idx.p;
    const double *C = c->C.p;
    // D^m = C_occ (X^m C_vir^T): T[m][j][l] = sum_b X_mjb C_lb, then D[m][k][l] = sum_j C_kj T[m][j][l]
    Batch b1;
    b1.n1 = mm;
    b1.sA1 = nov;
    b1.sC1 = (long long)nocc * nao;
    dgemm(pf, st, "J_ao_density", false, true, nocc, nao, nvir, 1.0, X, nvir, C + nocc, nmo, 0.0, T, nao, b1,
          nullptr, 0);
    Batch b2;
    b2.n1 = mm;
    b2.sB1 = (long long)nocc * nao;
    b2.sC1 = nao2;
    dgemm(pf, st, "J_ao_density", false, false, nao, nao, nocc, 1.0, C, nmo, T, nao, 0.0, D, nao, b2, nullptr, 0);
    TR_LAUNCH(pf, st, "J_ao_pack", 0, 16.0 * mm * (double)nkl,
              gather_pairs<<<pair_grid(mm * nkl), 256, 0, st>>>(D, nao2, mm, kl, nkl, Dp));
    // R[Q][m] = sum_kl (Q|kl) D^m_kl over the kept pairs, chunk by chunk
    const int npc = jao_chunk(c);
    const bool one_chunk = npc >= nJ;
    auto chunk = [&](int p0, int np) {
        compute_int3c_chunk(c, 0, p0, np, I);
        TR_LAUNCH(pf, st, "J_ao_pack", 0, 16.0 * np * (double)nkl,
                  gather_pairs<<<pair_grid(np * nkl), 256, 0, st>>>(I, nao2, np, kl, nkl, Ip));
    };
    for (int p0 = 0; p0 < nJ; p0 += npc) {
        const int np = std::min(npc, nJ - p0);
        chunk(p0, np);
        dgemm(pf, st, "J_ao_fit", false, true, np, mm, (int)nkl, 1.0, Ip, nkl, Dp, nkl, 0.0, R + (long long)p0 * mm,
              mm, Batch(), c->ws_split.p, c->ws_split.n);
    }
    // R~ = (P|Q)^-1 R
    dgemm(pf, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, R, mm, 0.0, Rt, mm, Batch(), nullptr, 0);
    // U^m = sum_P R~_mP (P|kl) on the kept pairs: the chunks again (kept from the first pass when there is one)
    for (int p0 = 0; p0 < nJ; p0 += npc) {
        const int np = std::min(npc, nJ - p0);
        if (!one_chunk) chunk(p0, np);
        dgemm(pf, st, "J_ao_potential", true, false, mm, (int)nkl, np, 1.0, Rt + (long long)p0 * mm, mm, Ip, nkl,
              p0 == 0 ? 0.0 : 1.0, Up, nkl, Batch(), nullptr, 0);
    }
    TR_CUDA(cudaMemsetAsync(U, 0, sizeof(double) * (size_t)mm * nao2, st));
    TR_LAUNCH(pf, st, "J_ao_pack", 0, 16.0 * mm * (double)nkl,
              scatter_pairs<<<pair_grid(mm * nkl), 256, 0, st>>>(Up, nao2, mm, kl, nkl, U));
    // AX_mia += 2 sum_kl C_ki C_la U^m_kl: T[m][i][l] = sum_k C_ki U^m_kl, then AX += 2 T C_vir
    Batch b3;
    b3.n1 = mm;
    b3.sB1 = nao2;
    b3.sC1 = (long long)nocc * nao;
    dgemm(pf, st, "J_ao_back", true, false, nocc, nao, nao, 1.0, C, nmo, U, nao, 0.0, T, nao, b3, nullptr, 0);
    Batch b4;
    b4.n1 = mm;
    b4.sA1 = (long long)nocc * nao;
    b4.sC1 = nov;
    dgemm(pf, st, "J_ao_back", false, false, nocc, nvir, nao, 2.0, T, nao, C + nocc, nmo, 1.0, AX, nvir, b4, nullptr,
          0);
}

}  // namespace
}  // namespace tr
