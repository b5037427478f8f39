// Coulomb term on the fly in the AO basis (Sec. 3.1, Eq. J_mia and the four
// contractions that follow it): no (P|ia) tensor is stored.  For a block of
// m trial vectors
//   D^m_kl  = sum_jb C_kj C_lb X_mjb                (AO transition densities)
//   R_mQ    = sum_kl (Q|kl) D^m_kl                  (integrals per auxiliary chunk)
//   R~_mP   = sum_Q (P|Q)^-1 R_mQ
//   U^m_mn  = sum_P (mn|P) R~_mP                    (the chunks generated again)
//   J_mia   = sum_mn C_mi C_na U^m_mn,              AX += 2 J
// all in FP64.  The three-centre integrals of a chunk are the full symmetric
// nao x nao matrices of its auxiliary functions, so D need not be symmetrised
// and the contractions are dense GEMMs.  When every auxiliary function fits in
// one chunk the integrals are generated once per pass and serve both contractions.
// The integral chunk and the vectors' AO densities and potentials are each held
// within the chunk budget (aux_chunk_bytes): a large molecule runs a few vectors
// per pass, over many chunks, but never stores an N_aux x nov tensor.
#include <algorithm>

#include "ctx.cuh"

namespace tr {

namespace {

// auxiliary functions per integral chunk: whole J atoms (multiples of 4) within
// the chunk budget
int jao_chunk(const tr_ctx *c)
{
    const double per = 8.0 * (double)c->nao * c->nao;
    int npc = (int)std::max(1.0, std::floor((double)c->opt.aux_chunk_bytes / per));
    npc = std::min(npc, std::max(c->nJ, 1));
    if (npc >= 4) npc = npc / 4 * 4;
    return npc;
}

// vectors per pass: their AO densities and potentials (2 nao^2 doubles each) within
// the same budget, so that large molecules run a few vectors at a time
int jao_vectors(const tr_ctx *c, int mb)
{
    const double per = 16.0 * (double)c->nao * c->nao;
    return std::max(1, std::min(mb, (int)std::floor((double)c->opt.aux_chunk_bytes / per)));
}

}  // namespace

void reserve_jao(tr_ctx *c, int mb)
{
    const long long nao = c->nao, nao2 = nao * nao;
    const int mv = jao_vectors(c, mb);
    c->ws_jT.reserve((size_t)mv * c->nocc * nao, &c->budget, "AO J half-transformed densities");
    c->ws_jD.reserve((size_t)mv * nao2, &c->budget, "AO transition densities");
    c->ws_jU.reserve((size_t)mv * nao2, &c->budget, "AO J potential");
    c->ws_jR.reserve((size_t)2 * std::max(c->nJ, 1) * mv, &c->budget, "AO J fit coefficients");
    if (c->nJ > 0) c->ws_jI.reserve((size_t)jao_chunk(c) * nao2, &c->budget, "AO J integral chunk");
}

int jao_chunk_size(const tr_ctx *c) { return jao_chunk(c); }

size_t jao_bytes(const tr_ctx *c, int mb)
{
    const double nao = c->nao, nao2 = nao * nao;
    const double mv = jao_vectors(c, mb);
    const double chunk = c->nJ > 0 ? (double)jao_chunk(c) * nao2 : 0.0;
    return (size_t)(8.0 * (mv * c->nocc * nao + 2.0 * mv * nao2 + 2.0 * std::max(c->nJ, 1) * mv + chunk));
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
    double *T = c->ws_jT.p, *D = c->ws_jD.p, *U = c->ws_jU.p, *R = c->ws_jR.p, *Rt = c->ws_jR.p + (size_t)nJ * mm;
    double *I = c->ws_jI.p;
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
    // R[Q][m] = sum_kl (Q|kl) D^m_kl, chunk by chunk
    const int npc = jao_chunk(c);
    const bool one_chunk = npc >= nJ;
    for (int p0 = 0; p0 < nJ; p0 += npc) {
        const int np = std::min(npc, nJ - p0);
        compute_int3c_chunk(c, 0, p0, np, I);
        dgemm(pf, st, "J_ao_fit", false, true, np, mm, (int)nao2, 1.0, I, nao2, D, nao2, 0.0, R + (long long)p0 * mm,
              mm, Batch(), c->ws_split.p, c->ws_split.n);
    }
    // R~ = (P|Q)^-1 R
    dgemm(pf, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, R, mm, 0.0, Rt, mm, Batch(), nullptr, 0);
    // U^m = sum_P R~_mP (P|kl): the chunks again (kept from the first pass when there is one)
    for (int p0 = 0; p0 < nJ; p0 += npc) {
        const int np = std::min(npc, nJ - p0);
        if (!one_chunk) compute_int3c_chunk(c, 0, p0, np, I);
        dgemm(pf, st, "J_ao_potential", true, false, mm, (int)nao2, np, 1.0, Rt + (long long)p0 * mm, mm, I, nao2,
              p0 == 0 ? 0.0 : 1.0, U, nao2, Batch(), nullptr, 0);
    }
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
