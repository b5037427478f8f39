// Transition properties of the converged states (Sec. 2, Eqs.
// oscillator_strength and transition, Tamm-Dancoff: Y = 0):
//   r^d_ia = sum_mn C_mi <m| r_d - O_d |n> C_na            (dipole length form)
//   mu_kd  = sqrt(2) sum_ia r^d_ia X_kia                    (singlet, unit-norm X)
//   f_k    = 2/3 Omega_k |mu_k|^2
// The AO dipole integrals come from the McMurchie-Davidson kernel over the
// screened shell pairs; the MO transform and the contraction with X are FP64
// GEMMs; f is formed on the device.
#include <cmath>

#include "ctx.cuh"

namespace tr {

namespace {

__global__ void osc_kernel(const double *__restrict__ omega, const double *__restrict__ mu, int n,
                           double *__restrict__ f)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double x = mu[3 * k], y = mu[3 * k + 1], z = mu[3 * k + 2];
    f[k] = (2.0 / 3.0) * omega[k] * (x * x + y * y + z * z);
}

}  // namespace

void transition_dipoles(tr_ctx *c, int n, const double *X, const double O[3], double *mu)
{
    TR_REQUIRE(c->have_mol && c->have_orb, TR_EINVAL, "transition dipoles: molecule and orbitals required");
    if (n <= 0) return;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nao = c->nao, nmo = c->nmo, nocc = c->nocc, nvir = c->nvir;
    const long long nov = c->nov, nao2 = (long long)nao * nao;
    DevBuf<double> M, T, R;
    M.alloc((size_t)3 * nao2, &c->budget, "dipole integrals");
    T.alloc((size_t)3 * nocc * nao, &c->budget, "dipole half transform");
    R.alloc((size_t)3 * nov, &c->budget, "dipole MO integrals");
    dipole_ints(pf, st, c->shells.p, c->pairs.p, c->prange.p, c->prim.p, c->pl.off, nao, O, M.p);
    // r^d = C_occ^T M^d C_vir for d = x, y, z
    Batch b1;
    b1.n1 = 3;
    b1.sB1 = nao2;
    b1.sC1 = (long long)nocc * nao;
    dgemm(pf, st, "dipole_mo", true, false, nocc, nao, nao, 1.0, c->C.p, nmo, M.p, nao, 0.0, T.p, nao, b1, nullptr, 0);
    Batch b2;
    b2.n1 = 3;
    b2.sA1 = (long long)nocc * nao;
    b2.sC1 = nov;
    dgemm(pf, st, "dipole_mo", false, false, nocc, nvir, nao, 1.0, T.p, nao, c->C.p + nocc, nmo, 0.0, R.p, nvir, b2,
          nullptr, 0);
    // mu[k][d] = sqrt(2) sum_ia X[k][ia] r^d_ia
    dgemm(pf, st, "transition_dipole", false, true, n, 3, (int)nov, std::sqrt(2.0), X, nov, R.p, nov, 0.0, mu, 3,
          Batch(), c->ws_split.p, c->ws_split.n);
    TR_CUDA(cudaStreamSynchronize(st));  // the scratch is freed on return
}

void oscillator_strengths(tr_ctx *c, int n, const double *omega, const double *X, double *f)
{
    if (n <= 0) return;
    DevBuf<double> mu;
    mu.alloc((size_t)3 * n, &c->budget, "transition dipoles");
    const double O[3] = {0.0, 0.0, 0.0};
    transition_dipoles(c, n, X, O, mu.p);
    TR_LAUNCH(c->prof, c->st, "oscillator", 0, 0, osc_kernel<<<cdiv(n, 64), 64, 0, c->st>>>(omega, mu.p, n, f));
    TR_CUDA(cudaStreamSynchronize(c->st));
}

}  // namespace tr
