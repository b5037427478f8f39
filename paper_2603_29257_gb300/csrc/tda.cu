// TDA-risp operator on the GPU: molecule and orbital set-up, the build of
// the factorised operator and the matrix-vector product.
//
//   A X = (e_a - e_i) X + 2 J - c_x K                                Sec. 2, Eq. TDA-risp
//   J_mia = sum_P (P|ia) Zt_Pm,  Zt = (P|Q)^-1 Z,  Z_Qm = sum_jb (Q|jb) X_mjb
//          (RI in the Coulomb metric, Sec. 2 Eq. RI; the paper's J engine
//           applies (P|Q)^-1 to the small aux-by-state intermediate, Sec. 3.1)
//   K_mia = sum_P sum_j T_ij^P M^P_mja,  M^P_mja = sum_b T_ab^P X_mjb,
//          T_ij^P = sum_Q (ij|Q)(Q|P)^-1,  T_ab^P = (ab|P)             Sec. 3.2
//   with i, j, a, b inside the exchange window and K zero outside it.
#include <algorithm>
#include <numeric>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "ozgemm.cuh"

namespace tr {
namespace {

constexpr double HARTREE_EV = 27.211386245988;

__global__ void diag_kernel(const double *__restrict__ D, const double *__restrict__ X,
                            double *__restrict__ AX, long long nov, int m)
{
    // one pass over the index ia: D read once, then the m vectors (no division per element)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nov; i += (long long)gridDim.x * blockDim.x) {
        const double d = D[i];
#pragma unroll 4
        for (int j = 0; j < m; ++j) AX[(long long)j * nov + i] = d * X[(long long)j * nov + i];
    }
}

__global__ void gather_window(const double *__restrict__ X, double *__restrict__ Xw, int m, int nocc,
                              int nvir, int o0, int oK, int vK)
{
    long long tot = (long long)m * oK * vK;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int b = (int)(t % vK);
        long long r = t / vK;
        int j = (int)(r % oK);
        int mm = (int)(r / oK);
        Xw[t] = X[((long long)mm * nocc + o0 + j) * nvir + b];
    }
}

__global__ void orbital_diff(const double *__restrict__ eps, int nocc, int nvir, double *__restrict__ D)
{
    long long tot = (long long)nocc * nvir;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int a = (int)(t % nvir), i = (int)(t / nvir);
        D[t] = eps[nocc + a] - eps[i];
    }
}

// [P][i][j] <- [i][P][j]
__global__ void unpermute_T2(const double *__restrict__ T2, int nK, int oK, double *__restrict__ out)
{
    long long tot = (long long)nK * oK * oK;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int j = (int)(t % oK);
        long long r = t / oK;
        int i = (int)(r % oK);
        int P = (int)(r / oK);
        out[t] = T2[((long long)i * nK + P) * oK + j];
    }
}

// J functions per integral chunk: whole atoms (s, p_x, p_y, p_z), and a
// multiple of 8 atoms (the lane tile of the heavy integral kernels) where at
// least 8 fit
int j_chunk(int npc)
{
    if (npc >= 32) return npc / 32 * 32;
    return npc >= 4 ? npc / 4 * 4 : npc;
}

unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>(cdiv(n, 256), 152 * 16)); }

// class-sorted copy of auxiliary functions with out index in [p0, p0+np);
// cls[0..4] offsets for comp -1, 0, 1, 2; with grouped, the s functions of the
// chunk's atoms follow (their count in *natoms)
void aux_chunk(tr_ctx *c, const std::vector<AuxDev> &all, int p0, int np, int cls[5], bool grouped, int *natoms)
{
    std::vector<AuxDev> sorted;
    cls[0] = 0;
    for (int cd = -1; cd <= 2; ++cd) {
        for (const AuxDev &a : all)
            if (a.comp == cd && a.out >= p0 && a.out < p0 + np) {
                AuxDev b = a;
                b.out -= p0;
                sorted.push_back(b);
            }
        cls[cd + 2] = (int)sorted.size();
    }
    *natoms = 0;
    if (grouped) {
        for (int i = cls[0]; i < cls[1]; ++i) sorted.push_back(sorted[i]);  // s functions = whole atoms
        *natoms = cls[1] - cls[0];
    }
    c->aux_ws.reserve(std::max<size_t>(sorted.size(), 1), &c->budget, "aux list");
    if (!sorted.empty())
        TR_CUDA(cudaMemcpyAsync(c->aux_ws.p, sorted.data(), sizeof(AuxDev) * sorted.size(),
                                cudaMemcpyHostToDevice, c->st));
}

void compute_int3c(tr_ctx *c, const std::vector<AuxDev> &all, int p0, int np, double *out,
                   double ka, double kb, double omega)
{
    const int which = &all == &c->auxJ_h ? 0 : 1;
    TR_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * (size_t)np * c->nao * c->nao, c->st));
    for (const tr_ctx::AuxChunk &k : c->aux_cache_idx)
        if (k.which == which && k.p0 == p0 && k.np == np) {
            const AuxDev *a = c->aux_cache.p + k.off;
            int3c(c->prof, c->st, &c->side, c->shells.p, c->pairs.p, c->prange.p, c->prim.p, c->pl.off, a, k.cls,
                  a + k.cls[4], k.natoms, c->nao, out, ka, kb, omega, c->boys.p);
            return;
        }
    int cls[5], natoms = 0;
    // J chunks of whole atoms (s, p_x, p_y, p_z at out indices 4a .. 4a+3)
    const bool grouped = which == 0 && p0 % 4 == 0 && np % 4 == 0;
    aux_chunk(c, all, p0, np, cls, grouped, &natoms);
    int3c(c->prof, c->st, &c->side, c->shells.p, c->pairs.p, c->prange.p, c->prim.p, c->pl.off, c->aux_ws.p, cls,
          c->aux_ws.p + cls[4], natoms, c->nao, out, ka, kb, omega, c->boys.p);
    // the aux list lives in aux_ws until the kernels have read it
    TR_CUDA(cudaStreamSynchronize(c->st));
}


void metric(tr_ctx *c, const std::vector<AuxDev> &all, double ka, double kb, double omega, double *G)
{
    int n = (int)all.size();
    if (n == 0) return;
    c->aux_ws.reserve(n, &c->budget, "aux list");
    TR_CUDA(cudaMemcpyAsync(c->aux_ws.p, all.data(), sizeof(AuxDev) * n, cudaMemcpyHostToDevice, c->st));
    int2c(c->prof, c->st, c->aux_ws.p, n, ka, kb, omega, c->boys.p, G);
    TR_CUDA(cudaStreamSynchronize(c->st));
}

// Cholesky factor and inverse of a metric; throws TR_ENOTPD if not positive definite.
// Linv (optional, n x n): the inverse of the lower Cholesky factor L, G = L L^T.
void metric_inverse(tr_ctx *c, double *G, int n, double *Ginv, const char *what, DevBuf<double> *Linv = nullptr)
{
    if (n == 0) return;
    DevBuf<double> own;
    DevBuf<double> &work = Linv ? *Linv : own;
    work.alloc((size_t)n * n, &c->budget, "metric work");
    TR_CUDA(cudaMemsetAsync(c->flag.p, 0, sizeof(int), c->st));
    cholesky(c->prof, c->st, G, n, c->flag.p);
    int h = 0;
    TR_CUDA(cudaMemcpyAsync(&h, c->flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    TR_CUDA(cudaStreamSynchronize(c->st));
    if (h) throw Error(TR_ENOTPD, std::string(what) + " metric is not positive definite (column " +
                                      std::to_string(h - 1) + ")");
    chol_inverse(c->prof, c->st, G, n, Ginv, work.p);
    TR_CUDA(cudaStreamSynchronize(c->st));
}

}  // namespace

void prepare_aux_chunks(tr_ctx *c, int which, int npc)
{
    const std::vector<AuxDev> &all = which == 0 ? c->auxJ_h : c->auxK_h;
    const int n = which == 0 ? c->nJ : c->nK;
    std::vector<AuxDev> lists;
    std::vector<tr_ctx::AuxChunk> idx;
    for (int p0 = 0; p0 < n; p0 += npc) {
        const int np = std::min(npc, n - p0);
        tr_ctx::AuxChunk k;
        k.which = which;
        k.p0 = p0;
        k.np = np;
        k.off = (long long)lists.size();
        const bool grouped = which == 0 && p0 % 4 == 0 && np % 4 == 0;
        std::vector<AuxDev> sorted;
        k.cls[0] = 0;
        for (int cd = -1; cd <= 2; ++cd) {
            for (const AuxDev &a : all)
                if (a.comp == cd && a.out >= p0 && a.out < p0 + np) {
                    AuxDev b = a;
                    b.out -= p0;
                    sorted.push_back(b);
                }
            k.cls[cd + 2] = (int)sorted.size();
        }
        k.natoms = 0;
        if (grouped) {
            for (int i = k.cls[0]; i < k.cls[1]; ++i) sorted.push_back(sorted[i]);
            k.natoms = k.cls[1] - k.cls[0];
        }
        lists.insert(lists.end(), sorted.begin(), sorted.end());
        idx.push_back(k);
    }
    c->aux_cache_idx.clear();
    c->aux_cache.alloc(std::max<size_t>(lists.size(), 1), &c->budget, "auxiliary chunk lists");
    if (!lists.empty())
        TR_CUDA(cudaMemcpy(c->aux_cache.p, lists.data(), sizeof(AuxDev) * lists.size(), cudaMemcpyHostToDevice));
    c->aux_cache_idx = idx;
}


void refresh_molecule(tr_ctx *c)
{
    const int natm = (int)c->Z.size();
    c->aux_cache_idx.clear();  // the cached chunk lists belong to the previous molecule
    c->aux_cache.release();
    // auxiliary functions (Sec. 3.2): J = s, px, py, pz and K = s on every atom that
    // carries an exponent, hydrogen excluded unless aux_on_h
    c->auxJ_h.clear();
    c->auxK_h.clear();
    for (int a = 0; a < natm; ++a) {
        if (!(c->aux_exp[a] > 0.0)) continue;
        if (c->Z[a] == 1 && !c->opt.aux_on_h) continue;
        int j0 = (int)c->auxJ_h.size();
        for (int comp = -1; comp <= 2; ++comp) {
            AuxDev f;
            f.x = c->xyz[3 * a];
            f.y = c->xyz[3 * a + 1];
            f.z = c->xyz[3 * a + 2];
            f.e = c->aux_exp[a];
            f.comp = comp;
            f.out = j0 + comp + 1;
            c->auxJ_h.push_back(f);
            if (comp < 0) {
                f.out = (int)c->auxK_h.size();
                c->auxK_h.push_back(f);
            }
        }
    }
    c->nJ = (int)c->auxJ_h.size();
    c->nK = (int)c->auxK_h.size();
    c->pl = make_pairs(c->shells_h, c->pexp_h, c->pcoef_h, c->opt.screen);
    c->nkl = -1;  // the packed pair list of the AO Coulomb term follows the new pairs
    c->shells.alloc(c->shells_h.size(), &c->budget, "shells");
    c->pexp.alloc(c->pexp_h.size(), &c->budget, "primitives");
    c->pcoef.alloc(c->pcoef_h.size(), &c->budget, "primitives");
    c->pairs.alloc(std::max<size_t>(c->pl.pairs.size(), 1), &c->budget, "pairs");
    c->prange.alloc(std::max<size_t>(c->pl.range.size(), 1), &c->budget, "pairs");
    c->prim.alloc(std::max<size_t>(c->pl.prim.size(), 1), &c->budget, "primitive pairs");
    if (!c->pl.range.empty())
        TR_CUDA(cudaMemcpy(c->prange.p, c->pl.range.data(), sizeof(int2) * c->pl.range.size(), cudaMemcpyHostToDevice));
    if (!c->pl.prim.empty())
        TR_CUDA(cudaMemcpy(c->prim.p, c->pl.prim.data(), sizeof(double) * c->pl.prim.size(), cudaMemcpyHostToDevice));
    TR_CUDA(cudaMemcpy(c->shells.p, c->shells_h.data(), sizeof(ShellDev) * c->shells_h.size(), cudaMemcpyHostToDevice));
    TR_CUDA(cudaMemcpy(c->pexp.p, c->pexp_h.data(), sizeof(double) * c->pexp_h.size(), cudaMemcpyHostToDevice));
    TR_CUDA(cudaMemcpy(c->pcoef.p, c->pcoef_h.data(), sizeof(double) * c->pcoef_h.size(), cudaMemcpyHostToDevice));
    if (!c->pl.pairs.empty())
        TR_CUDA(cudaMemcpy(c->pairs.p, c->pl.pairs.data(), sizeof(int2) * c->pl.pairs.size(), cudaMemcpyHostToDevice));
    // row tiles (16 functions) of each column tile (64 functions) of (P|mn) that a
    // kept shell pair touches; both orders, the matrices being symmetric
    {
        const int nao = c->nao, ntk = cdiv(std::max(nao, 1), 16), ntn = cdiv(std::max(nao, 1), 64);
        std::vector<unsigned char> hit((size_t)ntn * ntk, 0);
        auto mark = [&](int r0, int nr, int c0, int nc) {
            for (int kt = r0 / 16; kt <= (r0 + nr - 1) / 16; ++kt)
                for (int nt = c0 / 64; nt <= (c0 + nc - 1) / 64; ++nt) hit[(size_t)nt * ntk + kt] = 1;
        };
        for (const int2 &ab : c->pl.pairs) {
            const ShellDev &A = c->shells_h[ab.x], &B = c->shells_h[ab.y];
            const int na = 2 * A.l + 1, nb = 2 * B.l + 1;
            mark(A.ao, na, B.ao, nb);
            mark(B.ao, nb, A.ao, na);
        }
        c->kt_list_h.assign((size_t)ntn * ntk, 0);
        c->kt_count_h.assign(ntn, 0);
        long long active = 0;
        for (int nt = 0; nt < ntn; ++nt) {
            int n = 0;
            for (int kt = 0; kt < ntk; ++kt)
                if (hit[(size_t)nt * ntk + kt]) c->kt_list_h[(size_t)nt * ntk + n++] = kt;
            c->kt_count_h[nt] = n;
            active += n;
        }
        c->kt_list.alloc(c->kt_list_h.size(), &c->budget, "integral block sparsity");
        c->kt_count.alloc(c->kt_count_h.size(), &c->budget, "integral block sparsity");
        TR_CUDA(cudaMemcpy(c->kt_list.p, c->kt_list_h.data(), sizeof(int) * c->kt_list_h.size(), cudaMemcpyHostToDevice));
        TR_CUDA(cudaMemcpy(c->kt_count.p, c->kt_count_h.data(), sizeof(int) * c->kt_count_h.size(),
                           cudaMemcpyHostToDevice));
        c->ktiles.list = c->kt_list.p;
        c->ktiles.count = c->kt_count.p;
        c->ktiles.ld = ntk;
        c->ktiles.active = active;
        // K blocks of 32 for the tensor-core transforms
        const int nkb = cdiv(std::max(nao, 1), 32);
        std::vector<unsigned char> hb((size_t)ntn * nkb, 0);
        for (int nt = 0; nt < ntn; ++nt)
            for (int kt = 0; kt < ntk; ++kt)
                if (hit[(size_t)nt * ntk + kt]) hb[(size_t)nt * nkb + kt / 2] = 1;
        c->kb_list_h.assign((size_t)ntn * nkb, 0);
        c->kb_count_h.assign(ntn, 0);
        for (int nt = 0; nt < ntn; ++nt) {
            int n = 0;
            for (int kb = 0; kb < nkb; ++kb)
                if (hb[(size_t)nt * nkb + kb]) c->kb_list_h[(size_t)nt * nkb + n++] = kb;
            c->kb_count_h[nt] = n;
        }
        c->kb_list.alloc(c->kb_list_h.size(), &c->budget, "integral block sparsity");
        c->kb_count.alloc(c->kb_count_h.size(), &c->budget, "integral block sparsity");
        TR_CUDA(cudaMemcpy(c->kb_list.p, c->kb_list_h.data(), sizeof(int) * c->kb_list_h.size(), cudaMemcpyHostToDevice));
        TR_CUDA(cudaMemcpy(c->kb_count.p, c->kb_count_h.data(), sizeof(int) * c->kb_count_h.size(),
                           cudaMemcpyHostToDevice));
        c->kb_mask.alloc(hb.size(), &c->budget, "integral block sparsity");
        TR_CUDA(cudaMemcpy(c->kb_mask.p, hb.data(), hb.size(), cudaMemcpyHostToDevice));
        c->kb_ld = nkb;
    }
}

void refresh_window(tr_ctx *c)
{
    // exchange window (Sec. 3.2): occupied e > -W, virtual e < W, contiguous for sorted eps
    const int nocc = c->nocc;
    c->o0 = 0;
    c->oK = nocc;
    c->vK = c->nvir;
    if (c->opt.window_ev > 0) {
        double w = c->opt.window_ev / HARTREE_EV;
        int o0 = 0;
        while (o0 < nocc && !(c->eps_h[o0] > -w)) ++o0;
        int vk = 0;
        while (vk < c->nvir && c->eps_h[nocc + vk] < w) ++vk;
        c->o0 = o0;
        c->oK = nocc - o0;
        c->vK = vk;
    }
}

void set_molecule(tr_ctx *c, int natm, const int *Z, const double *xyz, const double *aux_exp,
                  int nshell, const tr_shell *shells)
{
    TR_REQUIRE(natm > 0 && Z && xyz && aux_exp, TR_EINVAL, "set_molecule: empty molecule");
    TR_REQUIRE(nshell > 0 && shells, TR_EINVAL, "set_molecule: no AO shells");
    c->have_mol = false;
    c->built = false;
    c->Z.assign(Z, Z + natm);
    c->xyz.assign(xyz, xyz + 3 * natm);
    c->aux_exp.assign(aux_exp, aux_exp + natm);
    for (int i = 0; i < 3 * natm; ++i) TR_REQUIRE(std::isfinite(xyz[i]), TR_EINVAL, "set_molecule: non-finite coordinate");
    c->shells_h.clear();
    c->pexp_h.clear();
    c->pcoef_h.clear();
    int ao = 0;
    for (int s = 0; s < nshell; ++s) {
        const tr_shell &sh = shells[s];
        TR_REQUIRE(sh.l >= 0 && sh.l <= 2, TR_EINVAL, "set_molecule: shell l must be 0, 1 or 2");
        TR_REQUIRE(sh.nprim >= 1 && sh.nprim <= 16, TR_EINVAL, "set_molecule: nprim must be 1..16");
        TR_REQUIRE(sh.atom >= 0 && sh.atom < natm, TR_EINVAL, "set_molecule: shell atom out of range");
        TR_REQUIRE(sh.exp && sh.coef, TR_EINVAL, "set_molecule: null primitive arrays");
        ShellDev d;
        d.x = xyz[3 * sh.atom];
        d.y = xyz[3 * sh.atom + 1];
        d.z = xyz[3 * sh.atom + 2];
        d.l = sh.l;
        d.nprim = sh.nprim;
        d.pstart = (int)c->pexp_h.size();
        d.ao = ao;
        for (int k = 0; k < sh.nprim; ++k) {
            TR_REQUIRE(sh.exp[k] > 0.0 && std::isfinite(sh.exp[k]) && std::isfinite(sh.coef[k]),
                       TR_EINVAL, "set_molecule: invalid primitive");
            c->pexp_h.push_back(sh.exp[k]);
            c->pcoef_h.push_back(sh.coef[k]);
        }
        c->shells_h.push_back(d);
        ao += 2 * sh.l + 1;
    }
    c->nao = ao;
    refresh_molecule(c);
    if (!c->boys.p) {
        std::vector<double> tab;
        boys_table(tab);
        c->boys.alloc(tab.size(), &c->budget, "boys table");
        TR_CUDA(cudaMemcpy(c->boys.p, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    }
    if (!c->flag.p) c->flag.alloc(4, &c->budget, "flags");
    c->have_mol = true;
}

void set_orbitals(tr_ctx *c, int nao, int nmo, int nocc, const double *C, const double *eps, int on_device)
{
    TR_REQUIRE(c->have_mol, TR_EINVAL, "set_orbitals: call tr_set_molecule first");
    TR_REQUIRE(nao == c->nao, TR_EINVAL, "set_orbitals: nao does not match the AO basis");
    TR_REQUIRE(nmo > 0 && nmo <= nao && nocc > 0 && nocc < nmo, TR_EINVAL, "set_orbitals: bad nmo/nocc");
    TR_REQUIRE(C && eps, TR_EINVAL, "set_orbitals: null pointer");
    c->have_orb = false;
    c->built = false;
    c->eps_h.resize(nmo);
    if (on_device)
        TR_CUDA(cudaMemcpy(c->eps_h.data(), eps, sizeof(double) * nmo, cudaMemcpyDeviceToHost));
    else
        std::memcpy(c->eps_h.data(), eps, sizeof(double) * nmo);
    for (int i = 0; i < nmo; ++i) {
        TR_REQUIRE(std::isfinite(c->eps_h[i]), TR_EINVAL, "set_orbitals: non-finite orbital energy");
        if (i) TR_REQUIRE(c->eps_h[i] >= c->eps_h[i - 1], TR_EINVAL, "set_orbitals: eps must be ascending");
    }
    c->nmo = nmo;
    c->nocc = nocc;
    c->nvir = nmo - nocc;
    c->nov = (long long)nocc * c->nvir;
    c->C.alloc((size_t)nao * nmo, &c->budget, "MO coefficients");
    c->eps.alloc(nmo, &c->budget, "orbital energies");
    TR_CUDA(cudaMemcpyAsync(c->C.p, C, sizeof(double) * (size_t)nao * nmo,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
    TR_CUDA(cudaMemcpyAsync(c->eps.p, c->eps_h.data(), sizeof(double) * nmo, cudaMemcpyHostToDevice, c->st));
    TR_CUDA(cudaStreamSynchronize(c->st));
    refresh_window(c);
    c->have_orb = true;
}

void compute_int3c_chunk(tr_ctx *c, int which, int p0, int np, double *out)
{
    if (which == 0)
        compute_int3c(c, c->auxJ_h, p0, np, out, 1.0, 0.0, 0.0);
    else
        compute_int3c(c, c->auxK_h, p0, np, out, c->opt.k_alpha, c->opt.k_beta, c->opt.omega);
}

// FP64 MO transforms: (P|ia); (P|ij), (P|ab) on the window; T_ij = G_K^-1 (P|ij);
// with Iia (full TDDFT) also (P|ia) on the window with the K operator
static void transforms_fp64(tr_ctx *c, DevBuf<double> &Iij, DevBuf<double> *Iia)
{
    const int nao = c->nao, nocc = c->nocc, nvir = c->nvir, nmo = c->nmo, nJ = c->nJ, nK = c->nK;
    const long long nov = c->nov;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nJt = c->opt.j_ao ? 0 : nJ;  // the AO form of J (j_ao) stores no (P|ia)
    c->Y.alloc((size_t)nJt * nov, &c->budget, "(P|ia)");
    const int hrows = std::max(nocc, std::max(c->oK, c->vK));
    size_t per = (size_t)nao * nao + (size_t)hrows * nao;
    int npc = (int)std::max<size_t>(1, c->opt.aux_chunk_bytes / (per * sizeof(double)));
    npc = std::max(1, std::min(npc, std::max(nJt, nK)));
    DevBuf<double> I, H;
    I.alloc((size_t)npc * nao * nao, &c->budget, "AO integral chunk");
    H.alloc((size_t)npc * hrows * nao, &c->budget, "half-transform chunk");
    const int npcJ = j_chunk(npc);
    for (int p0 = 0; p0 < nJt; p0 += npcJ) {
        int np = std::min(npcJ, nJt - p0);
        compute_int3c_chunk(c, 0, p0, np, I.p);
        Batch b1;
        b1.n1 = np;
        b1.sB1 = (long long)nao * nao;
        b1.sC1 = (long long)nocc * nao;
        // the integrals are block-sparse in mu (screened pairs): only the listed row tiles
        dgemm_ktiles(pf, st, "xform_J1", true, nocc, nao, nao, 1.0, c->C.p, nmo, I.p, nao, 0.0, H.p, nao, b1,
                     c->ktiles);
        Batch b2;
        b2.n1 = np;
        b2.sA1 = (long long)nocc * nao;
        b2.sC1 = nov;
        dgemm(pf, st, "xform_J2", false, false, nocc, nvir, nao, 1.0, H.p, nao, c->C.p + nocc, nmo, 0.0,
              c->Y.p + (long long)p0 * nov, nvir, b2, nullptr, 0);
    }
    if (!c->k_active) return;
    const int oK = c->oK, vK = c->vK, o0 = c->o0;
    c->Tab.alloc((size_t)nK * vK * vK, &c->budget, "T_ab");
    for (int p0 = 0; p0 < nK; p0 += npc) {
        int np = std::min(npc, nK - p0);
        compute_int3c_chunk(c, 1, p0, np, I.p);
        Batch h;
        h.n1 = np;
        h.sB1 = (long long)nao * nao;
        h.sC1 = (long long)oK * nao;
        dgemm_ktiles(pf, st, "xform_K1", true, oK, nao, nao, 1.0, c->C.p + o0, nmo, I.p, nao, 0.0, H.p, nao, h,
                     c->ktiles);
        Batch g;
        g.n1 = np;
        g.sA1 = (long long)oK * nao;
        g.sC1 = (long long)oK * oK;
        dgemm(pf, st, "xform_K2", false, false, oK, oK, nao, 1.0, H.p, nao, c->C.p + o0, nmo, 0.0,
              Iij.p + (long long)p0 * oK * oK, oK, g, nullptr, 0);
        if (Iia) {
            // (P|ia) = (C_occK^T (P|mn)) C_virK, the half transform shared with (P|ij)
            Batch x = g;
            x.sC1 = (long long)oK * vK;
            dgemm(pf, st, "xform_Kx", false, false, oK, vK, nao, 1.0, H.p, nao, c->C.p + nocc, nmo, 0.0,
                  Iia->p + (long long)p0 * oK * vK, vK, x, nullptr, 0);
        }
        h.sC1 = (long long)vK * nao;
        dgemm_ktiles(pf, st, "xform_K1", true, vK, nao, nao, 1.0, c->C.p + nocc, nmo, I.p, nao, 0.0, H.p, nao, h,
                     c->ktiles);
        g.sA1 = (long long)vK * nao;
        g.sC1 = (long long)vK * vK;
        dgemm(pf, st, "xform_K2", false, false, vK, vK, nao, 1.0, H.p, nao, c->C.p + nocc, nmo, 0.0,
              c->Tab.p + (long long)p0 * vK * vK, vK, g, nullptr, 0);
    }
}

// Slices of the Ozaki-scheme transforms for this context: 0 when the FP64
// transforms run on the FP64 pipe
int dav_slices(const tr_ctx *c) { return c->opt.precision == TR_MIXED ? OZ_SLICES_DAV_MIXED : OZ_SLICES_FP64; }

int xform_slices(const tr_ctx *c)
{
    const int s = c->opt.xform_slices;
    if (s < 0) return 0;
    if (s == 0)
        return c->opt.precision == TR_MIXED ? OZ_DEFAULT_SLICES_MIXED
             : c->opt.precision == TR_FP64_TC ? OZ_SLICES_FP64
                                              : 0;
    return s;
}

// The same MO transforms on the bf16 tensor cores (Ozaki scheme with S slices):
// the MO coefficients are sliced once (rows = orbitals, K = AO index), each AO
// integral chunk and each half-transformed chunk before its product.
static void transforms_oz(tr_ctx *c, DevBuf<double> &Iij, DevBuf<double> *Iia, int S)
{
    const int nao = c->nao, nocc = c->nocc, nvir = c->nvir, nmo = c->nmo, nJ = c->nJ, nK = c->nK;
    const long long nov = c->nov;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    int *err = c->flag.p + 2;
    TR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    DevBuf<double> cbuf;
    cbuf.alloc(cdiv(oz_bytes(nmo, nao, S), 8), &c->budget, "sliced MO coefficients");
    OzMat Cs;
    oz_bind(Cs, cbuf.p, nmo, nao, S);
    oz_split(pf, st, "oz_split_C", c->C.p, 1, nmo, Cs);
    const int nJt = c->opt.j_ao ? 0 : nJ;  // the AO form of J (j_ao) stores no (P|ia)
    c->Y.alloc((size_t)nJt * nov, &c->budget, "(P|ia)");
    const int hrows = std::max(nocc, std::max(c->oK, c->vK));
    const size_t per = sizeof(double) * ((size_t)nao * nao + (size_t)hrows * nao) + oz_bytes(nao, nao, S) +
                       oz_bytes(hrows, nao, S);
    int npc = (int)std::max<size_t>(1, c->opt.aux_chunk_bytes / per);
    npc = std::max(1, std::min(npc, std::max(nJt, nK)));
    DevBuf<double> I, H, Ib, Hb;
    I.alloc((size_t)npc * nao * nao, &c->budget, "AO integral chunk");
    H.alloc((size_t)npc * hrows * nao, &c->budget, "half-transform chunk");
    Ib.alloc(cdiv(oz_bytes((long long)npc * nao, nao, S), 8), &c->budget, "sliced integral chunk");
    Hb.alloc(cdiv(oz_bytes((long long)npc * hrows, nao, S), 8), &c->budget, "sliced half-transform chunk");
    OzMat Is, Hs;
    // H[p][r][nu] = sum_mu C[mu][r0 + r] (P|mu nu) for rows r < nr, then
    // out[p][r][s] = sum_nu H[p][r][nu] C[nu][s0 + s] for s < ns
    auto pair_transform = [&](int np, int r0, int nr, int s0, int ns, double *out, long long ldo, const char *n1,
                              const char *n2) {
        // the integrals are block-sparse in mu: each 64-column tile contracts
        // only the K blocks its kept shell pairs touch
        oz_gemm(pf, st, n1, Cs, r0, 0, Is, 0, nao, nr, nao, np, H.p, (long long)nr * nao, nao, 1, 1.0, err,
                c->kb_list.p, c->kb_count.p, c->kb_ld);
        oz_bind(Hs, Hb.p, (long long)np * nr, nao, S);
        oz_split(pf, st, "oz_split_H", H.p, nao, 1, Hs);
        oz_gemm(pf, st, n2, Hs, 0, nr, Cs, s0, 0, nr, ns, np, out, (long long)nr * ldo, ldo, 1, 1.0, err);
    };
    const int npcJ = j_chunk(npc);
    for (int p0 = 0; p0 < nJt; p0 += npcJ) {
        const int np = std::min(npcJ, nJt - p0);
        compute_int3c_chunk(c, 0, p0, np, I.p);
        oz_bind(Is, Ib.p, (long long)np * nao, nao, S);
        oz_split(pf, st, "oz_split_I", I.p, nao, 1, Is, c->kb_mask.p, nao, c->kb_ld);
        pair_transform(np, 0, nocc, nocc, nvir, c->Y.p + (long long)p0 * nov, nvir, "xform_J1_oz", "xform_J2_oz");
    }
    if (c->k_active) {
        const int oK = c->oK, vK = c->vK, o0 = c->o0;
        c->Tab.alloc((size_t)nK * vK * vK, &c->budget, "T_ab");
        for (int p0 = 0; p0 < nK; p0 += npc) {
            const int np = std::min(npc, nK - p0);
            compute_int3c_chunk(c, 1, p0, np, I.p);
            oz_bind(Is, Ib.p, (long long)np * nao, nao, S);
            oz_split(pf, st, "oz_split_I", I.p, nao, 1, Is, c->kb_mask.p, nao, c->kb_ld);
            pair_transform(np, o0, oK, o0, oK, Iij.p + (long long)p0 * oK * oK, oK, "xform_K1_oz", "xform_K2_oz");
            pair_transform(np, nocc, vK, nocc, vK, c->Tab.p + (long long)p0 * vK * vK, vK, "xform_K1_oz",
                           "xform_K2_oz");
            if (Iia)
                pair_transform(np, o0, oK, nocc, vK, Iia->p + (long long)p0 * oK * vK, vK, "xform_K1_oz",
                               "xform_Kx_oz");
        }
    }
    int h = 0;
    TR_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    TR_REQUIRE(h == 0, TR_ETIMEOUT, "build: a tensor-core transform pipeline wait ran out (code " + std::to_string(h) + ")");
}

// T^P_ij = sum_Q (P|Q)^-1 (Q|ij), stored [i][P][j], as an Ozaki product on the
// tensor cores with the transforms' slice count: A = (P|Q)^-1 (rows P, K = Q),
// B = (Q|ij) read as rows (i, j) with K = Q, one batch entry per i
static void apply_metric_oz(tr_ctx *c, const double *Ginv, const double *Iij, int nK, int oK, double *T2, int S)
{
    Prof &pf = c->prof;
    cudaStream_t st = c->st;
    int *err = c->flag.p + 2;
    const long long nij = (long long)oK * oK;
    DevBuf<double> ab, bb;
    ab.alloc(cdiv(oz_bytes(nK, nK, S), 8), &c->budget, "sliced K metric inverse");
    bb.alloc(cdiv(oz_bytes(nij, nK, S), 8), &c->budget, "sliced (ij|P)");
    OzMat As, Bs;
    oz_bind(As, ab.p, nK, nK, S);
    oz_split(pf, st, "oz_split_GK", Ginv, nK, 1, As);
    oz_bind(Bs, bb.p, nij, nK, S);
    oz_split(pf, st, "oz_split_Iij", Iij, 1, nij, Bs);
    TR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    oz_gemm(pf, st, "apply_K_metric_oz", As, 0, 0, Bs, 0, oK, nK, oK, oK, T2, (long long)nK * oK, oK, 1, 1.0, err);
    int h = 0;
    TR_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));  // the sliced operands are freed on return
    TR_REQUIRE(h == 0, TR_ETIMEOUT, "build: a tensor-core metric product wait ran out (code " + std::to_string(h) + ")");
}

void build(tr_ctx *c)
{
    TR_REQUIRE(c->have_mol && c->have_orb, TR_EINVAL, "build: molecule and orbitals required");
    c->built = false;
    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ, nK = c->nK;
    const long long nov = c->nov;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const bool mixed = c->opt.precision == TR_MIXED;
    c->ws_split.reserve((size_t)32 << 20, &c->budget, "split-K workspace");
    c->k_active = nK > 0 && c->oK > 0 && c->vK > 0 && c->opt.cx != 0.0;
    c->Y.release();
    c->Y32.release();
    c->Tab.release();
    c->T2.release();
    c->GinvK.release();
    c->Tia.release();
    const bool tddft = c->opt.tddft != 0;

    // metrics and their inverses (Sec. 2, Eq. RI; K metric with the K operator, Sec. 3.2)
    c->GinvJ.alloc((size_t)nJ * nJ, &c->budget, "J metric");
    if (nJ) {
        DevBuf<double> G;
        G.alloc((size_t)nJ * nJ, &c->budget, "J metric");
        metric(c, c->auxJ_h, 1.0, 0.0, 0.0, G.p);
        metric_inverse(c, G.p, nJ, c->GinvJ.p, "Coulomb");
    }
    DevBuf<double> LinvK;  // full TDDFT: inverse Cholesky factor of the K metric
    if (c->k_active) {
        DevBuf<double> G;
        G.alloc((size_t)nK * nK, &c->budget, "K metric");
        c->GinvK.alloc((size_t)nK * nK, &c->budget, "K metric");
        metric(c, c->auxK_h, c->opt.k_alpha, c->opt.k_beta, c->opt.omega, G.p);
        metric_inverse(c, G.p, nK, c->GinvK.p, "exchange", tddft ? &LinvK : nullptr);
    }
    // MO transforms
    {
        DevBuf<double> Iij, Iia;
        const int oK = c->oK, vK = c->vK;
        if (c->k_active) Iij.alloc((size_t)nK * oK * oK, &c->budget, "(ij|P)");
        const bool kx = tddft && c->k_active;
        if (kx) Iia.alloc((size_t)nK * oK * vK, &c->budget, "(ia|P) on the window");
        const int S = xform_slices(c);
        if (S > 0) transforms_oz(c, Iij, kx ? &Iia : nullptr, S);
        else transforms_fp64(c, Iij, kx ? &Iia : nullptr);
        if (kx) {
            // t^P_ia = sum_Q (L^-1)_PQ (Q|ia): sum_P t^P_ib t^P_ja = (ib|ja) with (P|Q)^-1 = L^-T L^-1
            c->Tia.alloc((size_t)nK * oK * vK, &c->budget, "T_ia");
            dgemm(pf, st, "apply_K_factor", false, false, nK, (int)((long long)oK * vK), nK, 1.0, LinvK.p, nK, Iia.p,
                  (long long)oK * vK, 0.0, c->Tia.p, (long long)oK * vK, Batch(), nullptr, 0);
        }
        if (c->k_active) {
            // T_ij^P = sum_Q (ij|Q) (Q|P)^-1, stored [i][P][j]
            c->T2.alloc((size_t)oK * nK * oK, &c->budget, "T_ij");
            Batch t;
            t.n1 = oK;
            t.sB1 = oK;
            t.sC1 = (long long)nK * oK;
            // the reduced-precision form keeps T_ij in FP32: its metric product
            // runs on the tensor cores; the FP64 forms keep it on the FP64 pipe
            if (S > 0 && mixed)
                apply_metric_oz(c, c->GinvK.p, Iij.p, nK, oK, c->T2.p, S);
            else
                dgemm(pf, st, "apply_K_metric", false, false, nK, oK, nK, 1.0, c->GinvK.p, nK, Iij.p,
                      (long long)oK * oK, 0.0, c->T2.p, oK, t, nullptr, 0);
        }
        TR_CUDA(cudaStreamSynchronize(st));
    }
    // the AO form of J generates integrals in every product: its chunk lists once
    c->aux_cache_idx.clear();
    c->aux_cache.release();
    if (c->opt.j_ao && nJ > 0) prepare_aux_chunks(c, 0, jao_chunk_size(c));
    c->D.alloc(std::max<long long>(nov, 1), &c->budget, "orbital differences");
    TR_LAUNCH(pf, st, "orbital_diff", 0, 0, orbital_diff<<<grid_for(nov), 256, 0, st>>>(c->eps.p, nocc, nvir, c->D.p));
    TR_CUDA(cudaStreamSynchronize(st));
    if (mixed) build_mixed(c);
    if (c->opt.precision == TR_FP64_TC) build_tc(c);
    c->built = true;
}

void int3c_ao(tr_ctx *c, int which, int p0, int np, double *out)
{
    TR_REQUIRE(c->have_mol, TR_EINVAL, "int3c: call tr_set_molecule first");
    const std::vector<AuxDev> &all = which == 0 ? c->auxJ_h : c->auxK_h;
    int n = which == 0 ? c->nJ : c->nK;
    TR_REQUIRE(which == 0 || which == 1, TR_EINVAL, "int3c: which must be 0 or 1");
    TR_REQUIRE(p0 >= 0 && np >= 0 && p0 + np <= n, TR_EINVAL, "int3c: aux range out of bounds");
    if (np == 0) return;
    if (which == 0)
        compute_int3c(c, all, p0, np, out, 1.0, 0.0, 0.0);
    else
        compute_int3c(c, all, p0, np, out, c->opt.k_alpha, c->opt.k_beta, c->opt.omega);
}

void int2c_aux(tr_ctx *c, int which, double *out)
{
    TR_REQUIRE(c->have_mol, TR_EINVAL, "int2c: call tr_set_molecule first");
    TR_REQUIRE(which == 0 || which == 1, TR_EINVAL, "int2c: which must be 0 or 1");
    if (which == 0)
        metric(c, c->auxJ_h, 1.0, 0.0, 0.0, out);
    else
        metric(c, c->auxK_h, c->opt.k_alpha, c->opt.k_beta, c->opt.omega, out);
}

void get_tensor(tr_ctx *c, int which, double *out, int on_device)
{
    TR_REQUIRE(c->built, TR_EINVAL, "get_tensor: call tr_build first");
    TR_REQUIRE(which != 0 || !c->opt.j_ao, TR_EINVAL, "get_tensor: (P|ia) is not built with j_ao = 1");
    const double *src = nullptr;
    size_t n = 0;
    DevBuf<double> tmp;
    if (c->opt.precision == TR_MIXED && (which == 0 || which == 2)) {
        get_tensor_mixed(c, which, out, on_device);
        return;
    }
    switch (which) {
        case 0: src = c->Y.p; n = (size_t)c->nJ * c->nov; break;
        case 1:
            n = c->k_active ? (size_t)c->nK * c->oK * c->oK : 0;
            if (n) {
                tmp.alloc(n, &c->budget, "tensor copy");
                TR_LAUNCH(c->prof, c->st, "unpermute", 0, 0,
                          unpermute_T2<<<grid_for(n), 256, 0, c->st>>>(c->T2.p, c->nK, c->oK, tmp.p));
                src = tmp.p;
            }
            break;
        case 2: src = c->Tab.p; n = c->k_active ? (size_t)c->nK * c->vK * c->vK : 0; break;
        case 3: src = c->D.p; n = (size_t)c->nov; break;
        case 4:
            TR_REQUIRE(c->opt.tddft, TR_EINVAL, "get_tensor: T_ia is built with tddft = 1 only");
            src = c->Tia.p;
            n = c->k_active ? (size_t)c->nK * c->oK * c->vK : 0;
            break;
        default: throw Error(TR_EINVAL, "get_tensor: unknown tensor");
    }
    if (n)
        TR_CUDA(cudaMemcpyAsync(out, src, sizeof(double) * n,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
    TR_CUDA(cudaStreamSynchronize(c->st));
}

static int matvec_pchunk(tr_ctx *c, int mb)
{
    if (!c->k_active) return 0;
    size_t perP = (size_t)mb * c->oK * c->vK;
    size_t cap = std::max<size_t>(perP, c->opt.matvec_ws_bytes / sizeof(double));
    int npk = (int)std::min<size_t>(c->nK, std::max<size_t>(1, cap / perP));
    return std::min(npk, 65535 / mb);
}

// Estimated peak device bytes of build + solve for the current sizes and options.
size_t footprint(tr_ctx *c)
{
    const double d = 8.0, f = 4.0;
    const double nao = c->nao, nmo = c->nmo, nocc = c->nocc, nov = (double)c->nov;
    const double nJ = c->nJ, oK = c->oK, vK = c->vK;
    const double nJt = c->opt.j_ao ? 0.0 : nJ;  // stored (P|ia) rows (none with the AO form of J)
    const double nK = (c->nK > 0 && c->oK > 0 && c->vK > 0 && c->opt.cx != 0.0) ? c->nK : 0;
    const bool mixed = c->opt.precision == TR_MIXED;
    const double base = d * (nao * nmo + nmo + nov) + d * (nJ * nJ + nK * nK) + 128.0 * (1 << 20) +
                        (double)c->shells_h.size() * 64 + (double)c->pl.pairs.size() * 16 + (double)c->pl.prim.size() * 8;
    // build: integral and half-transform chunks, FP64 tensors
    const double hrows = std::max(nocc, std::max(oK, vK));
    const int S = xform_slices(c);
    const double per = d * (nao * nao + hrows * nao) +
                       (S > 0 ? (double)oz_bytes(c->nao, c->nao, S) + (double)oz_bytes((long long)hrows, c->nao, S) : 0.0);
    const double npc = std::max(1.0, std::min(std::floor((double)c->opt.aux_chunk_bytes / per), std::max(nJt, nK)));
    const double cs = S > 0 ? (double)oz_bytes(c->nmo, c->nao, S) : 0.0;
    const double t64 = d * (nJt * nov + nK * vK * vK + 2.0 * nK * oK * oK);
    const double oKp = std::ceil(std::max(oK, 1.0) / 32) * 32, vKp = std::ceil(std::max(vK, 1.0) / 32) * 32;
    const double t32 = mixed ? f * (nJt * nov + 2.0 * nK * vK * vKp + 2.0 * oK * nK * oKp) : 0.0;
    double tcb = 0.0;
    if (c->opt.precision == TR_FP64_TC) {
        const int Sf = OZ_SLICES_FP64;
        tcb = (nJt > 0 ? (double)oz_bytes((long long)nJt, (int)nov, Sf) + (double)oz_bytes((long long)nov, (int)nJt, Sf) : 0.0) +
              (nK > 0 ? (double)oz_bytes((long long)(nK * vK), (int)vK, Sf) + (double)oz_bytes((long long)oK, (int)(nK * oK), Sf) : 0.0);
    }
    // full TDDFT: T_ia on the window (and its unfactored copy during the build)
    const bool rpa = c->opt.tddft != 0;
    const double tx = rpa ? d * nK * oK * vK : 0.0;
    // the split-K workspace reserved at the start of the build is held throughout
    const double wsplit = d * 32.0 * (1 << 20);
    const double build_peak = wsplit + std::max(npc * per + cs + t64 + t32 + 2.0 * tx, t64 + tcb + tx);
    // solve: tensors kept, Davidson storage and product workspaces
    const double kept = (mixed ? t32 + d * oK * nK * oK : t64 - d * nK * oK * oK) + tx;
    const int n = (int)std::min<double>(c->opt.nstates, nov);
    const int b0 = (int)std::min<double>(std::max(c->opt.block > 0 ? c->opt.block : 2 * n, n), nov);
    int maxsp = c->opt.max_space > 0 ? c->opt.max_space : 20 * n;
    maxsp = (int)std::min<double>(std::max(maxsp, b0 + (rpa ? 2 : 1) * n), std::max(nov, (double)b0));
    const double pmax = std::max(b0, (rpa ? 2 : 1) * n);
    const double mb = std::min<double>(pmax, c->mblk);
    // V and W (and the A - B products) by rows; new vectors, products and scratch; Ritz vectors and residuals
    const double dav = d * nov * ((rpa ? 3.0 : 2.0) * maxsp + (rpa ? 5.0 : 4.0) * pmax + (rpa ? 4.0 : 2.0) * n) +
                       d * ((rpa ? 10.0 : 5.0) * maxsp * maxsp + 2.0 * maxsp * pmax + 6.0 * n * maxsp + 5.0 * maxsp + 16.0 + n);
    const double mw = rpa ? std::max(oK, vK) : vK;
    const double mws = nK > 0 ? std::min<double>((double)c->opt.matvec_ws_bytes, d * mb * nK * oK * vK) * (mw / std::max(vK, 1.0)) +
                                    (mixed ? 2.0 * f * mb * oK * vKp + f * mb * nov : d * mb * oK * vK)
                              : 0.0;
    const double ws = d * 32.0 * (1 << 20) + 2.0 * d * std::max(nJ, 1.0) * mb + mws;
    double tcx = 0.0;
    if (c->opt.precision == TR_FP64_TC) {
        // slices kept for the products, and the per-block sliced operands
        const int Sf = OZ_SLICES_FP64;
        const double sl = (nJt > 0 ? (double)oz_bytes((long long)nJt, (int)nov, Sf) + (double)oz_bytes((long long)nov, (int)nJt, Sf) : 0.0) +
                          (nK > 0 ? (double)oz_bytes((long long)(nK * vK), (int)vK, Sf) + (double)oz_bytes((long long)oK, (int)(nK * oK), Sf) : 0.0);
        const double mbl = std::min<double>(pmax, c->mblk);
        const double npk = nK > 0 ? std::min<double>(nK, std::max(8.0, (double)c->opt.matvec_ws_bytes / (mbl * vK * oK * 24.0)) + 8.0) : 0.0;
        tcx = sl + (double)oz_bytes((long long)mbl, (int)nov, Sf) + 16.0 * (2 << 20) +
              (nK > 0 ? d * mbl * oK * vK + 16.0 * mbl * oK * (vK + 32) + 24.0 * mbl * vK * (npk * oK + 32) : 0.0) +
              (nJt > 0 ? 16.0 * mbl * (nJt + 32) : 0.0);
    }
    // sliced V, W and new directions of the Davidson subspace products
    const double dtc = (c->opt.precision == TR_MIXED || c->opt.precision == TR_FP64_TC)
                           ? 2.0 * (double)oz_bytes(maxsp, (int)nov, dav_slices(c)) +
                                 (double)oz_bytes((long long)pmax, (int)nov, dav_slices(c)) +
                                 2.0 * (double)oz_bytes((long long)nov, maxsp, dav_slices(c)) +
                                 2.0 * (double)oz_bytes((long long)std::max<double>(n, pmax), maxsp, dav_slices(c))
                           : 0.0;
    const double jao = c->opt.j_ao ? (double)jao_bytes(c, (int)mb) : 0.0;
    // full TDDFT on the tensor cores: T_ia sliced by rows (P, i) and by rows a
    if (rpa && c->opt.precision == TR_FP64_TC && nK > 0)
        tcx += (double)oz_bytes((long long)(nK * oK), (int)vK, OZ_SLICES_FP64) +
               (double)oz_bytes((long long)vK, (int)(nK * oK), OZ_SLICES_FP64);
    const double solve_peak = kept + dav + ws + tcx + dtc + jao;
    return (size_t)(1.1 * (base + std::max(build_peak, solve_peak + (mixed ? 0.0 : 0.0))));
}

void reserve_matvec(tr_ctx *c, int m)
{
    const int mb = std::max(1, std::min(m, c->mblk));
    c->ws_split.reserve((size_t)32 << 20, &c->budget, "split-K workspace");
    if (c->opt.j_ao) reserve_jao(c, mb);
    c->ws_Z.reserve((size_t)std::max(c->nJ, 1) * mb, &c->budget, "J workspace");
    c->ws_Z2.reserve((size_t)std::max(c->nJ, 1) * mb, &c->budget, "J workspace");
    if (c->opt.precision == TR_MIXED) {
        reserve_mixed(c, mb);
        return;
    }
    if (c->opt.precision == TR_FP64_TC) {
        reserve_tc(c, mb);
        return;
    }
    if (c->k_active) {
        c->ws_Xw.reserve((size_t)mb * c->oK * c->vK, &c->budget, "K workspace");
        // full TDDFT: the (ib|ja) intermediate E [m][i][P][j] of a chunk takes oK in place of vK
        const size_t w = c->opt.tddft ? (size_t)std::max(c->oK, c->vK) : (size_t)c->vK;
        c->ws_M.reserve((size_t)matvec_pchunk(c, mb) * mb * c->oK * w, &c->budget, "K workspace");
    }
}

// Coulomb term from the stored (P|ia), FP64: Z = (Q|jb) X; Zt = (P|Q)^-1 Z;
// out = 2 (P|ia) Zt + beta out (Sec. 3.1 order, in the MO basis)
static void j_stored_fp64(tr_ctx *c, int mm, const double *x, double *out, double beta)
{
    Prof &pf = c->prof;
    cudaStream_t st = c->st;
    const int nJ = c->nJ;
    const long long nov = c->nov;
    dgemm(pf, st, "J_contract", false, true, nJ, mm, (int)nov, 1.0, c->Y.p, nov, x, nov, 0.0, c->ws_Z.p, mm, Batch(),
          c->ws_split.p, c->ws_split.n);
    dgemm(pf, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, c->ws_Z.p, mm, 0.0, c->ws_Z2.p, mm,
          Batch(), nullptr, 0);
    dgemm(pf, st, "J_expand", true, false, mm, (int)nov, nJ, 2.0, c->ws_Z2.p, mm, c->Y.p, nov, beta, out, nov,
          Batch(), nullptr, 0);
}

void matvec(tr_ctx *c, int m, const double *X, double *AX)
{
    TR_REQUIRE(c->built, TR_EINVAL, "matvec: call tr_build first");
    if (m <= 0) return;
    if (c->opt.precision == TR_MIXED) {
        matvec_mixed(c, m, X, AX);
        return;
    }
    if (c->opt.precision == TR_FP64_TC) {
        matvec_tc(c, m, X, AX);
        return;
    }
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ, nK = c->nK;
    const long long nov = c->nov;
    const int mb = std::min(m, c->mblk);
    reserve_matvec(c, mb);
    const int oK = c->oK, vK = c->vK, o0 = c->o0;
    const int npk = matvec_pchunk(c, mb);
    for (int m0 = 0; m0 < m; m0 += mb) {
        const int mm = std::min(mb, m - m0);
        const double *x = X + (long long)m0 * nov;
        double *ax = AX + (long long)m0 * nov;
        // diagonal (e_a - e_i) X
        TR_LAUNCH(pf, st, "diag", 0, 8.0 * nov * (2.0 * mm + 1.0),
                  diag_kernel<<<grid_for(nov), 256, 0, st>>>(c->D.p, x, ax, nov, mm));
        if (nJ && c->opt.j_ao) {
            j_ao_block(c, mm, x, ax);
        } else if (nJ) {
            j_stored_fp64(c, mm, x, ax, 1.0);  // AX += 2 J
        }
        if (c->k_active) {
            long long tot = (long long)mm * oK * vK;
            TR_LAUNCH(pf, st, "gather_window", 0, 16.0 * tot,
                      gather_window<<<grid_for(tot), 256, 0, st>>>(x, c->ws_Xw.p, mm, nocc, nvir, o0, oK, vK));
            for (int P0 = 0; P0 < nK; P0 += npk) {
                const int np = std::min(npk, nK - P0);
                // M^P_mja = sum_b X_mjb T_ab^P
                Batch b1;
                b1.n1 = mm;
                b1.n2 = np;
                b1.sA1 = (long long)oK * vK;
                b1.sC1 = (long long)np * oK * vK;
                b1.sB2 = (long long)vK * vK;
                b1.sC2 = (long long)oK * vK;
                // algorithmic bytes: M written once, X window and T_ab^P read once
                const double kb1 = 8.0 * ((double)mm * np * oK * vK + (double)mm * oK * vK + (double)np * vK * vK);
                dgemm(pf, st, "K_stage1", false, false, oK, vK, vK, 1.0, c->ws_Xw.p, vK,
                      c->Tab.p + (long long)P0 * vK * vK, vK, 0.0, c->ws_M.p, vK, b1, nullptr, 0, kb1);
                // AX_mia -= cx sum_(P,j) T_ij^P M^P_mja  (window rows/cols)
                Batch b2;
                b2.n1 = mm;
                b2.sB1 = (long long)np * oK * vK;
                b2.sC1 = nov;
                // algorithmic bytes: M and the T_ij chunk read once, the AX window read and written
                const double kb2 = 8.0 * ((double)mm * np * oK * vK + (double)oK * np * oK + 2.0 * mm * oK * vK);
                dgemm(pf, st, "K_stage2", false, false, oK, vK, np * oK, -c->opt.cx,
                      c->T2.p + (long long)P0 * oK, (long long)nK * oK, c->ws_M.p, vK, 1.0,
                      ax + (long long)o0 * nvir, nvir, b2, c->ws_split.p, c->ws_split.n, kb2);
            }
        }
    }
}


// ---------------------------------------------------------------- full TDDFT-risp

namespace {

// P = A X + B X, M = A X - B X in place (P holds A X, M holds B X on entry)
__global__ void pm_combine(double *__restrict__ P, double *__restrict__ M, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const double a = P[t], b = M[t];
        P[t] = a + b;
        M[t] = a - b;
    }
}

}  // namespace

// B X = 2 J X - c_x K' X for m device vectors (Sec. 2, Eq. hessian), with
//   K'_mia = sum_jb (ib|ja) X_mjb = sum_P sum_j E^P_mij t^P_ja,  E^P_mij = sum_b t^P_ib X_mjb,
// t^P = L_K^-1 (P|ia) on the window (Sec. 3.2: the T_ia^P' tensor of full TDDFT);
// i, j, a, b inside the exchange window and K' zero outside it.  FP64.
void matvec_b(tr_ctx *c, int m, const double *X, double *BX)
{
    TR_REQUIRE(c->built && c->opt.tddft, TR_EINVAL, "matvec_b: needs a context built with tddft = 1");
    if (m <= 0) return;
    if (c->opt.precision == TR_FP64_TC) {
        matvec_b_tc(c, m, X, BX);
        return;
    }
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ, nK = c->nK;
    const long long nov = c->nov;
    const int mb = std::min(m, c->mblk);
    reserve_matvec(c, mb);
    const int oK = c->oK, vK = c->vK, o0 = c->o0;
    const int npk = matvec_pchunk(c, mb);
    for (int m0 = 0; m0 < m; m0 += mb) {
        const int mm = std::min(mb, m - m0);
        const double *x = X + (long long)m0 * nov;
        double *bx = BX + (long long)m0 * nov;
        if (nJ && !c->opt.j_ao) {
            j_stored_fp64(c, mm, x, bx, 0.0);  // BX = 2 J, as in A X
        } else {
            TR_CUDA(cudaMemsetAsync(bx, 0, sizeof(double) * (size_t)mm * nov, st));
            if (nJ) j_ao_block(c, mm, x, bx);
        }
        if (!c->k_active) continue;
        long long tot = (long long)mm * oK * vK;
        TR_LAUNCH(pf, st, "gather_window", 0, 16.0 * tot,
                  gather_window<<<grid_for(tot), 256, 0, st>>>(x, c->ws_Xw.p, mm, nocc, nvir, o0, oK, vK));
        for (int P0 = 0; P0 < nK; P0 += npk) {
            const int np = std::min(npk, nK - P0);
            const double *tP = c->Tia.p + (long long)P0 * oK * vK;
            // E[m][i][p][j] = sum_b t^(P0+p)_ib X_mjb
            Batch e;
            e.n1 = mm;
            e.n2 = np;
            e.sB1 = (long long)oK * vK;
            e.sC1 = (long long)oK * np * oK;
            e.sA2 = (long long)oK * vK;
            e.sC2 = oK;
            const double eb = 8.0 * ((double)np * oK * vK + (double)mm * oK * vK + (double)mm * np * oK * oK);
            dgemm(pf, st, "Kx_stage1", false, true, oK, oK, vK, 1.0, tP, vK, c->ws_Xw.p, vK, 0.0, c->ws_M.p,
                  (long long)np * oK, e, nullptr, 0, eb);
            // BX_mia -= c_x sum_(p,j) E[m][i][(p,j)] t^(P0+p)_ja  (window rows/cols)
            Batch f;
            f.n1 = mm;
            f.sA1 = (long long)oK * np * oK;
            f.sC1 = nov;
            const double fb = 8.0 * ((double)mm * np * oK * oK + (double)np * oK * vK + 2.0 * mm * oK * vK);
            dgemm(pf, st, "Kx_stage2", false, false, oK, vK, np * oK, -c->opt.cx, c->ws_M.p, (long long)np * oK, tP,
                  vK, 1.0, bx + (long long)o0 * nvir, nvir, f, c->ws_split.p, c->ws_split.n, fb);
        }
    }
}

// (A + B) X and (A - B) X from A X and B X (Sec. 2, Eq. hessian)
void matvec_pm(tr_ctx *c, int m, const double *X, double *P, double *M)
{
    if (m <= 0) return;
    matvec(c, m, X, P);
    matvec_b(c, m, X, M);
    const long long n = (long long)m * c->nov;
    TR_LAUNCH(c->prof, c->st, "pm_combine", 0, 32.0 * n, pm_combine<<<grid_for(n), 256, 0, c->st>>>(P, M, n));
}

// ---------------------------------------------------------------- FP64 form on the tensor cores

// Sliced copies of the built FP64 tensors (7 slices, FP64-level products):
// (P|ia) by rows P (J contraction) and by rows ia (J expansion), T_ab^P by rows
// (P, a) with K = b, T_ij by rows i with K = (P, j).
void build_tc(tr_ctx *c)
{
    const int S = OZ_SLICES_FP64;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const long long nov = c->nov;
    if (c->nJ > 0 && !c->opt.j_ao) {
        c->ozs_Y.alloc(cdiv(oz_bytes(c->nJ, (int)nov, S), 8), &c->budget, "sliced (P|ia)");
        oz_bind(c->oz_Y, c->ozs_Y.p, c->nJ, (int)nov, S);
        oz_split(pf, st, "oz_split_Y", c->Y.p, nov, 1, c->oz_Y);
        c->ozs_YT.alloc(cdiv(oz_bytes(nov, c->nJ, S), 8), &c->budget, "sliced (P|ia) by ia");
        oz_bind(c->oz_YT, c->ozs_YT.p, nov, c->nJ, S);
        oz_split(pf, st, "oz_split_YT", c->Y.p, 1, nov, c->oz_YT);
    }
    if (c->k_active) {
        const int nK = c->nK, oK = c->oK, vK = c->vK;
        c->ozs_Tab.alloc(cdiv(oz_bytes((long long)nK * vK, vK, S), 8), &c->budget, "sliced T_ab");
        oz_bind(c->oz_Tab, c->ozs_Tab.p, (long long)nK * vK, vK, S);
        oz_split(pf, st, "oz_split_Tab", c->Tab.p, vK, 1, c->oz_Tab);
        c->ozs_T2.alloc(cdiv(oz_bytes(oK, nK * oK, S), 8), &c->budget, "sliced T_ij");
        oz_bind(c->oz_T2, c->ozs_T2.p, oK, nK * oK, S);
        oz_split(pf, st, "oz_split_T2", c->T2.p, (long long)nK * oK, 1, c->oz_T2);
        if (c->opt.tddft) {
            // full TDDFT: t^P_ia by rows (P, i) with K = a, and by rows a with K = (P, i)
            c->ozs_Tia.alloc(cdiv(oz_bytes((long long)nK * oK, vK, S), 8), &c->budget, "sliced T_ia");
            oz_bind(c->oz_Tia, c->ozs_Tia.p, (long long)nK * oK, vK, S);
            oz_split(pf, st, "oz_split_Tia", c->Tia.p, vK, 1, c->oz_Tia);
            c->ozs_TiaT.alloc(cdiv(oz_bytes(vK, nK * oK, S), 8), &c->budget, "sliced T_ia by a");
            oz_bind(c->oz_TiaT, c->ozs_TiaT.p, vK, nK * oK, S);
            oz_split(pf, st, "oz_split_TiaT", c->Tia.p, 1, vK, c->oz_TiaT);
        }
    }
    TR_CUDA(cudaStreamSynchronize(st));
}

// P chunk of the exchange stages: M in FP64 plus its slices, at most
// matvec_ws_bytes; chunk starts P0 oK fall on 32-value K blocks of T_ij
static int tc_pchunk(const tr_ctx *c, int mb)
{
    if (!c->k_active) return 0;
    const int q = 32 / std::gcd(c->oK, 32);
    const double per = (double)mb * c->vK * c->oK * (8.0 + 2.0 * ((OZ_SLICES_FP64 + 1) & ~1));
    int npk = (int)std::max(1.0, std::floor((double)c->opt.matvec_ws_bytes / per));
    npk = std::max(q, npk / q * q);
    npk = std::min(npk, 65535 / std::max(mb, 1) / q * q);
    return std::max(1, std::min(npk, c->nK));
}

void reserve_tc(tr_ctx *c, int mb)
{
    const int S = OZ_SLICES_FP64;
    const long long nov = c->nov;
    c->ws_split.reserve((size_t)2 << 20, &c->budget, "split-K workspace");
    c->ozw_X.reserve(cdiv(oz_bytes(mb, (int)nov, S), 8), &c->budget, "sliced trial vectors");
    if (c->nJ > 0 && !c->opt.j_ao) c->ozw_Z.reserve(cdiv(oz_bytes(mb, c->nJ, S), 8), &c->budget, "sliced J intermediate");
    if (c->k_active) {
        const int npk = tc_pchunk(c, mb);
        c->tc_npk = npk;
        c->ws_Xw.reserve((size_t)mb * c->oK * c->vK, &c->budget, "K workspace");
        c->ozw_Xw.reserve(cdiv(oz_bytes((long long)mb * c->oK, c->vK, S), 8), &c->budget, "sliced window");
        // full TDDFT: the (ib|ja) intermediate E [m][i][(P, j)] has oK rows per vector in place of vK
        const long long w = c->opt.tddft ? std::max(c->oK, c->vK) : c->vK;
        c->ws_Mf.reserve((size_t)mb * w * npk * c->oK, &c->budget, "K intermediate");
        c->ozw_M.reserve(cdiv(oz_bytes((long long)mb * w, npk * c->oK, S), 8), &c->budget,
                         "sliced K intermediate");
    }
}

// Coulomb term from the stored (P|ia) on the tensor cores (7 slices):
// out += 2 (P|ia) (P|Q)^-1 (Q|jb) X, the metric step in FP64
static void j_stored_tc(tr_ctx *c, int mm, const double *x, double *out)
{
    const int S = OZ_SLICES_FP64;
    Prof &pf = c->prof;
    cudaStream_t st = c->st;
    const int nJ = c->nJ;
    const long long nov = c->nov;
    int *err = c->flag.p + 1;
    OzMat Xs, Zs;
    oz_bind(Xs, c->ozw_X.p, mm, (int)nov, S);
    oz_split(pf, st, "oz_split_X", x, nov, 1, Xs);
    // Z[P][m] = sum_ia (P|ia) X_m,ia   (long K: split over CTAs)
    OzOut oz;
    oz.d = c->ws_Z.p;
    oz.ldm = mm;
    oz.ldn = 1;
    const int tiles = cdiv(nJ, 128) * cdiv(mm, 64);
    int ks = std::max(1, 2 * 152 / tiles);
    ks = (int)std::min<long long>(ks, (long long)c->ws_split.n / ((long long)nJ * mm));
    oz_gemm(pf, st, "J_contract_tc", c->oz_Y, 0, 0, 0, 0, Xs, 0, 0, 0, 0, nJ, mm, c->oz_Y.nkb, 1, 1, oz, err,
            std::max(ks, 1), c->ws_split.p, c->ws_split.n);
    dgemm(pf, st, "J_metric", false, false, nJ, mm, nJ, 1.0, c->GinvJ.p, nJ, c->ws_Z.p, mm, 0.0, c->ws_Z2.p, mm,
          Batch(), nullptr, 0);
    // out[m][ia] += 2 sum_P (P|ia) Zt[P][m]: rows ia of the output, columns m
    oz_bind(Zs, c->ozw_Z.p, mm, nJ, S);
    oz_split(pf, st, "oz_split_Z", c->ws_Z2.p, 1, mm, Zs);
    OzOut oe;
    oe.d = out;
    oe.ldm = 1;
    oe.ldn = nov;
    oe.alpha = 2.0;
    oe.accumulate = true;
    oz_gemm(pf, st, "J_expand_tc", c->oz_YT, 0, 0, 0, 0, Zs, 0, 0, 0, 0, (int)nov, mm, c->oz_YT.nkb, 1, 1, oe, err);
}

// A X with every large product on the tensor cores (7 slices): the same steps
// and order as the FP64 matvec (Sec. 3.1 for J, Sec. 3.2 for K)
void matvec_tc(tr_ctx *c, int m, const double *X, double *AX)
{
    const int S = OZ_SLICES_FP64;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ;
    const long long nov = c->nov;
    const int mb = std::min(m, c->mblk);
    reserve_matvec(c, mb);  // J workspaces and the sliced operands
    const int oK = c->oK, vK = c->vK, o0 = c->o0, nK = c->nK;
    int *err = c->flag.p + 1;
    for (int m0 = 0; m0 < m; m0 += mb) {
        const int mm = std::min(mb, m - m0);
        const double *x = X + (long long)m0 * nov;
        double *ax = AX + (long long)m0 * nov;
        TR_LAUNCH(pf, st, "diag", 0, 8.0 * nov * (2.0 * mm + 1.0),
                  diag_kernel<<<grid_for(nov), 256, 0, st>>>(c->D.p, x, ax, nov, mm));
        if (nJ && c->opt.j_ao) {
            j_ao_block(c, mm, x, ax);
        } else if (nJ) {
            j_stored_tc(c, mm, x, ax);  // AX += 2 J
        }
        if (c->k_active) {
            const long long tot = (long long)mm * oK * vK;
            TR_LAUNCH(pf, st, "gather_window", 0, 16.0 * tot,
                      gather_window<<<grid_for(tot), 256, 0, st>>>(x, c->ws_Xw.p, mm, nocc, nvir, o0, oK, vK));
            OzMat Xws, Ms;
            oz_bind(Xws, c->ozw_Xw.p, (long long)mm * oK, vK, S);
            oz_split(pf, st, "oz_split_Xw", c->ws_Xw.p, vK, 1, Xws);
            const int npk = c->tc_npk;
            for (int P0 = 0; P0 < nK; P0 += npk) {
                const int np = std::min(npk, nK - P0);
                const long long Kp = (long long)np * oK;
                // M[m][a][P oK + j] = sum_b T_ab^P X_m,jb   (batches P, m)
                OzOut o1;
                o1.d = c->ws_Mf.p;
                o1.s1 = oK;
                o1.s2 = (long long)vK * Kp;
                o1.ldm = Kp;
                o1.ldn = 1;
                oz_gemm(pf, st, "K_stage1_tc", c->oz_Tab, (long long)P0 * vK, vK, 0, 0, Xws, 0, 0, oK, 0, vK, oK,
                        c->oz_Tab.nkb, np, mm, o1, err);
                oz_bind(Ms, c->ozw_M.p, (long long)mm * vK, (int)Kp, S);
                oz_split(pf, st, "oz_split_M", c->ws_Mf.p, Kp, 1, Ms);
                // AX_m[o0 + i][a] -= cx sum_(P,j) T_ij^P M[m][a][P oK + j]
                OzOut o2;
                o2.d = ax + (long long)o0 * nvir;
                o2.s1 = nov;
                o2.ldm = nvir;
                o2.ldn = 1;
                o2.alpha = -c->opt.cx;
                o2.accumulate = true;
                oz_gemm(pf, st, "K_stage2_tc", c->oz_T2, 0, 0, 0, (int)((long long)P0 * oK / 32), Ms, 0, vK, 0, 0, oK,
                        vK, Ms.nkb, mm, 1, o2, err);
            }
        }
    }
}

// B X of full TDDFT with every large product on the tensor cores (7 slices): the
// steps and order of matvec_b
void matvec_b_tc(tr_ctx *c, int m, const double *X, double *BX)
{
    const int S = OZ_SLICES_FP64;
    cudaStream_t st = c->st;
    Prof &pf = c->prof;
    const int nocc = c->nocc, nvir = c->nvir, nJ = c->nJ;
    const long long nov = c->nov;
    const int mb = std::min(m, c->mblk);
    reserve_matvec(c, mb);
    const int oK = c->oK, vK = c->vK, o0 = c->o0, nK = c->nK;
    int *err = c->flag.p + 1;
    for (int m0 = 0; m0 < m; m0 += mb) {
        const int mm = std::min(mb, m - m0);
        const double *x = X + (long long)m0 * nov;
        double *bx = BX + (long long)m0 * nov;
        TR_CUDA(cudaMemsetAsync(bx, 0, sizeof(double) * (size_t)mm * nov, st));
        if (nJ && c->opt.j_ao) {
            j_ao_block(c, mm, x, bx);
        } else if (nJ) {
            j_stored_tc(c, mm, x, bx);  // BX += 2 J (BX zeroed above)
        }
        if (!c->k_active) continue;
        const long long tot = (long long)mm * oK * vK;
        TR_LAUNCH(pf, st, "gather_window", 0, 16.0 * tot,
                  gather_window<<<grid_for(tot), 256, 0, st>>>(x, c->ws_Xw.p, mm, nocc, nvir, o0, oK, vK));
        OzMat Xws, Es;
        oz_bind(Xws, c->ozw_Xw.p, (long long)mm * oK, vK, S);
        oz_split(pf, st, "oz_split_Xw", c->ws_Xw.p, vK, 1, Xws);
        const int npk = c->tc_npk;
        for (int P0 = 0; P0 < nK; P0 += npk) {
            const int np = std::min(npk, nK - P0);
            const long long Kp = (long long)np * oK;
            // E[m][i][P oK + j] = sum_b t^P_ib X_m,jb   (batches P, m)
            OzOut o1;
            o1.d = c->ws_Mf.p;
            o1.s1 = oK;
            o1.s2 = (long long)oK * Kp;
            o1.ldm = Kp;
            o1.ldn = 1;
            oz_gemm(pf, st, "Kx_stage1_tc", c->oz_Tia, (long long)P0 * oK, oK, 0, 0, Xws, 0, 0, oK, 0, oK, oK,
                    c->oz_Tia.nkb, np, mm, o1, err);
            oz_bind(Es, c->ozw_M.p, (long long)mm * oK, (int)Kp, S);
            oz_split(pf, st, "oz_split_E", c->ws_Mf.p, Kp, 1, Es);
            // BX_m[o0 + i][a] -= cx sum_(P,j) E[m][i][P oK + j] t^P_ja
            OzOut o2;
            o2.d = bx + (long long)o0 * nvir;
            o2.s1 = nov;
            o2.ldm = nvir;
            o2.ldn = 1;
            o2.alpha = -c->opt.cx;
            o2.accumulate = true;
            oz_gemm(pf, st, "Kx_stage2_tc", Es, 0, oK, 0, 0, c->oz_TiaT, 0, 0, 0, (int)((long long)P0 * oK / 32), oK,
                    vK, Es.nkb, mm, 1, o2, err);
        }
    }
}

}  // namespace tr
