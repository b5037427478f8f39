// Context of libtdarisp (internal): molecule, orbitals, built tensors and
// workspaces of one TDA-risp problem on one GPU.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"
#include "ints.cuh"
#include "linalg.cuh"
#include "ozgemm.cuh"
#include "tcgemm.cuh"

struct tr_ctx {
    tr_options opt{};
    cudaStream_t st = nullptr;
    std::string err;
    tr::Prof prof;
    tr::Budget budget;
    int device = 0;

    // molecule (Sec. 2: geometry, AO basis, auxiliary exponents)
    bool have_mol = false;
    std::vector<int> Z;
    std::vector<double> xyz, aux_exp;
    std::vector<tr::ShellDev> shells_h;
    std::vector<double> pexp_h, pcoef_h;
    int nao = 0;
    tr::PairList pl;
    // block sparsity of an AO integral matrix (P|mn) from the kept shell pairs: per
    // column tile of 64 functions, the row tiles of 16 with a kept pair (the same
    // for every auxiliary function)
    std::vector<int> kt_list_h, kt_count_h;
    tr::DevBuf<int> kt_list, kt_count;
    tr::KTiles ktiles;
    // the same pattern in K blocks of 32 functions per 64-function tile, for the
    // tensor-core transforms: kb_list[nt * kb_ld + t] for t < kb_count[nt]
    std::vector<int> kb_list_h, kb_count_h;
    tr::DevBuf<int> kb_list, kb_count;
    tr::DevBuf<unsigned char> kb_mask;  // [nt][kb]: block kb listed for tile nt
    int kb_ld = 0;
    tr::DevBuf<tr::ShellDev> shells;
    tr::DevBuf<double> pexp, pcoef, boys, prim;
    tr::DevBuf<int2> pairs, prange;
    // auxiliary functions (Sec. 3.2): J = s + p on non-H atoms, K = s on non-H atoms
    std::vector<tr::AuxDev> auxJ_h, auxK_h;  // in output order
    int nJ = 0, nK = 0;
    tr::DevBuf<tr::AuxDev> aux_ws;           // per-chunk class-sorted copy
    // class-sorted auxiliary lists of fixed chunkings uploaded once (the AO form of
    // J): a chunk found here needs no upload and no synchronisation, so its
    // integrals can be captured in a graph
    struct AuxChunk {
        int which, p0, np, natoms;
        long long off;
        int cls[5];
    };
    tr::DevBuf<tr::AuxDev> aux_cache;
    std::vector<AuxChunk> aux_cache_idx;

    // orbitals
    bool have_orb = false;
    int nmo = 0, nocc = 0, nvir = 0;
    long long nov = 0;
    tr::DevBuf<double> C, eps;
    std::vector<double> eps_h;
    int o0 = 0, oK = 0, vK = 0;              // exchange window (Sec. 3.2)

    // built operator
    bool built = false;
    tr::DevBuf<double> Y;      // (P|ia) [nJ][nocc][nvir], Coulomb
    tr::DevBuf<double> GinvJ;  // (P|Q)^-1 [nJ][nJ]
    tr::DevBuf<double> GinvK;  // K-operator metric inverse [nK][nK]
    tr::DevBuf<double> T2;     // T_ij^P stored [i][P][j]
    tr::DevBuf<double> Tab;    // T_ab^P = (ab|P) [nK][vK][vK]
    tr::DevBuf<double> D;      // e_a - e_i [nocc][nvir]
    tr::DevBuf<double> Tia;    // full TDDFT: L_K^-1 (P|ia) on the window [nK][oK][vK]
    bool k_active = false;

    // reduced-precision form: FP32 copies (value and tf32 remainder) and tensor maps
    tr::DevBuf<float> Y32, Tab_h, Tab_l, T2_h, T2_l, Xw_h, Xw_l, Mt_h, Mt_l, X32, Z32;
    tr::TcMat tm_tab, tm_t2, tm_xw, tm_mt;
    int oKp = 0, vKp = 0, mixed_mb = 0, mixed_npk = 0;
    int tc_bn = 128;  // tensor-core output tile width of the K stages (64 or 128)

    // FP64 form on the tensor cores (TR_FP64_TC): sliced tensors (built once) and
    // per-block sliced operands
    tr::DevBuf<double> ozs_Y, ozs_YT, ozs_Tab, ozs_T2, ozw_X, ozw_Xw, ozw_Z, ozw_M, ws_Mf;
    tr::OzMat oz_Y, oz_YT, oz_Tab, oz_T2;
    tr::DevBuf<double> ozs_Tia, ozs_TiaT;  // full TDDFT: T_ia by rows (P, i) and by rows a
    tr::OzMat oz_Tia, oz_TiaT;
    int tc_npk = 0;

    // workspaces
    tr::DevBuf<double> ws_split, ws_Z, ws_Z2, ws_Xw, ws_M;
    // Coulomb term on the fly in the AO basis (j_ao): half-transformed and AO
    // transition densities, AO potentials, fit coefficients, integral chunk
    tr::DevBuf<double> ws_jT, ws_jD, ws_jU, ws_jR, ws_jI;
    // the function pairs (k, l) of the kept shell pairs as flat indices k nao + l
    // (ascending; -1: not yet listed for this molecule) and the packed copies of
    // the integral chunk, the AO densities and the AO potentials over them
    tr::DevBuf<int> kl_idx;
    long long nkl = -1;
    tr::DevBuf<double> ws_jIp, ws_jDp, ws_jUp;
    tr::DevBuf<int> flag;
    int mblk = 32;

    // Davidson state
    tr::DevBuf<double> V, W, Hs, Hw, Yev, Yw, theta, Xr, R, T, Tt, Tn, Wn, Cs, Ss, Gc, rn, part;
    // full TDDFT: (A - B) products of V and of the new vectors, their subspace
    // matrix, and the reduced problem's Cholesky factor, copies and coefficients
    tr::DevBuf<double> Wm, Wnm, Hsm, Lr, Mr, Qr, Ca, Cb;
    // sliced copies of V and W (and of the new directions) for the subspace
    // products on the tensor cores (forms that use them, when all rows are on the device)
    tr::DevBuf<double> dvs_V, dvs_W, dvs_T, dvs_Vt, dvs_Wt, dvs_Y, dvs_C;
    tr::OzMat dz_V, dz_W, dz_Vt, dz_Wt;  // dz_Vt, dz_Wt: V and W by columns (rows = nov, K = subspace index)
    tr::DevBuf<int> dz_eW;               // the one exponent of dz_Wt
    // full TDDFT: the (A - B) V rows sliced by rows and by columns, and the exponent of the latter
    tr::DevBuf<double> dvs_Wm, dvs_Wmt;
    tr::OzMat dz_Wm, dz_Wmt;
    tr::DevBuf<int> dz_eWm;
    tr::DevBuf<int> idx_dev;
    tr::DevBuf<double> gsel;  // candidates of the initial-guess selection
    double *h_pin = nullptr;  // pinned: residual norms, Ritz values, flags of the Davidson
    // spill of V/W rows to pinned host memory: staging slots, copy stream, events
    tr::DevBuf<double> stage;
    cudaStream_t cst = nullptr;
    cudaEvent_t sev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // side streams for the independent integral launches of one chunk
    tr::SideStreams side;

    ~tr_ctx()
    {
        if (st) cudaStreamSynchronize(st);
        side.release();
        if (cst) {
            cudaStreamSynchronize(cst);
            cudaStreamDestroy(cst);
        }
        for (auto e : sev)
            if (e) cudaEventDestroy(e);
        if (h_pin) cudaFreeHost(h_pin);
    }
};

namespace tr {

void set_molecule(tr_ctx *c, int natm, const int *Z, const double *xyz, const double *aux_exp,
                  int nshell, const tr_shell *shells);
void set_orbitals(tr_ctx *c, int nao, int nmo, int nocc, const double *C, const double *eps,
                  int on_device);
void refresh_molecule(tr_ctx *c);
void refresh_window(tr_ctx *c);
void build(tr_ctx *c);
void int3c_ao(tr_ctx *c, int which, int p0, int np, double *out);
void int2c_aux(tr_ctx *c, int which, double *out);
void get_tensor(tr_ctx *c, int which, double *out, int on_device);
// AX = A X for m device vectors (asynchronous on c->st)
void matvec(tr_ctx *c, int m, const double *X, double *AX);
// allocate the matvec workspaces for blocks of up to m vectors
void reserve_matvec(tr_ctx *c, int m);
// full TDDFT (asynchronous on c->st): BX = B X; P = (A + B) X and M = (A - B) X
void matvec_b(tr_ctx *c, int m, const double *X, double *BX);
void matvec_pm(tr_ctx *c, int m, const double *X, double *P, double *M);
// slices of the tensor-core MO transforms (0: FP64 pipe)
int xform_slices(const tr_ctx *c);
// Ozaki slices of the Davidson subspace products on the tensor cores
int dav_slices(const tr_ctx *c);
// estimated peak device bytes of tr_build + tr_solve
size_t footprint(tr_ctx *c);
// FP64 form on the tensor cores: slice the built tensors; matvec workspaces; A X
void build_tc(tr_ctx *c);
void reserve_tc(tr_ctx *c, int mb);
void matvec_tc(tr_ctx *c, int m, const double *X, double *AX);
void matvec_b_tc(tr_ctx *c, int m, const double *X, double *BX);
// three-centre integrals of aux functions [p0, p0+np) of set which (0 = J, 1 = K)
void compute_int3c_chunk(tr_ctx *c, int which, int p0, int np, double *out);
// Coulomb term on the fly in the AO basis (jao.cu): AX += 2 J for mm vectors;
// workspaces for blocks of up to mb vectors, and their bytes
void j_ao_block(tr_ctx *c, int mm, const double *X, double *AX);
void reserve_jao(tr_ctx *c, int mb);
size_t jao_bytes(const tr_ctx *c, int mb);
int jao_chunk_size(const tr_ctx *c);
// transition properties (props.cu): mu[n][3] electric transition dipoles about O,
// f[n] oscillator strengths; device pointers, synchronous
void transition_dipoles(tr_ctx *c, int n, const double *X, const double O[3], double *mu);
void oscillator_strengths(tr_ctx *c, int n, const double *omega, const double *X, double *f);
// upload the class-sorted auxiliary lists of every chunk of npc functions of set
// which (0 = J, 1 = K) once
void prepare_aux_chunks(tr_ctx *c, int which, int npc);
// reduced-precision form (mixed.cu)
void get_tensor_mixed(tr_ctx *c, int which, double *out, int on_device);
void build_mixed(tr_ctx *c);
void reserve_mixed(tr_ctx *c, int mb);
void matvec_mixed(tr_ctx *c, int m, const double *X, double *AX);
// Davidson; with opt.tddft the full problem, X+Y into X and X-Y into Xm (may be null)
int solve(tr_ctx *c, double *omega, double *X, double *Xm, double *resid, int on_device, tr_solve_info *info);
int solve_batch(tr_ctx **ctxs, int nb, double **omega, double **X, double **resid, int on_device,
                tr_solve_info *infos, int autotune_tiles);

}  // namespace tr
