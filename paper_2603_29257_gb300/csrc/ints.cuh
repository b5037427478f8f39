// Gaussian integral kernels of libtdarisp (internal): Boys table, three-
// and two-centre two-electron integrals for the operator
// (ka + kb erf(omega r))/r over spherical AO shells (l <= 2) and
// uncontracted auxiliary s/p primitives.
#pragma once

#include <vector>

#include "common.cuh"

namespace tr {

struct ShellDev {
    double x, y, z;
    int l, nprim, pstart, ao;
};

// auxiliary function: comp = -1 for s, 0/1/2 for p_x/p_y/p_z; out = row index
struct AuxDev {
    double x, y, z, e;
    int comp, out;
};

constexpr int BOYS_NPTS = 1921;          // T = 0 .. 60 step 1/32
constexpr int BOYS_NCOL = 14;            // F_0 .. F_12, then e^{-T}
constexpr int BOYS_COL_EXP = 13;
constexpr double BOYS_DT = 1.0 / 32.0;
constexpr double BOYS_TMAX = 60.0;       // beyond: asymptotic form (e^{-T} < 1e-26 dropped)

// Host: tabulate F_n(T_k) and e^{-T_k} for the device Taylor interpolation.
void boys_table(std::vector<double> &tab);

// AO shell pairs grouped by angular class (la, lb), la >= lb, in the order
// (0,0) (1,0) (1,1) (2,0) (2,1) (2,2).  off[c] .. off[c+1] index pairs[].
struct PairList {
    std::vector<int2> pairs;
    int off[7];
    int ntotal;
    // primitive pairs of each kept shell pair that pass the screening, with the
    // data no auxiliary function changes: range[i] = (first, count) into prim,
    // prim = 6 doubles (P_x, P_y, P_z, p, 1/p, c_a c_b exp(-ab/p |AB|^2))
    std::vector<int2> range;
    std::vector<double> prim;
};

// Host: screened pair list and primitive-pair table.  A primitive pair is kept
// when |c_a c_b| exp(-ab/(a+b) |AB|^2) (pi/(a+b))^{3/2} (1 + |AB|)^{la+lb} >= screen.
PairList make_pairs(const std::vector<ShellDev> &sh, const std::vector<double> &pexp,
                    const std::vector<double> &pcoef, double screen);

// out[f][mu][nu] (+= nothing: caller zeroes) for auxiliary functions aux[0..naux)
// of which aux_class_off[c]..aux_class_off[c+1] have comp = c - 1.
// The launches run on the side streams when side is not null (forked from and
// joined back to st).
// atoms[0..natoms): s functions (out = first of s, p_x, p_y, p_z) of whole J
// atoms in the chunk; when natoms > 0 the light pair classes compute all four
// functions of an atom per thread and the remaining classes use aux (which then
// must hold the same functions by component).
void int3c(Prof &prof, cudaStream_t st, SideStreams *side, const ShellDev *sh, const int2 *pairs,
           const int2 *prange, const double *prim, const int *pair_off, const AuxDev *aux, const int *aux_class_off,
           const AuxDev *atoms, int natoms, int nao, double *out, double ka, double kb, double omega,
           const double *boys);

// out[i][j] = (P_i|Q_j) for auxiliary functions aux[0..n) with out index aux[i].out.
// <mu| r - O |nu> for the screened AO shell pairs: out[3][nao][nao] (x, y, z),
// zero for pairs dropped by the screening
void dipole_ints(Prof &prof, cudaStream_t st, const ShellDev *sh, const int2 *pairs, const int2 *prange,
                 const double *prim, const int *off, int nao, const double O[3], double *out);

void int2c(Prof &prof, cudaStream_t st, const AuxDev *aux, int n, double ka, double kb, double omega,
           const double *boys, double *out);

}  // namespace tr
