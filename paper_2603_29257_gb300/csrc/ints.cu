// Three- and two-centre Gaussian integrals by the McMurchie-Davidson scheme.
//
// For an AO primitive pair (a at A, b at B) the product of Cartesian factors
// is expanded in Hermite Gaussians at P = (aA + bB)/p with coefficients
// E^{ij}_t; the auxiliary primitive at C is a Hermite Gaussian of order 0
// (s) or 1 (p, coefficient 1/(2c)); the Coulomb-type integral of two Hermite
// Gaussians is 2 pi^{5/2}/(p c sqrt(p+c)) (-1)^{ket order} R_{tuv}(P - C)
// with R^n_{000} = (-2 rho)^n G_n and the usual Hermite recursion.
// For (ka + kb erf(omega r))/r:  G_n = ka F_n(T) + kb s^{n+1/2} F_n(s T),
// s = omega^2/(omega^2 + rho), T = rho |P-C|^2  (attenuated Boys function).
//
// One thread computes one (AO shell pair, auxiliary function) block,
// contracting over primitive pairs in registers, then transforms d shells
// to the real solid harmonics xy, yz, (2zz-xx-yy)/(2 sqrt3), xz, (xx-yy)/2.
#include "ints.cuh"

#include <algorithm>
#include <cmath>

namespace tr {

// ---------------------------------------------------------------- Boys table

void boys_table(std::vector<double> &tab)
{
    tab.assign((size_t)BOYS_NPTS * BOYS_NCOL, 0.0);
    const int nmax = BOYS_COL_EXP - 1;
    for (int k = 0; k < BOYS_NPTS; ++k) {
        long double T = (long double)k * (long double)BOYS_DT;
        // F_nmax(T) = e^{-T} sum_j (2T)^j / prod_{i=0..j} (2 nmax + 2i + 1)
        long double term = 1.0L / (2 * nmax + 1), sum = term;
        for (int j = 1; j < 2000; ++j) {
            term *= 2.0L * T / (long double)(2 * nmax + 2 * j + 1);
            sum += term;
            if (term <= sum * 1e-21L) break;
        }
        long double e = expl(-T);
        long double f[BOYS_COL_EXP];
        f[nmax] = e * sum;
        for (int n = nmax - 1; n >= 0; --n) f[n] = (2.0L * T * f[n + 1] + e) / (long double)(2 * n + 1);
        for (int n = 0; n <= nmax; ++n) tab[(size_t)k * BOYS_NCOL + n] = (double)f[n];
        tab[(size_t)k * BOYS_NCOL + BOYS_COL_EXP] = (double)e;
    }
}

// ---------------------------------------------------------------- pair list

PairList make_pairs(const std::vector<ShellDev> &sh, const std::vector<double> &pexp,
                    const std::vector<double> &pcoef, double screen)
{
    PairList pl;
    // a kept shell pair with its primitive pairs that pass the screening
    struct Kept {
        int2 ab;
        std::vector<double> prim;  // 6 doubles per primitive pair
    };
    std::vector<Kept> cls[6];
    const int nsh = (int)sh.size();
    pl.ntotal = 0;
    for (int i = 0; i < nsh; ++i) {
        for (int j = 0; j <= i; ++j) {
            pl.ntotal += 1;
            int a = i, b = j;
            if (sh[a].l < sh[b].l) std::swap(a, b);
            const ShellDev &A = sh[a], &B = sh[b];
            const double ABx = A.x - B.x, ABy = A.y - B.y, ABz = A.z - B.z;
            const double AB2 = ABx * ABx + ABy * ABy + ABz * ABz;
            const double poly = std::pow(1.0 + std::sqrt(AB2), A.l + B.l);
            Kept k;
            k.ab = make_int2(a, b);
            for (int u = 0; u < A.nprim; ++u)
                for (int v = 0; v < B.nprim; ++v) {
                    const double ea = pexp[A.pstart + u], eb = pexp[B.pstart + v];
                    const double p = ea + eb, ip = 1.0 / p;
                    const double K = pcoef[A.pstart + u] * pcoef[B.pstart + v] * std::exp(-ea * eb * ip * AB2);
                    if (std::fabs(K) * M_PI * ip * std::sqrt(M_PI * ip) * poly < screen) continue;
                    const double P[6] = {(ea * A.x + eb * B.x) * ip, (ea * A.y + eb * B.y) * ip,
                                         (ea * A.z + eb * B.z) * ip, p, ip, K};
                    k.prim.insert(k.prim.end(), P, P + 6);
                }
            if (k.prim.empty()) continue;  // no primitive pair passes: the shell pair is dropped
            const int c = A.l == 0 ? 0 : (A.l == 1 ? 1 + B.l : 3 + B.l);
            cls[c].push_back(std::move(k));
        }
    }
    // within a class, shell pairs with equal numbers of kept primitive pairs sit
    // next to each other: the threads of a warp then run loops of equal length
    pl.off[0] = 0;
    for (int c = 0; c < 6; ++c) {
        std::stable_sort(cls[c].begin(), cls[c].end(),
                         [](const Kept &x, const Kept &y) { return x.prim.size() < y.prim.size(); });
        for (const Kept &k : cls[c]) {
            const int first = (int)(pl.prim.size() / 6);
            pl.pairs.push_back(k.ab);
            pl.prim.insert(pl.prim.end(), k.prim.begin(), k.prim.end());
            pl.range.push_back(make_int2(first, (int)(k.prim.size() / 6)));
        }
        pl.off[c + 1] = (int)pl.pairs.size();
    }
    return pl;
}

namespace {

constexpr double TWO_PI_52 = 34.98683665524972;  // 2 pi^{5/2}

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// exponent of direction d in Cartesian component k of shell l
// (l=1: x,y,z; l=2: xx,xy,xz,yy,yz,zz)
__host__ __device__ constexpr int cexp(int l, int k, int d)
{
    return l == 0 ? 0
         : l == 1 ? (k == d ? 1 : 0)
         : (d == 0 ? (k == 0 ? 2 : (k == 1 || k == 2) ? 1 : 0)
          : d == 1 ? (k == 3 ? 2 : (k == 1 || k == 4) ? 1 : 0)
                   : (k == 5 ? 2 : (k == 2 || k == 4) ? 1 : 0));
}

template <int L>
__device__ __forceinline__ void boys_eval(double T, const double *__restrict__ tab, double *F)
{
    // F_L first, then the downward recursion F_n = (2T F_{n+1} + e^{-T}) / (2n+1)
    double e = 0.0;
    if (T < BOYS_TMAX) {
        const int k = __double2int_rn(T * (1.0 / BOYS_DT));
        const double dT = k * BOYS_DT - T;  // T_k - T, |dT| <= 1/64
        const double *f = tab + k * BOYS_NCOL;
        // F_L(T) = sum_j F_{L+j}(T_k) (T_k - T)^j / j!
        double s = __ldg(f + L + 6);
#pragma unroll
        for (int j = 5; j >= 0; --j) s = fma(s, dT * (1.0 / (j + 1)), __ldg(f + L + j));
        F[L] = s;
        if (L > 0) {
            // e^{-T} = e^{-T_k} e^{T_k - T}: degree-8 Taylor polynomial of e^{dT}
            double x = 1.0;
#pragma unroll
            for (int j = 8; j >= 1; --j) x = fma(x, dT * (1.0 / j), 1.0);
            e = __ldg(f + BOYS_COL_EXP) * x;
        }
    } else {
        // F_n(T) = (2n-1)!! / 2^{n+1} sqrt(pi) T^{-n-1/2} up to terms in e^{-T} (< 1e-26)
        const double r = rsqrt(T);
        const double h = 0.5 * r * r;       // 1 / (2T)
        double fn = 0.88622692545275801365 * r;  // sqrt(pi) / 2 / sqrt(T)
#pragma unroll
        for (int n = 0; n < L; ++n) fn *= (2 * n + 1) * h;
        F[L] = fn;
    }
#pragma unroll
    for (int n = L - 1; n >= 0; --n) F[n] = fma(2.0 * T, F[n + 1], e) * (1.0 / (2 * n + 1));
}

// R^n_000 = (-2 rho)^n G_n for the operator (ka + kb erf(omega r))/r
template <int L>
__device__ __forceinline__ void coulomb_aux(double rho, double T, double ka, double kb, double omega,
                                            const double *__restrict__ tab, double *Rn)
{
    double F[L + 1];
    double G[L + 1];
#pragma unroll
    for (int n = 0; n <= L; ++n) G[n] = 0.0;
    if (ka != 0.0) {
        boys_eval<L>(T, tab, F);
#pragma unroll
        for (int n = 0; n <= L; ++n) G[n] = ka * F[n];
    }
    if (kb != 0.0 && omega > 0.0) {
        double s = omega * omega / (omega * omega + rho);
        boys_eval<L>(s * T, tab, F);
        double f = kb * sqrt(s);
#pragma unroll
        for (int n = 0; n <= L; ++n) {
            G[n] = fma(f, F[n], G[n]);
            f *= s;
        }
    }
    double m = 1.0;
#pragma unroll
    for (int n = 0; n <= L; ++n) {
        Rn[n] = m * G[n];
        m *= -2.0 * rho;
    }
}

// Hermite Coulomb integrals R_{tuv} (n = 0 level) for t+u+v <= L, in place.
template <int L>
__device__ __forceinline__ void hermite_R(double X, double Y, double Z, const double *Rn,
                                          double (&R)[L + 1][L + 1][L + 1])
{
    R[0][0][0] = Rn[L];
#pragma unroll
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll
        for (int s = L - n; s >= 1; --s) {
#pragma unroll
            for (int t = s; t >= 0; --t) {
#pragma unroll
                for (int u = s - t; u >= 0; --u) {
                    const int v = s - t - u;
                    if (t > 0)
                        R[t][u][v] = (t > 1 ? (t - 1) * R[t > 1 ? t - 2 : 0][u][v] : 0.0) + X * R[t - 1][u][v];
                    else if (u > 0)
                        R[0][u][v] = (u > 1 ? (u - 1) * R[0][u > 1 ? u - 2 : 0][v] : 0.0) + Y * R[0][u - 1][v];
                    else
                        R[0][0][v] = (v > 1 ? (v - 1) * R[0][0][v > 1 ? v - 2 : 0] : 0.0) + Z * R[0][0][v - 1];
                }
            }
        }
        R[0][0][0] = Rn[n];
    }
}

// Hermite expansion coefficients E^{ij}_t of one direction
template <int LA, int LB>
__device__ __forceinline__ void hermite_E(double PA, double PB, double inv2p,
                                          double (&E)[LA + 1][LB + 1][LA + LB + 1])
{
#pragma unroll
    for (int i = 0; i <= LA; ++i)
#pragma unroll
        for (int j = 0; j <= LB; ++j)
#pragma unroll
            for (int t = 0; t <= LA + LB; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
#pragma unroll
    for (int i = 0; i < LA; ++i)
#pragma unroll
        for (int t = 0; t <= i + 1; ++t)
            E[i + 1][0][t] = (t > 0 ? inv2p * E[i][0][t > 0 ? t - 1 : 0] : 0.0) + PA * E[i][0][t] +
                             (t + 1 <= i ? (t + 1) * E[i][0][t + 1 <= i ? t + 1 : 0] : 0.0);
#pragma unroll
    for (int j = 0; j < LB; ++j)
#pragma unroll
        for (int i = 0; i <= LA; ++i)
#pragma unroll
            for (int t = 0; t <= i + j + 1; ++t)
                E[i][j + 1][t] = (t > 0 ? inv2p * E[i][j][t > 0 ? t - 1 : 0] : 0.0) + PB * E[i][j][t] +
                                 (t + 1 <= i + j ? (t + 1) * E[i][j][t + 1 <= i + j ? t + 1 : 0] : 0.0);
}

// spherical transform of a d shell: row s, Cartesian k
__device__ __forceinline__ double d_sph(int s, int k)
{
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    switch (s) {
        case 0: return k == 1 ? 1.0 : 0.0;
        case 1: return k == 4 ? 1.0 : 0.0;
        case 2: return k == 5 ? r3 : ((k == 0 || k == 3) ? -0.5 * r3 : 0.0);
        case 3: return k == 2 ? 1.0 : 0.0;
        default: return k == 0 ? 0.5 : (k == 3 ? -0.5 : 0.0);
    }
}

// SACC (d-d): the NCA x NCB sums in shared memory, one column per thread, so
// that the Hermite coefficients and R keep the registers.
template <int LA, int LB, int CD, bool SACC>
__global__ void __launch_bounds__(128)
    int3c_kernel(const ShellDev *__restrict__ sh, const int2 *__restrict__ pairs, const int2 *__restrict__ prange,
                 const double *__restrict__ prim, int npair, const AuxDev *__restrict__ aux, int nao,
                 double *__restrict__ out, double ka, double kb, double omega, const double *__restrict__ boys)
{
    constexpr int LC = CD >= 0 ? 1 : 0;
    constexpr int L = LA + LB + LC;
    constexpr int NCA = ncart(LA), NCB = ncart(LB);
    constexpr int DX = CD == 0, DY = CD == 1, DZ = CD == 2;
    extern __shared__ double sacc[];
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npair) return;
    const AuxDev c = aux[blockIdx.y];
    const int2 pr = pairs[ip];
    const ShellDev A = sh[pr.x], B = sh[pr.y];

    double racc[SACC ? 1 : NCA][SACC ? 1 : NCB];
    auto acc = [&](int i, int j) -> double & {
        if constexpr (SACC)
            return sacc[(i * NCB + j) * blockDim.x + threadIdx.x];
        else
            return racc[i][j];
    };
#pragma unroll
    for (int i = 0; i < NCA; ++i)
#pragma unroll
        for (int j = 0; j < NCB; ++j) acc(i, j) = 0.0;

    const double ce = c.e, ice = 1.0 / ce;
    const int2 rg = prange[ip];

    {
        for (int q = rg.x; q < rg.x + rg.y; ++q) {
            // primitive pair (screened on the host): P, p, 1/p, c_a c_b exp(-ab/p |AB|^2)
            const double *pq = prim + 6LL * q;
            const double Px = pq[0], Py = pq[1], Pz = pq[2], p = pq[3], ip_ = pq[4], Kab = pq[5];
            double Ex[LA + 1][LB + 1][LA + LB + 1], Ey[LA + 1][LB + 1][LA + LB + 1],
                Ez[LA + 1][LB + 1][LA + LB + 1];
            hermite_E<LA, LB>(Px - A.x, Px - B.x, 0.5 * ip_, Ex);
            hermite_E<LA, LB>(Py - A.y, Py - B.y, 0.5 * ip_, Ey);
            hermite_E<LA, LB>(Pz - A.z, Pz - B.z, 0.5 * ip_, Ez);
            const double u = 1.0 / (p + ce);
            const double rho = p * ce * u;
            const double X = Px - c.x, Y = Py - c.y, Z = Pz - c.z;
            double Rn[L + 1];
            coulomb_aux<L>(rho, rho * (X * X + Y * Y + Z * Z), ka, kb, omega, boys, Rn);
            double R[L + 1][L + 1][L + 1];
            hermite_R<L>(X, Y, Z, Rn, R);
            double pref = TWO_PI_52 * Kab * ip_ * ice * sqrt(u);  // 2 pi^{5/2} K / (p c sqrt(p + c))
            if (LC) pref *= -0.5 * ice;
#pragma unroll
            for (int ka_ = 0; ka_ < NCA; ++ka_) {
                constexpr int dummy = 0;
                (void)dummy;
#pragma unroll
                for (int kb_ = 0; kb_ < NCB; ++kb_) {
                    const int ax = cexp(LA, ka_, 0), ay = cexp(LA, ka_, 1), az = cexp(LA, ka_, 2);
                    const int bx = cexp(LB, kb_, 0), by = cexp(LB, kb_, 1), bz = cexp(LB, kb_, 2);
                    // sum_t Ex_t sum_u Ey_u sum_v Ez_v R_{t,u,v}: one direction at a time
                    double s = 0.0;
#pragma unroll
                    for (int t = 0; t <= ax + bx; ++t) {
                        double st = 0.0;
#pragma unroll
                        for (int u = 0; u <= ay + by; ++u) {
                            double su = 0.0;
#pragma unroll
                            for (int v = 0; v <= az + bz; ++v)
                                su = fma(Ez[az][bz][v], R[t + DX][u + DY][v + DZ], su);
                            st = fma(Ey[ay][by][u], su, st);
                        }
                        s = fma(Ex[ax][bx][t], st, s);
                    }
                    acc(ka_, kb_) = fma(pref, s, acc(ka_, kb_));
                }
            }
        }
    }

    constexpr int NSA = 2 * LA + 1, NSB = 2 * LB + 1;
    double* o = out + (long long)c.out * nao * nao;
#pragma unroll
    for (int sa = 0; sa < NSA; ++sa) {
#pragma unroll
        for (int sb = 0; sb < NSB; ++sb) {
            double v = 0.0;
#pragma unroll
            for (int ka_ = 0; ka_ < NCA; ++ka_) {
                const double wa = LA == 2 ? d_sph(sa, ka_) : (ka_ == sa ? 1.0 : 0.0);
                if (wa == 0.0) continue;
#pragma unroll
                for (int kb_ = 0; kb_ < NCB; ++kb_) {
                    const double wb = LB == 2 ? d_sph(sb, kb_) : (kb_ == sb ? 1.0 : 0.0);
                    if (wb == 0.0) continue;
                    v = fma(wa * wb, acc(ka_, kb_), v);
                }
            }
            const int mu = A.ao + sa, nu = B.ao + sb;
            o[(long long)mu * nao + nu] = v;
            o[(long long)nu * nao + mu] = v;
        }
    }
}

// The four J functions of one atom (s, p_x, p_y, p_z: same centre and
// exponent, out indices out .. out+3) from one pass over the primitive pairs:
// the Hermite integrals R up to LA+LB+1 serve the s component (R_tuv) and the
// p components (R_{t+1,u,v}, ...), so the Boys values, R recursion and Hermite
// expansion coefficients are shared.
// SACC (the heavy classes d-p, d-d): the 4 x NCA x NCB sums live in shared
// memory, one column per thread (sacc[k * blockDim.x + thread]), so that the
// Hermite coefficients and R keep the registers; otherwise in registers.
template <int LA, int LB, bool SACC>
__global__ void __launch_bounds__(SACC ? 64 : 128)
    int3c_grp_kernel(const ShellDev *__restrict__ sh, const int2 *__restrict__ pairs, const int2 *__restrict__ prange,
                     const double *__restrict__ prim, int npair, const AuxDev *__restrict__ aux, int nao,
                     double *__restrict__ out, double ka, double kb, double omega, const double *__restrict__ boys)
{
    constexpr int L = LA + LB + 1;
    constexpr int NCA = ncart(LA), NCB = ncart(LB);
    extern __shared__ double sacc[];
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npair) return;
    const AuxDev c = aux[blockIdx.y];
    const int2 pr = pairs[ip];
    const ShellDev A = sh[pr.x], B = sh[pr.y];

    double racc[SACC ? 1 : 4][SACC ? 1 : NCA][SACC ? 1 : NCB];
    auto acc = [&](int f, int i, int j) -> double & {
        if constexpr (SACC)
            return sacc[((f * NCA + i) * NCB + j) * blockDim.x + threadIdx.x];
        else
            return racc[f][i][j];
    };
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int i = 0; i < NCA; ++i)
#pragma unroll
            for (int j = 0; j < NCB; ++j) acc(f, i, j) = 0.0;
    const double ce = c.e, ice = 1.0 / ce;
    const int2 rg = prange[ip];
    for (int q = rg.x; q < rg.x + rg.y; ++q) {
        const double *pq = prim + 6LL * q;
        const double Px = pq[0], Py = pq[1], Pz = pq[2], p = pq[3], ip_ = pq[4], Kab = pq[5];
        double Ex[LA + 1][LB + 1][LA + LB + 1], Ey[LA + 1][LB + 1][LA + LB + 1], Ez[LA + 1][LB + 1][LA + LB + 1];
        hermite_E<LA, LB>(Px - A.x, Px - B.x, 0.5 * ip_, Ex);
        hermite_E<LA, LB>(Py - A.y, Py - B.y, 0.5 * ip_, Ey);
        hermite_E<LA, LB>(Pz - A.z, Pz - B.z, 0.5 * ip_, Ez);
        const double u = 1.0 / (p + ce);
        const double rho = p * ce * u;
        const double X = Px - c.x, Y = Py - c.y, Z = Pz - c.z;
        double Rn[L + 1];
        coulomb_aux<L>(rho, rho * (X * X + Y * Y + Z * Z), ka, kb, omega, boys, Rn);
        double R[L + 1][L + 1][L + 1];
        hermite_R<L>(X, Y, Z, Rn, R);
        const double ps_ = TWO_PI_52 * Kab * ip_ * ice * sqrt(u);  // 2 pi^{5/2} K / (p c sqrt(p + c))
        const double pp_ = -0.5 * ice * ps_;
#pragma unroll
        for (int ka_ = 0; ka_ < NCA; ++ka_) {
#pragma unroll
            for (int kb_ = 0; kb_ < NCB; ++kb_) {
                const int ax = cexp(LA, ka_, 0), ay = cexp(LA, ka_, 1), az = cexp(LA, ka_, 2);
                const int bx = cexp(LB, kb_, 0), by = cexp(LB, kb_, 1), bz = cexp(LB, kb_, 2);
                // one direction at a time, as in int3c_kernel; the p components
                // read R one step further along x, y or z
                double s0 = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
                for (int t = 0; t <= ax + bx; ++t) {
                    double t0 = 0.0, tx = 0.0, ty = 0.0, tz = 0.0;
#pragma unroll
                    for (int w = 0; w <= ay + by; ++w) {
                        double w0 = 0.0, wx = 0.0, wy = 0.0, wz = 0.0;
#pragma unroll
                        for (int v = 0; v <= az + bz; ++v) {
                            const double e = Ez[az][bz][v];
                            w0 = fma(e, R[t][w][v], w0);
                            wx = fma(e, R[t + 1][w][v], wx);
                            wy = fma(e, R[t][w + 1][v], wy);
                            wz = fma(e, R[t][w][v + 1], wz);
                        }
                        const double e = Ey[ay][by][w];
                        t0 = fma(e, w0, t0);
                        tx = fma(e, wx, tx);
                        ty = fma(e, wy, ty);
                        tz = fma(e, wz, tz);
                    }
                    const double e = Ex[ax][bx][t];
                    s0 = fma(e, t0, s0);
                    sx = fma(e, tx, sx);
                    sy = fma(e, ty, sy);
                    sz = fma(e, tz, sz);
                }
                acc(0, ka_, kb_) = fma(ps_, s0, acc(0, ka_, kb_));
                acc(1, ka_, kb_) = fma(pp_, sx, acc(1, ka_, kb_));
                acc(2, ka_, kb_) = fma(pp_, sy, acc(2, ka_, kb_));
                acc(3, ka_, kb_) = fma(pp_, sz, acc(3, ka_, kb_));
            }
        }
    }
    constexpr int NSA = 2 * LA + 1, NSB = 2 * LB + 1;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        double *o = out + (long long)(c.out + f) * nao * nao;
#pragma unroll
        for (int sa = 0; sa < NSA; ++sa) {
#pragma unroll
            for (int sb = 0; sb < NSB; ++sb) {
                double v = 0.0;
#pragma unroll
                for (int ka_ = 0; ka_ < NCA; ++ka_) {
                    const double wa = LA == 2 ? d_sph(sa, ka_) : (ka_ == sa ? 1.0 : 0.0);
                    if (wa == 0.0) continue;
#pragma unroll
                    for (int kb_ = 0; kb_ < NCB; ++kb_) {
                        const double wb = LB == 2 ? d_sph(sb, kb_) : (kb_ == sb ? 1.0 : 0.0);
                        if (wb == 0.0) continue;
                        v = fma(wa * wb, acc(f, ka_, kb_), v);
                    }
                }
                const int mu = A.ao + sa, nu = B.ao + sb;
                o[(long long)mu * nao + nu] = v;
                o[(long long)nu * nao + mu] = v;
            }
        }
    }
}

// Cartesian index of (ax, ay, l - ax - ay) in the order of cexp
__host__ __device__ constexpr int cidx(int l, int ax, int ay) { return (l - ax) * (l - ax + 1) / 2 + (l - ax - ay); }

// Heavy pair classes: a warp takes 32 / TW AO shell pairs, TW lanes each, one
// lane per auxiliary atom (the s, p_x, p_y, p_z functions of a J atom, which
// share the Boys values and R up to LA+LB+1) or per auxiliary s function.
// CM selects the functions a launch computes (bit 0 s, 1 p_x, 2 p_y, 3 p_z;
// the outputs go to planes out + 0 .. 3 of the atom).  Small tiles keep the
// lanes busy for chunks of few atoms; the shell pairs of a class are sorted by
// their number of kept primitive pairs, so the pairs of a warp mostly run
// loops of equal length (a shorter one idles with a zero prefactor to the end
// of the warp's loop).
//  - The Hermite coefficients of a primitive pair depend on the pair alone:
//    three lanes of the pair's group compute them (one direction each) into
//    shared memory, and the group reads them from there.
//  - The prefactor 2 pi^{5/2} K / (p c sqrt(p+c)) is folded into R^n_000
//    (R is linear in it); the p functions' common factor -1/(2c) is applied
//    once, after the sums over primitive pairs.
//  - The contraction sum_tuv Ex_t Ey_u Ez_v R_{t+dx,u+dy,v+dz} is factorised:
//    W(t,u) = sum_v Ez_v R_{t,u,v(+1)} per z exponent pair, then
//    V(t) = sum_u Ey_u W(t,u(+1)) per y exponent pair, then the x sum, which
//    starts from the running total.  Every partial sum is computed once and
//    shared by the outputs that use it; the x exponents of an output follow
//    from its y and z exponents, since the shells' l are fixed.
// FP64 instructions are the scarce resource on this GPU, so the warp spends
// them on the contraction and little else.
__host__ __device__ constexpr int popc4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

template <int LA, int LB, int CM>
struct WarpK {
    static constexpr int TW = 8;          // lanes (auxiliary atoms or functions) per shell pair
    static constexpr int PPW = 32 / TW;   // shell pairs per warp
    static constexpr int NAB = ncart(LA) * ncart(LB);
    static constexpr int NF = popc4(CM);
    static constexpr int NACC = NF * NAB;
    // the sums in shared memory, one column per lane, where registers would spill
    static constexpr bool SACC = NACC > 40 || (LA == 2 && LB == 2);
    static constexpr int WARPS = NACC > 80 ? 1 : 2;  // warps per block
    static constexpr size_t SMEM = SACC ? sizeof(double) * 32 * WARPS * NACC : 0;
    // slot of function f (0..3) among the selected ones
    __host__ __device__ static constexpr int slot(int f) { return popc4(CM & ((1 << f) - 1)); }
};

template <int LA, int LB, int CM>
__global__ void __launch_bounds__(32 * WarpK<LA, LB, CM>::WARPS)
    int3c_warp_kernel(const ShellDev *__restrict__ sh, const int2 *__restrict__ pairs, const int2 *__restrict__ prange,
                      const double *__restrict__ prim, int npair, const AuxDev *__restrict__ aux, int naux, int nao,
                      double *__restrict__ out, double ka, double kb, double omega, const double *__restrict__ boys)
{
    using K = WarpK<LA, LB, CM>;
    constexpr bool FS = CM & 1, FX = CM & 2, FY = CM & 4, FZ = CM & 8;
    constexpr int G = (FX || FY || FZ) ? 1 : 0;  // one more Hermite order for the p functions
    constexpr int L = LA + LB + G;
    constexpr int NCB = ncart(LB), NAB = K::NAB;
    constexpr int NT = LA + LB + 1, NE = (LA + 1) * (LB + 1) * NT;
    __shared__ double sE[K::WARPS][K::PPW][3 * NE];
    extern __shared__ double sacc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / K::TW, sl = lane % K::TW;
    const int ip0 = (blockIdx.x * K::WARPS + warp) * K::PPW;
    if (ip0 >= npair) return;  // whole warps leave: the kernel has no block-wide barrier
    const bool own = ip0 + sub < npair;
    const int ip = own ? ip0 + sub : npair - 1;
    const int ic = blockIdx.y * K::TW + sl;
    const bool store = own && ic < naux;
    // idle lanes compute on a valid pair and function and store nothing
    const AuxDev c = aux[ic < naux ? ic : naux - 1];
    const int2 pr = pairs[ip];
    const ShellDev A = sh[pr.x], B = sh[pr.y];
    double *E = sE[warp][sub];
    // the contraction re-reads the coefficients where it uses them (shared
    // memory reads are cheap here) rather than holding all of them in registers
    const volatile double *Ev = E;

    double racc[K::SACC ? 1 : K::NACC];
    double *wacc = sacc + (size_t)warp * K::NACC * 32 + lane;
    // running sum of function f (0..3) for Cartesian pair k
    auto acc = [&](int f, int k) -> double & {
        if constexpr (K::SACC)
            return wacc[(K::slot(f) * NAB + k) * 32];
        else
            return racc[K::slot(f) * NAB + k];
    };
#pragma unroll
    for (int f = 0; f < 4; ++f)
        if (CM & (1 << f))
#pragma unroll
            for (int k = 0; k < NAB; ++k) acc(f, k) = 0.0;

    const double ce = c.e, ice = 1.0 / ce;
    const double cpre = TWO_PI_52 * ice;
    const int2 rg = prange[ip];  // every kept shell pair has at least one primitive pair
    const int nq = own ? rg.y : 0;
    const int nqmax = __reduce_max_sync(0xffffffffu, nq);
    for (int it = 0; it < nqmax; ++it) {
        const bool live = it < nq;
        const double *pq = prim + 6LL * (rg.x + (live ? it : 0));
        const double Px = pq[0], Py = pq[1], Pz = pq[2], p = pq[3], ip_ = pq[4];
        const double Kab = live ? pq[5] : 0.0;  // a finished pair adds exact zeros
        __syncwarp();  // the previous primitive pair's coefficients are read by all lanes
        if (sl < 3) {
            const double Pd = sl == 0 ? Px : (sl == 1 ? Py : Pz);
            const double Ad = sl == 0 ? A.x : (sl == 1 ? A.y : A.z);
            const double Bd = sl == 0 ? B.x : (sl == 1 ? B.y : B.z);
            double Ed[LA + 1][LB + 1][NT];
            hermite_E<LA, LB>(Pd - Ad, Pd - Bd, 0.5 * ip_, Ed);
#pragma unroll
            for (int i = 0; i <= LA; ++i)
#pragma unroll
                for (int j = 0; j <= LB; ++j)
#pragma unroll
                    for (int t = 0; t <= i + j; ++t) E[sl * NE + (i * (LB + 1) + j) * NT + t] = Ed[i][j][t];
        }
        __syncwarp();
        const double u = 1.0 / (p + ce);
        const double rho = p * ce * u;
        const double X = Px - c.x, Y = Py - c.y, Z = Pz - c.z;
        double Rn[L + 1];
        coulomb_aux<L>(rho, rho * (X * X + Y * Y + Z * Z), ka, kb, omega, boys, Rn);
        const double pref = (Kab * ip_) * (cpre * sqrt(u));
#pragma unroll
        for (int n = 0; n <= L; ++n) Rn[n] *= pref;
        double R[L + 1][L + 1][L + 1];
        hermite_R<L>(X, Y, Z, Rn, R);

        // pass 0: the s, x and y functions from W(t,w) = sum_v ez_v R_{t,w,v};
        // pass 1: the z function from W(t,w) = sum_v ez_v R_{t,w,v+1}; one W
        // at a time is live
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 0 && !(FS || FX || FY)) continue;
            if (pass == 1 && !FZ) continue;
#pragma unroll
            for (int az = 0; az <= LA; ++az)
#pragma unroll
                for (int bz = 0; bz <= LB; ++bz) {
                    const int nz = az + bz;
                    double ez[NT];
#pragma unroll
                    for (int v = 0; v <= nz; ++v) ez[v] = Ev[2 * NE + (az * (LB + 1) + bz) * NT + v];
                    double W[L + 1][L + 1];
#pragma unroll
                    for (int t = 0; t <= L; ++t)
#pragma unroll
                        for (int w = 0; w <= L - t; ++w)
                            if (t + w + nz + pass <= L) {
                                double s = 0.0;
#pragma unroll
                                for (int v = 0; v <= nz; ++v)
                                    s = fma(ez[v], R[t][w][v + pass <= L ? v + pass : L], s);
                                W[t][w] = s;
                            }
#pragma unroll
                    for (int ay = 0; ay <= LA - az; ++ay)
#pragma unroll
                        for (int by = 0; by <= LB - bz; ++by) {
                            const int ny = ay + by;
                            const int ax = LA - ay - az, bx = LB - by - bz, nx = ax + bx;
                            const int k = cidx(LA, ax, ay) * NCB + cidx(LB, bx, by);
                            double ey[NT], ex[NT];
#pragma unroll
                            for (int w = 0; w <= ny; ++w) ey[w] = Ev[NE + (ay * (LB + 1) + by) * NT + w];
#pragma unroll
                            for (int t = 0; t <= nx; ++t) ex[t] = Ev[(ax * (LB + 1) + bx) * NT + t];
                            if (pass == 0) {
                                // Vs(t) = sum_w ey_w W(t,w), for t <= nx + 1 when the x
                                // function reads it one step on; Vy(t) = sum_w ey_w W(t,w+1)
                                double Vs[L + 1], Vy[L + 1];
#pragma unroll
                                for (int t = 0; t <= nx + (FX ? 1 : 0); ++t) {
                                    if (FS || FX) {
                                        double s = 0.0;
#pragma unroll
                                        for (int w = 0; w <= ny; ++w) s = fma(ey[w], W[t][w], s);
                                        Vs[t] = s;
                                    }
                                    if (FY && t <= nx) {
                                        double sy = 0.0;
#pragma unroll
                                        for (int w = 0; w <= ny; ++w)
                                            sy = fma(ey[w], W[t][w + 1 <= L ? w + 1 : L], sy);
                                        Vy[t] = sy;
                                    }
                                }
                                if (FS) {
                                    double s0 = acc(0, k);
#pragma unroll
                                    for (int t = 0; t <= nx; ++t) s0 = fma(ex[t], Vs[t], s0);
                                    acc(0, k) = s0;
                                }
                                if (FX) {
                                    double sx = acc(1, k);
#pragma unroll
                                    for (int t = 0; t <= nx; ++t) sx = fma(ex[t], Vs[t + 1 <= L ? t + 1 : L], sx);
                                    acc(1, k) = sx;
                                }
                                if (FY) {
                                    double sy = acc(2, k);
#pragma unroll
                                    for (int t = 0; t <= nx; ++t) sy = fma(ex[t], Vy[t], sy);
                                    acc(2, k) = sy;
                                }
                            } else {
                                double sz = acc(3, k);
#pragma unroll
                                for (int t = 0; t <= nx; ++t) {
                                    double s = 0.0;
#pragma unroll
                                    for (int w = 0; w <= ny; ++w) s = fma(ey[w], W[t][w], s);
                                    sz = fma(ex[t], s, sz);
                                }
                                acc(3, k) = sz;
                            }
                        }
                }
        }
    }
    if (!store) return;
    constexpr int NSA = 2 * LA + 1, NSB = 2 * LB + 1, NCA = ncart(LA);
    const double pfac = -0.5 * ice;  // p functions: 1/(2c) and the sign of the derivative on the ket
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (!(CM & (1 << f))) continue;
        double *o = out + (long long)(c.out + f) * nao * nao;
#pragma unroll
        for (int sa = 0; sa < NSA; ++sa) {
#pragma unroll
            for (int sb = 0; sb < NSB; ++sb) {
                double v = 0.0;
#pragma unroll
                for (int ka_ = 0; ka_ < NCA; ++ka_) {
                    const double wa = LA == 2 ? d_sph(sa, ka_) : (ka_ == sa ? 1.0 : 0.0);
                    if (wa == 0.0) continue;
#pragma unroll
                    for (int kb_ = 0; kb_ < NCB; ++kb_) {
                        const double wb = LB == 2 ? d_sph(sb, kb_) : (kb_ == sb ? 1.0 : 0.0);
                        if (wb == 0.0) continue;
                        v = fma(wa * wb, acc(f, ka_ * NCB + kb_), v);
                    }
                }
                if (f) v *= pfac;
                const int mu = A.ao + sa, nu = B.ao + sb;
                o[(long long)mu * nao + nu] = v;
                o[(long long)nu * nao + mu] = v;
            }
        }
    }
}

// Dipole integrals <mu| r - O |nu> of one AO shell pair per thread (Sec. 2, Eq.
// transition): per direction the first moment about O of the Hermite expansion,
//   M^{ij} = (E^{ij}_1 + (P - O) E^{ij}_0) sqrt(pi/p),
// the other two directions the overlaps E^{ij}_0 sqrt(pi/p); contracted over the
// pair's primitive pairs and written to both triangles of out[d][nao][nao].
template <int LA, int LB>
__global__ void __launch_bounds__(128)
    dipole_kernel(const ShellDev *__restrict__ sh, const int2 *__restrict__ pairs, const int2 *__restrict__ prange,
                  const double *__restrict__ prim, int npair, int nao, double Ox, double Oy, double Oz,
                  double *__restrict__ out)
{
    constexpr int NCA = ncart(LA), NCB = ncart(LB);
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npair) return;
    const int2 pr = pairs[ip];
    const ShellDev A = sh[pr.x], B = sh[pr.y];
    double acc[3][NCA][NCB];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int i = 0; i < NCA; ++i)
#pragma unroll
            for (int j = 0; j < NCB; ++j) acc[d][i][j] = 0.0;
    const int2 rg = prange[ip];
    for (int q = rg.x; q < rg.x + rg.y; ++q) {
        const double *pq = prim + 6LL * q;
        const double Px = pq[0], Py = pq[1], Pz = pq[2], ip_ = pq[4], Kab = pq[5];
        double Ex[LA + 1][LB + 1][LA + LB + 1], Ey[LA + 1][LB + 1][LA + LB + 1], Ez[LA + 1][LB + 1][LA + LB + 1];
        hermite_E<LA, LB>(Px - A.x, Px - B.x, 0.5 * ip_, Ex);
        hermite_E<LA, LB>(Py - A.y, Py - B.y, 0.5 * ip_, Ey);
        hermite_E<LA, LB>(Pz - A.z, Pz - B.z, 0.5 * ip_, Ez);
        const double norm = Kab * 5.568327996831707845 * ip_ * sqrt(ip_);  // K (pi/p)^{3/2}
#pragma unroll
        for (int ka_ = 0; ka_ < NCA; ++ka_)
#pragma unroll
            for (int kb_ = 0; kb_ < NCB; ++kb_) {
                const int ax = cexp(LA, ka_, 0), ay = cexp(LA, ka_, 1), az = cexp(LA, ka_, 2);
                const int bx = cexp(LB, kb_, 0), by = cexp(LB, kb_, 1), bz = cexp(LB, kb_, 2);
                const double sx = Ex[ax][bx][0], sy = Ey[ay][by][0], sz = Ez[az][bz][0];
                const double mx = (ax + bx > 0 ? Ex[ax][bx][ax + bx > 0 ? 1 : 0] : 0.0) + (Px - Ox) * sx;
                const double my = (ay + by > 0 ? Ey[ay][by][ay + by > 0 ? 1 : 0] : 0.0) + (Py - Oy) * sy;
                const double mz = (az + bz > 0 ? Ez[az][bz][az + bz > 0 ? 1 : 0] : 0.0) + (Pz - Oz) * sz;
                acc[0][ka_][kb_] = fma(norm, mx * sy * sz, acc[0][ka_][kb_]);
                acc[1][ka_][kb_] = fma(norm, sx * my * sz, acc[1][ka_][kb_]);
                acc[2][ka_][kb_] = fma(norm, sx * sy * mz, acc[2][ka_][kb_]);
            }
    }
    constexpr int NSA = 2 * LA + 1, NSB = 2 * LB + 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double *o = out + (long long)d * nao * nao;
#pragma unroll
        for (int sa = 0; sa < NSA; ++sa)
#pragma unroll
            for (int sb = 0; sb < NSB; ++sb) {
                double v = 0.0;
#pragma unroll
                for (int ka_ = 0; ka_ < NCA; ++ka_) {
                    const double wa = LA == 2 ? d_sph(sa, ka_) : (ka_ == sa ? 1.0 : 0.0);
                    if (wa == 0.0) continue;
#pragma unroll
                    for (int kb_ = 0; kb_ < NCB; ++kb_) {
                        const double wb = LB == 2 ? d_sph(sb, kb_) : (kb_ == sb ? 1.0 : 0.0);
                        if (wb == 0.0) continue;
                        v = fma(wa * wb, acc[d][ka_][kb_], v);
                    }
                }
                const int mu = A.ao + sa, nu = B.ao + sb;
                o[(long long)mu * nao + nu] = v;
                o[(long long)nu * nao + mu] = v;
            }
    }
}

template <int LA, int LB, int CM>
void launch_warp(Prof &prof, cudaStream_t st, const char *name, const ShellDev *sh, const int2 *pairs,
                 const int2 *prange, const double *prim, int npair, const AuxDev *aux, int naux, int nao, double *out,
                 double ka, double kb, double omega, const double *boys)
{
    using K = WarpK<LA, LB, CM>;
    static const cudaError_t attr =
        K::SMEM > 48 * 1024 ? cudaFuncSetAttribute(int3c_warp_kernel<LA, LB, CM>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM)
                            : cudaSuccess;
    TR_CUDA(attr);
    dim3 grid(cdiv(npair, K::WARPS * K::PPW), cdiv(naux, K::TW));
    double bytes = 8.0 * 2.0 * K::NF * npair * naux * (2 * LA + 1) * (2 * LB + 1);
    int tok = prof.begin(st, name, 0, bytes);
    int3c_warp_kernel<LA, LB, CM><<<grid, 32 * K::WARPS, K::SMEM, st>>>(sh, pairs, prange, prim, npair, aux, naux,
                                                                         nao, out, ka, kb, omega, boys);
    TR_CHECK_LAUNCH(name);
    prof.end(st, tok);
}

template <int LA, int LB>
void launch_pair_class(Prof &prof, const cudaStream_t *streams, int nstreams, int &next, int cls,
                       const ShellDev *sh, const int2 *pairs, const int2 *prange, const double *prim, int npair,
                       const AuxDev *aux, const int *aoff, const AuxDev *atoms, int natoms, int nao, double *out,
                       double ka, double kb, double omega, const double *boys)
{
    static const char *names[6] = {"int3c_ss", "int3c_ps", "int3c_pp", "int3c_ds", "int3c_dp", "int3c_dd"};
    if constexpr (LA + LB >= 2) {
        // classes whose Hermite coefficients are worth sharing across the
        // auxiliary functions: shell pairs by warps, auxiliary atoms (the whole
        // J atoms of a grouped chunk) or s functions by lanes.  A chunk of
        // fewer than one lane tile of them (large molecules, whose chunks hold
        // few functions) keeps the kernels with one lane per shell pair.
        if (npair <= 0) return;
        const int ns = aoff[1] - aoff[0];
        constexpr int TW = WarpK<LA, LB, 1>::TW;
        if (natoms >= TW) {
            if constexpr (LA == 2 && LB == 2) {
                // d-d: the s, p_x and the p_y, p_z functions in two launches, so
                // that a warp's sums leave room for more warps on an SM
                launch_warp<LA, LB, 3>(prof, streams[next++ % nstreams], names[cls], sh, pairs, prange, prim, npair,
                                       atoms, natoms, nao, out, ka, kb, omega, boys);
                launch_warp<LA, LB, 12>(prof, streams[next++ % nstreams], names[cls], sh, pairs, prange, prim, npair,
                                        atoms, natoms, nao, out, ka, kb, omega, boys);
            } else {
                launch_warp<LA, LB, 15>(prof, streams[next++ % nstreams], names[cls], sh, pairs, prange, prim, npair,
                                        atoms, natoms, nao, out, ka, kb, omega, boys);
            }
            return;
        }
        if (ns >= TW && aoff[4] == aoff[1]) {
            launch_warp<LA, LB, 1>(prof, streams[next++ % nstreams], names[cls], sh, pairs, prange, prim, npair,
                                   aux + aoff[0], ns, nao, out, ka, kb, omega, boys);
            return;
        }
    }
    if constexpr (ncart(LA) * ncart(LB) <= 18) {
    if (natoms > 0 && npair > 0) {
        // whole J atoms (s + p) in one pass: sums in registers for the light
        // classes, in shared memory for d-p (d-d runs per component: its Hermite
        // coefficients and R alone fill the registers)
        constexpr bool SACC = ncart(LA) * ncart(LB) > 9;
        constexpr int NT = SACC ? 64 : 128;
        constexpr size_t SMEM = SACC ? sizeof(double) * 4 * ncart(LA) * ncart(LB) * NT : 0;
        static const cudaError_t attr =
            SMEM > 48 * 1024 ? cudaFuncSetAttribute(int3c_grp_kernel<LA, LB, SACC>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM)
                             : cudaSuccess;
        TR_CUDA(attr);
        cudaStream_t st = streams[next++ % nstreams];
        dim3 grid(cdiv(npair, NT), natoms);
        double bytes = 8.0 * 2.0 * 4 * npair * natoms * (2 * LA + 1) * (2 * LB + 1);
        int tok = prof.begin(st, names[cls], 0, bytes);
        int3c_grp_kernel<LA, LB, SACC><<<grid, NT, SMEM, st>>>(sh, pairs, prange, prim, npair, atoms, nao, out, ka,
                                                                kb, omega, boys);
        TR_CHECK_LAUNCH(names[cls]);
        prof.end(st, tok);
        return;
    }
    }
    for (int cd = -1; cd <= 2; ++cd) {
        int n = aoff[cd + 2] - aoff[cd + 1];
        if (n <= 0 || npair <= 0) continue;
        cudaStream_t st = streams[next++ % nstreams];
        dim3 grid(cdiv(npair, 128), n);
        const AuxDev *a = aux + aoff[cd + 1];
        double bytes = 8.0 * 2.0 * npair * n * (2 * LA + 1) * (2 * LB + 1);
        int tok = prof.begin(st, names[cls], 0, bytes);
        // d-d: sums in shared memory (36 x 128 doubles)
        constexpr bool SACC = ncart(LA) * ncart(LB) > 18;
        constexpr size_t SMEM = SACC ? sizeof(double) * ncart(LA) * ncart(LB) * 128 : 0;
        switch (cd) {
            case -1: int3c_kernel<LA, LB, -1, SACC><<<grid, 128, SMEM, st>>>(sh, pairs, prange, prim, npair, a, nao, out, ka, kb, omega, boys); break;
            case 0: int3c_kernel<LA, LB, 0, SACC><<<grid, 128, SMEM, st>>>(sh, pairs, prange, prim, npair, a, nao, out, ka, kb, omega, boys); break;
            case 1: int3c_kernel<LA, LB, 1, SACC><<<grid, 128, SMEM, st>>>(sh, pairs, prange, prim, npair, a, nao, out, ka, kb, omega, boys); break;
            default: int3c_kernel<LA, LB, 2, SACC><<<grid, 128, SMEM, st>>>(sh, pairs, prange, prim, npair, a, nao, out, ka, kb, omega, boys); break;
        }
        TR_CHECK_LAUNCH(names[cls]);
        prof.end(st, tok);
    }
}

__global__ void int2c_kernel(const AuxDev *__restrict__ aux, int n, double ka, double kb, double omega,
                             const double *__restrict__ boys, double *__restrict__ out)
{
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const AuxDev P = aux[i], Q = aux[j];
    const double a = P.e, b = Q.e;
    const double rho = a * b / (a + b);
    const double d[3] = {P.x - Q.x, P.y - Q.y, P.z - Q.z};
    double Rn[3];
    coulomb_aux<2>(rho, rho * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), ka, kb, omega, boys, Rn);
    double v;
    if (P.comp < 0 && Q.comp < 0)
        v = Rn[0];
    else if (Q.comp < 0)
        v = (0.5 / a) * d[P.comp] * Rn[1];
    else if (P.comp < 0)
        v = -(0.5 / b) * d[Q.comp] * Rn[1];
    else
        v = -(0.25 / (a * b)) * ((P.comp == Q.comp ? Rn[1] : 0.0) + d[P.comp] * d[Q.comp] * Rn[2]);
    out[(long long)P.out * n + Q.out] = TWO_PI_52 / (a * b * sqrt(a + b)) * v;
}

}  // namespace

void int3c(Prof &prof, cudaStream_t st, SideStreams *side, const ShellDev *sh, const int2 *pairs,
           const int2 *prange, const double *prim, const int *off, const AuxDev *aux, const int *aoff,
           const AuxDev *atoms, int natoms, int nao, double *out, double ka, double kb, double omega,
           const double *boys)
{
    // the 6 pair classes x 4 aux components are independent launches writing
    // disjoint outputs: spread them over the side streams (heaviest classes first)
    cudaStream_t one[1] = {st};
    const cudaStream_t *streams = one;
    int nstreams = 1, next = 0;
    if (side) {
        side->begin(st);
        streams = side->s;
        nstreams = SideStreams::N;
    }
#define TR_CLASS(LA, LB, C)                                                                                        \
    launch_pair_class<LA, LB>(prof, streams, nstreams, next, C, sh, pairs + off[C], prange + off[C], prim,       \
                              off[C + 1] - off[C], aux, aoff, atoms, natoms, nao, out, ka, kb, omega, boys)
    TR_CLASS(2, 2, 5);
    TR_CLASS(2, 1, 4);
    TR_CLASS(1, 1, 2);
    TR_CLASS(2, 0, 3);
    TR_CLASS(1, 0, 1);
    TR_CLASS(0, 0, 0);
#undef TR_CLASS
    if (side) side->end(st);
}

void dipole_ints(Prof &prof, cudaStream_t st, const ShellDev *sh, const int2 *pairs, const int2 *prange,
                 const double *prim, const int *off, int nao, const double O[3], double *out)
{
    TR_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 3 * (size_t)nao * nao, st));
#define TR_DIP(LA, LB, C)                                                                                          \
    if (off[C + 1] > off[C]) {                                                                                     \
        const int n = off[C + 1] - off[C];                                                                         \
        TR_LAUNCH(prof, st, "dipole", 0, 0,                                                                        \
                  dipole_kernel<LA, LB><<<cdiv(n, 128), 128, 0, st>>>(sh, pairs + off[C], prange + off[C], prim, n, \
                                                                      nao, O[0], O[1], O[2], out));                \
    }
    TR_DIP(0, 0, 0);
    TR_DIP(1, 0, 1);
    TR_DIP(1, 1, 2);
    TR_DIP(2, 0, 3);
    TR_DIP(2, 1, 4);
    TR_DIP(2, 2, 5);
#undef TR_DIP
}

void int2c(Prof &prof, cudaStream_t st, const AuxDev *aux, int n, double ka, double kb, double omega,
           const double *boys, double *out)
{
    if (n <= 0) return;
    TR_LAUNCH(prof, st, "int2c", 0, 8.0 * n * n,
              int2c_kernel<<<dim3(cdiv(n, 128), n), 128, 0, st>>>(aux, n, ka, kb, omega, boys, out));
}

}  // namespace tr
