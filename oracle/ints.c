/*
 * CPU oracle for the TDA-risp integrals -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU baseline leg of the benchmark
 * call this code; the product path never links it.  It shares no code with
 * the CUDA library.
 *
 * What it computes (plain FP64, no screening, no blocking):
 *   (P|mu nu)  three-centre two-electron integrals of an auxiliary primitive P
 *              (l = 0 or 1, coefficient 1, unnormalised) with a pair of
 *              contracted spherical AO functions, for the operator
 *              (alpha + beta erf(omega r12)) / r12                (Sec. 2, Eq. RI;
 *              Sec. 3.2, Eqs. RSH and K_mia_RSH),
 *   (P|Q)      the two-centre metric for the same operator         (Sec. 2, Eq. RI),
 *   <mu|r - O|nu>  dipole integrals of the AO functions, for the electric
 *              transition dipoles of the oscillator strengths (Sec. 2,
 *              Eqs. oscillator_strength and transition).
 *
 * Method: Obara-Saika vertical recursion (electron 1 then electron 2) on the
 * Boys-type auxiliary functions G_m, followed by the horizontal recursion
 * that moves angular momentum from centre A to centre B.  For the operator
 * (alpha + beta erf(omega r))/r the auxiliary function is
 *     G_m(rho, T) = alpha F_m(T) + beta s^(m+1/2) F_m(s T),  s = omega^2/(omega^2+rho),
 * and the recursions are those of the Coulomb operator.  F_m is the Boys
 * function, evaluated in long double by its positive power series (small T)
 * or by erf and upward recursion (large T).
 *
 * Data conventions: AO function = sum_k c_k Y(r-A) exp(-a_k |r-A|^2) with
 * the coefficients taken literally; Y = 1 (s); x, y, z (p); for d the real
 * solid harmonics xy, yz, (2zz-xx-yy)/(2 sqrt3), xz, (xx-yy)/2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EMAX 4   /* sum of the two AO angular momenta */
#define FMAX 2   /* auxiliary angular momentum */
#define MMAX (EMAX + FMAX)

/* ---------------------------------------------------------------- Boys */

void orc_boys(int mmax, double T, double *F)
{
    long double t = (long double)T, Fl[MMAX + 8];
    if (mmax > MMAX + 7) mmax = MMAX + 7;
    if (t < 60.0L) {
        /* F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) */
        long double term = 1.0L / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 4000; ++k) {
            term *= 2.0L * t / (2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-24L * sum) break;
        }
        long double e = expl(-t);
        Fl[mmax] = e * sum;
        for (int m = mmax - 1; m >= 0; --m) Fl[m] = (2.0L * t * Fl[m + 1] + e) / (2 * m + 1);
    } else {
        long double e = expl(-t);
        Fl[0] = 0.5L * sqrtl(3.14159265358979323846264338327950288L / t) * erfl(sqrtl(t));
        for (int m = 0; m < mmax; ++m) Fl[m + 1] = ((2 * m + 1) * Fl[m] - e) / (2.0L * t);
    }
    for (int m = 0; m <= mmax; ++m) F[m] = (double)Fl[m];
}

/* G_m for (alpha + beta erf(omega r))/r */
static void kernel_g(int mmax, double rho, double T, double ka, double kb, double omega, double *G)
{
    double F[MMAX + 8];
    for (int m = 0; m <= mmax; ++m) G[m] = 0.0;
    if (ka != 0.0) {
        orc_boys(mmax, T, F);
        for (int m = 0; m <= mmax; ++m) G[m] += ka * F[m];
    }
    if (kb != 0.0 && omega > 0.0) {
        double s = omega * omega / (omega * omega + rho);
        orc_boys(mmax, s * T, F);
        double f = sqrt(s);
        for (int m = 0; m <= mmax; ++m) {
            G[m] += kb * f * F[m];
            f *= s;
        }
    }
}

/* ---------------------------------------------------------------- OS VRR */

typedef struct {
    double PA[3], WP[3], WQ[3];
    double zeta, eta, rho;
    double base[MMAX + 1];
    double memo[EMAX + 1][EMAX + 1][EMAX + 1][FMAX + 1][FMAX + 1][FMAX + 1][MMAX + 1];
    uint32_t stamp[EMAX + 1][EMAX + 1][EMAX + 1][FMAX + 1][FMAX + 1][FMAX + 1][MMAX + 1];
    uint32_t cur;
} vrr_ctx;

/* [e 0 | f 0]^(m); the ket is the auxiliary primitive times a zero-exponent
 * s function on the same centre, so Q = C and the QC terms vanish. */
static double vrr(vrr_ctx *v, const int e[3], const int f[3], int m)
{
    if (e[0] < 0 || e[1] < 0 || e[2] < 0 || f[0] < 0 || f[1] < 0 || f[2] < 0) return 0.0;
    if (v->stamp[e[0]][e[1]][e[2]][f[0]][f[1]][f[2]][m] == v->cur)
        return v->memo[e[0]][e[1]][e[2]][f[0]][f[1]][f[2]][m];
    double val;
    if (e[0] + e[1] + e[2] + f[0] + f[1] + f[2] == 0) {
        val = v->base[m];
    } else if (f[0] + f[1] + f[2] > 0) {
        int i = f[0] > 0 ? 0 : (f[1] > 0 ? 1 : 2);
        int f1[3] = {f[0], f[1], f[2]};
        f1[i] -= 1;
        int f2[3] = {f1[0], f1[1], f1[2]};
        f2[i] -= 1;
        int e1[3] = {e[0], e[1], e[2]};
        e1[i] -= 1;
        val = v->WQ[i] * vrr(v, e, f1, m + 1);
        if (f1[i] > 0)
            val += f1[i] / (2.0 * v->eta) * (vrr(v, e, f2, m) - v->rho / v->eta * vrr(v, e, f2, m + 1));
        if (e[i] > 0) val += e[i] / (2.0 * (v->zeta + v->eta)) * vrr(v, e1, f1, m + 1);
    } else {
        int i = e[0] > 0 ? 0 : (e[1] > 0 ? 1 : 2);
        int e1[3] = {e[0], e[1], e[2]};
        e1[i] -= 1;
        int e2[3] = {e1[0], e1[1], e1[2]};
        e2[i] -= 1;
        val = v->PA[i] * vrr(v, e1, f, m) + v->WP[i] * vrr(v, e1, f, m + 1);
        if (e1[i] > 0)
            val += e1[i] / (2.0 * v->zeta) * (vrr(v, e2, f, m) - v->rho / v->zeta * vrr(v, e2, f, m + 1));
    }
    v->stamp[e[0]][e[1]][e[2]][f[0]][f[1]][f[2]][m] = v->cur;
    v->memo[e[0]][e[1]][e[2]][f[0]][f[1]][f[2]][m] = val;
    return val;
}

/* ---------------------------------------------------------------- angular tables */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }
static int nsph(int l) { return 2 * l + 1; }

/* Cartesian components in the order used below: l=1 x,y,z; l=2 xx,xy,xz,yy,yz,zz */
static void cart_exps(int l, int k, int out[3])
{
    static const int c0[1][3] = {{0, 0, 0}};
    static const int c1[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int c2[6][3] = {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
    const int *r = l == 0 ? c0[k] : (l == 1 ? c1[k] : c2[k]);
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
}

/* spherical function s of shell l as a combination of Cartesian components */
static double sph_coef(int l, int s, int k)
{
    if (l < 2) return s == k ? 1.0 : 0.0;
    const double r3 = 1.0 / sqrt(3.0);
    static double tab[5][6];
    static int init = 0;
    if (!init) {
        memset(tab, 0, sizeof tab);
        tab[0][1] = 1.0;                 /* xy */
        tab[1][4] = 1.0;                 /* yz */
        tab[2][5] = r3;                  /* (2zz - xx - yy)/(2 sqrt3) */
        tab[2][0] = -0.5 * r3;
        tab[2][3] = -0.5 * r3;
        tab[3][2] = 1.0;                 /* xz */
        tab[4][0] = 0.5;                 /* (xx - yy)/2 */
        tab[4][3] = -0.5;
        init = 1;
    }
    return tab[s][k];
}

/* ---------------------------------------------------------------- shell triple */

typedef struct {
    double A[3], B[3], C[3];
    int la, lb, lc;
    int na, nb;                  /* primitives on A and B */
    const double *ea, *ca, *eb, *cb;
    double ec;                   /* auxiliary exponent (one primitive, coefficient 1) */
    double ka, kb, omega;
} triple;

/* contracted [e 0 | f] with la <= |e| <= la+lb, indexed [ex][ey][ez][fx][fy][fz] */
typedef struct {
    double v[EMAX + 1][EMAX + 1][EMAX + 1][FMAX + 1][FMAX + 1][FMAX + 1];
} etab;

static double hrr(const etab *t, const double AB[3], const int a[3], const int b[3], const int f[3])
{
    if (b[0] + b[1] + b[2] == 0) return t->v[a[0]][a[1]][a[2]][f[0]][f[1]][f[2]];
    int i = b[0] > 0 ? 0 : (b[1] > 0 ? 1 : 2);
    int b1[3] = {b[0], b[1], b[2]};
    b1[i] -= 1;
    int a1[3] = {a[0], a[1], a[2]};
    a1[i] += 1;
    /* (a, b+1_i | = (a+1_i, b | + AB_i (a, b | */
    return hrr(t, AB, a1, b1, f) + AB[i] * hrr(t, AB, a, b1, f);
}

/* out[c][sa][sb] for the spherical components of the triple; c runs over the
 * Cartesian components of the auxiliary shell (identical to spherical for l<=1). */
static void triple_integrals(const triple *q, vrr_ctx *v, etab *et, double *out)
{
    const double PI = 3.14159265358979323846;
    int L = q->la + q->lb + q->lc;
    memset(et, 0, sizeof *et);
    double AB[3], AB2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        AB[d] = q->A[d] - q->B[d];
        AB2 += AB[d] * AB[d];
    }
    int nfc = ncart(q->lc);
    for (int i = 0; i < q->na; ++i) {
        for (int j = 0; j < q->nb; ++j) {
            double a = q->ea[i], b = q->eb[j], c = q->ec;
            double zeta = a + b, eta = c;
            double P[3], W[3];
            for (int d = 0; d < 3; ++d) P[d] = (a * q->A[d] + b * q->B[d]) / zeta;
            double rho = zeta * eta / (zeta + eta);
            double PQ2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                W[d] = (zeta * P[d] + eta * q->C[d]) / (zeta + eta);
                PQ2 += (P[d] - q->C[d]) * (P[d] - q->C[d]);
                v->PA[d] = P[d] - q->A[d];
                v->WP[d] = W[d] - P[d];
                v->WQ[d] = W[d] - q->C[d];
            }
            v->zeta = zeta;
            v->eta = eta;
            v->rho = rho;
            double Kab = exp(-a * b / zeta * AB2);
            double pref = 2.0 * pow(PI, 2.5) / (zeta * eta * sqrt(zeta + eta)) * Kab;
            double G[MMAX + 1];
            kernel_g(L, rho, rho * PQ2, q->ka, q->kb, q->omega, G);
            for (int m = 0; m <= L; ++m) v->base[m] = pref * G[m];
            v->cur += 1;
            double w = q->ca[i] * q->cb[j];
            for (int le = q->la; le <= q->la + q->lb; ++le)
                for (int ex = 0; ex <= le; ++ex)
                    for (int ey = 0; ey <= le - ex; ++ey) {
                        int e[3] = {ex, ey, le - ex - ey};
                        for (int k = 0; k < nfc; ++k) {
                            int f[3];
                            cart_exps(q->lc, k, f);
                            et->v[e[0]][e[1]][e[2]][f[0]][f[1]][f[2]] += w * vrr(v, e, f, 0);
                        }
                    }
        }
    }
    int nca = ncart(q->la), ncb = ncart(q->lb);
    int nsa = nsph(q->la), nsb = nsph(q->lb);
    double cart[6][6];
    for (int k = 0; k < nfc; ++k) {
        int f[3];
        cart_exps(q->lc, k, f);
        for (int x = 0; x < nca; ++x)
            for (int y = 0; y < ncb; ++y) {
                int ea[3], eb[3];
                cart_exps(q->la, x, ea);
                cart_exps(q->lb, y, eb);
                cart[x][y] = hrr(et, AB, ea, eb, f);
            }
        for (int sa = 0; sa < nsa; ++sa)
            for (int sb = 0; sb < nsb; ++sb) {
                double s = 0.0;
                for (int x = 0; x < nca; ++x)
                    for (int y = 0; y < ncb; ++y)
                        s += sph_coef(q->la, sa, x) * sph_coef(q->lb, sb, y) * cart[x][y];
                out[(k * nsa + sa) * nsb + sb] = s;
            }
    }
}

/* ---------------------------------------------------------------- public entry points */

typedef struct {
    int nsh;
    const double *xyz;   /* nsh*3 centre of each shell */
    const int *l;        /* nsh */
    const int *nprim;    /* nsh */
    const int *pstart;   /* nsh, offset into exps/coefs */
    const double *exps, *coefs;
} basis_view;

static int basis_nfunc(const int *l, int n, int *off)
{
    int s = 0;
    for (int i = 0; i < n; ++i) {
        off[i] = s;
        s += nsph(l[i]);
    }
    return s;
}

/* Three-centre integrals: out[P][mu][nu] (full square, row-major), with P over
 * the functions of the auxiliary shells (1 for s, 3 for p in x,y,z order). */
int orc_int3c(int nsh, const double *sh_xyz, const int *sh_l, const int *sh_nprim,
              const int *sh_pstart, const double *exps, const double *coefs,
              int naux, const double *aux_xyz, const int *aux_l, const double *aux_exp,
              double ka, double kb, double omega, double *out)
{
    for (int i = 0; i < nsh; ++i)
        if (sh_l[i] < 0 || sh_l[i] > 2) return -1;
    for (int i = 0; i < naux; ++i)
        if (aux_l[i] < 0 || aux_l[i] > 1) return -1;
    int *off = malloc(sizeof(int) * (nsh + 1));
    int *aoff = malloc(sizeof(int) * (naux + 1));
    int nao = basis_nfunc(sh_l, nsh, off);
    (void)basis_nfunc(aux_l, naux, aoff);
    long npair = (long)nsh * nsh;
#pragma omp parallel
    {
        vrr_ctx *v = calloc(1, sizeof(vrr_ctx));
        etab *et = malloc(sizeof(etab));
        double blk[3 * 5 * 5];
#pragma omp for schedule(dynamic, 4)
        for (long pq = 0; pq < npair; ++pq) {
            int i = (int)(pq / nsh), j = (int)(pq % nsh);
            if (j > i) continue;
            for (int k = 0; k < naux; ++k) {
                triple q;
                memcpy(q.A, sh_xyz + 3 * i, sizeof q.A);
                memcpy(q.B, sh_xyz + 3 * j, sizeof q.B);
                memcpy(q.C, aux_xyz + 3 * k, sizeof q.C);
                q.la = sh_l[i];
                q.lb = sh_l[j];
                q.lc = aux_l[k];
                q.na = sh_nprim[i];
                q.nb = sh_nprim[j];
                q.ea = exps + sh_pstart[i];
                q.ca = coefs + sh_pstart[i];
                q.eb = exps + sh_pstart[j];
                q.cb = coefs + sh_pstart[j];
                q.ec = aux_exp[k];
                q.ka = ka;
                q.kb = kb;
                q.omega = omega;
                triple_integrals(&q, v, et, blk);
                int nsa = nsph(q.la), nsb = nsph(q.lb), nc = ncart(q.lc);
                for (int c = 0; c < nc; ++c)
                    for (int sa = 0; sa < nsa; ++sa)
                        for (int sb = 0; sb < nsb; ++sb) {
                            double x = blk[(c * nsa + sa) * nsb + sb];
                            long P = aoff[k] + c;
                            out[(P * nao + off[i] + sa) * nao + off[j] + sb] = x;
                            out[(P * nao + off[j] + sb) * nao + off[i] + sa] = x;
                        }
            }
        }
        free(v);
        free(et);
    }
    free(off);
    free(aoff);
    return 0;
}

/* One block of three-centre integrals for AO shells i, j and auxiliary shell k:
 * out[c][sa][sb]. */
int orc_int3c_block(const double *A, int la, int na, const double *ea, const double *ca,
                    const double *B, int lb, int nb, const double *eb, const double *cb,
                    const double *C, int lc, double ec,
                    double ka, double kb, double omega, double *out)
{
    if (la < 0 || la > 2 || lb < 0 || lb > 2 || lc < 0 || lc > 1) return -1;
    triple q;
    memcpy(q.A, A, sizeof q.A);
    memcpy(q.B, B, sizeof q.B);
    memcpy(q.C, C, sizeof q.C);
    q.la = la;
    q.lb = lb;
    q.lc = lc;
    q.na = na;
    q.nb = nb;
    q.ea = ea;
    q.ca = ca;
    q.eb = eb;
    q.cb = cb;
    q.ec = ec;
    q.ka = ka;
    q.kb = kb;
    q.omega = omega;
    vrr_ctx *v = calloc(1, sizeof(vrr_ctx));
    etab *et = malloc(sizeof(etab));
    triple_integrals(&q, v, et, out);
    free(v);
    free(et);
    return 0;
}

/* Two-centre metric out[P][Q] over auxiliary functions: the bra pair is the
 * auxiliary primitive P times a zero-exponent s function on its own centre. */
int orc_int2c(int naux, const double *aux_xyz, const int *aux_l, const double *aux_exp,
              double ka, double kb, double omega, double *out)
{
    for (int i = 0; i < naux; ++i)
        if (aux_l[i] < 0 || aux_l[i] > 1) return -1;
    int *aoff = malloc(sizeof(int) * (naux + 1));
    int n = basis_nfunc(aux_l, naux, aoff);
    const double one = 1.0, zero = 0.0;
#pragma omp parallel
    {
        vrr_ctx *v = calloc(1, sizeof(vrr_ctx));
        etab *et = malloc(sizeof(etab));
        double blk[3 * 3];
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < naux; ++i)
            for (int k = 0; k < naux; ++k) {
                triple q;
                memcpy(q.A, aux_xyz + 3 * i, sizeof q.A);
                memcpy(q.B, aux_xyz + 3 * i, sizeof q.B);
                memcpy(q.C, aux_xyz + 3 * k, sizeof q.C);
                q.la = aux_l[i];
                q.lb = 0;
                q.lc = aux_l[k];
                q.na = 1;
                q.nb = 1;
                q.ea = aux_exp + i;
                q.ca = &one;
                q.eb = &zero;
                q.cb = &one;
                q.ec = aux_exp[k];
                q.ka = ka;
                q.kb = kb;
                q.omega = omega;
                triple_integrals(&q, v, et, blk);
                int nsa = nsph(q.la), nc = ncart(q.lc);
                for (int c = 0; c < nc; ++c)
                    for (int sa = 0; sa < nsa; ++sa)
                        out[(long)(aoff[i] + sa) * n + aoff[k] + c] = blk[c * nsa + sa];
            }
        free(v);
        free(et);
    }
    free(aoff);
    return 0;
}

/* ---------------------------------------------------------------- dipole integrals
 *
 * Obara-Saika recursion of the one-dimensional overlap of two Cartesian
 * Gaussian factors (exponents a at A, b at B; p = a + b, P = (aA + bB)/p):
 *   S(0,0)   = sqrt(pi/p) exp(-ab/p (A-B)^2)
 *   S(i+1,j) = (P-A) S(i,j) + (i S(i-1,j) + j S(i,j-1)) / (2p)
 *   S(i,j+1) = (P-B) S(i,j) + (i S(i-1,j) + j S(i,j-1)) / (2p)
 * and the first moment about O, x - O = (x - B) + (B - O):
 *   M(i,j) = S(i,j+1) + (B-O) S(i,j).
 * A three-dimensional integral is the product of the three directions, with
 * the moment in the direction of the dipole component. */
#define OS_MAX 4
static void os_overlap(double a, double b, double A, double B, double S[OS_MAX][OS_MAX])
{
    const double p = a + b, P = (a * A + b * B) / p, PA = P - A, PB = P - B, h = 0.5 / p;
    double T[OS_MAX][OS_MAX];
    memset(T, 0, sizeof T);
    T[0][0] = sqrt(M_PI / p) * exp(-a * b / p * (A - B) * (A - B));
    /* first the i direction with j = 0, then raise j for every i */
    for (int i = 0; i + 1 < OS_MAX; ++i) T[i + 1][0] = PA * T[i][0] + (i > 0 ? i * h * T[i - 1][0] : 0.0);
    for (int j = 0; j + 1 < OS_MAX; ++j)
        for (int i = 0; i < OS_MAX; ++i)
            T[i][j + 1] = PB * T[i][j] + h * ((i > 0 ? i * T[i - 1][j] : 0.0) + (j > 0 ? j * T[i][j - 1] : 0.0));
    memcpy(S, T, sizeof T);
}

/* out[d][mu][nu] = <mu| r_d - O_d |nu>, d = x, y, z, for the contracted
 * spherical AO functions of the shells (full square, row-major). */
int orc_dipole(int nsh, const double *sh_xyz, const int *sh_l, const int *sh_nprim, const int *sh_pstart,
               const double *exps, const double *coefs, const double *O, double *out)
{
    for (int i = 0; i < nsh; ++i)
        if (sh_l[i] < 0 || sh_l[i] > 2) return -1;
    int *off = malloc(sizeof(int) * (nsh + 1));
    int nao = basis_nfunc(sh_l, nsh, off);
    for (int i = 0; i < nsh; ++i)
        for (int j = 0; j < nsh; ++j) {
            const int la = sh_l[i], lb = sh_l[j];
            const double *A = sh_xyz + 3 * i, *B = sh_xyz + 3 * j;
            double cart[3][6][6];
            memset(cart, 0, sizeof cart);
            for (int u = 0; u < sh_nprim[i]; ++u)
                for (int w = 0; w < sh_nprim[j]; ++w) {
                    const double a = exps[sh_pstart[i] + u], b = exps[sh_pstart[j] + w];
                    const double cc = coefs[sh_pstart[i] + u] * coefs[sh_pstart[j] + w];
                    double S[3][OS_MAX][OS_MAX];
                    for (int d = 0; d < 3; ++d) os_overlap(a, b, A[d], B[d], S[d]);
                    for (int ka = 0; ka < ncart(la); ++ka)
                        for (int kb = 0; kb < ncart(lb); ++kb) {
                            int ea[3], eb[3];
                            cart_exps(la, ka, ea);
                            cart_exps(lb, kb, eb);
                            for (int d = 0; d < 3; ++d) {
                                double v = cc;
                                for (int e = 0; e < 3; ++e) {
                                    if (e == d)
                                        v *= S[e][ea[e]][eb[e] + 1] + (B[e] - O[e]) * S[e][ea[e]][eb[e]];
                                    else
                                        v *= S[e][ea[e]][eb[e]];
                                }
                                cart[d][ka][kb] += v;
                            }
                        }
                }
            for (int d = 0; d < 3; ++d)
                for (int sa = 0; sa < nsph(la); ++sa)
                    for (int sb = 0; sb < nsph(lb); ++sb) {
                        double v = 0.0;
                        for (int ka = 0; ka < ncart(la); ++ka)
                            for (int kb = 0; kb < ncart(lb); ++kb)
                                v += sph_coef(la, sa, ka) * sph_coef(lb, sb, kb) * cart[d][ka][kb];
                        out[((long)d * nao + off[i] + sa) * nao + off[j] + sb] = v;
                    }
        }
    free(off);
    return 0;
}
