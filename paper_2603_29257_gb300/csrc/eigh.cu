// Lowest eigenpairs of a small dense symmetric FP64 matrix (the Davidson
// subspace matrix, Sec. 3.3) in one thread-block cluster.
//
//  1. Householder reduction to tridiagonal form T = Q^T A Q.  The rows of A
//     are dealt cyclically to the CTAs of the cluster; at step j every CTA
//     reads row j (final after the previous step), forms the reflector
//     H_j = I - tau v v^T (v_0 = 1) that zeroes A[j][j+2:], computes
//     p = tau A22 v for its own rows, and after a cluster barrier (for the
//     partial sums p^T v and the whole p) applies the symmetric rank-2 update
//     A22 -= v w^T + w v^T, w = p - (tau/2)(p^T v) v, to its own rows; a
//     second barrier ends the step.
//  2. Each of the lowest nev eigenvalues of T by 32-way multisection on a
//     warp: lane l counts the eigenvalues of T below x_l with the Sturm
//     sequence of leading principal minors p_r = (d_r - x) p_{r-1}
//     - e_{r-1}^2 p_{r-2} (sign changes = eigenvalues below x), rescaled by
//     powers of two to stay in range (FMA only, no division; the sign, zero
//     and range tests work on the bit pattern, since FP64 instructions are
//     the scarce resource on this GPU).
//  3. Eigenvectors of T by inverse iteration (Gaussian elimination with
//     partial pivoting of T - lambda I, two solves from a fixed
//     pseudo-random start); eigenvalues closer than 1e-6 |T| form a group
//     whose vectors are orthogonalised against each other (modified
//     Gram-Schmidt) after every solve, and equal eigenvalues are shifted
//     apart by a few ulps of |T| as the inverse iteration needs.
//     The returned eigenvalue is the Rayleigh quotient of the computed vector.
//  4. Back-transformation z = H_0 H_1 ... H_{k-3} y with the stored reflectors.
//
// Global scratch (L2-resident for the sizes used) carries the matrix, the
// reflectors and the small vectors; the cluster barrier orders the writes of
// one CTA before the reads of the others (those reads bypass L1).
#include "linalg.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

namespace tr {
namespace {

namespace cg = cooperative_groups;

constexpr int EIG_THREADS = 512;
constexpr int EIG_WARPS = EIG_THREADS / 32;

struct EigArgs {
    double *A;      // k x k, destroyed
    int k, nev;
    double *w;      // nev eigenvalues, ascending
    double *Y;      // Y[r * ldy + i] = component r of eigenvector i (i < nev)
    int ldy;
    double *Vh;     // k x k: row j holds v_j at columns j+1 .. k-1
    double *tau;    // k
    double *d, *e;  // tridiagonal: k diagonal, k-1 off-diagonal
    double *P;      // k
    double *red;    // 16 partial sums
    double *lam;    // nev
    double *ws;     // nev x 6k: inverse-iteration factors and vectors
    int slots_in_smem;  // inverse-iteration work arrays in shared memory
    int rows_in_smem;   // each CTA's rows of A in shared memory during the reduction
    int *flag;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Number of eigenvalues of T below x: sign changes of the leading principal
// minors p_r = (d_r - x) p_{r-1} - e_{r-1}^2 p_{r-2}.  e2s[r] = e_{r-1}^2
// (e2s[0] = 0).  Three FP64 operations per step; signs, exact zeros and the
// power-of-two rescaling that keeps p in range are decided on the bit pattern.
// An exact zero minor counts as negative (its ratio to the previous one is
// taken as -2^-100).
__device__ int sturm_count(const double *__restrict__ d, const double *__restrict__ e2s, int k, double x)
{
    double pm1 = 1.0, pm2 = 0.0;
    long long bprev = 0;  // sign bit of p_{-1} = +1
    int cnt = 0;
    for (int r = 0; r < k; ++r) {
        double p = fma(d[r] - x, pm1, -e2s[r] * pm2);
        long long b = __double_as_longlong(p);
        if ((b << 1) == 0) {
            p = -pm1 * 0x1p-100;
            b = __double_as_longlong(p);
        }
        cnt += (int)((unsigned long long)(b ^ bprev) >> 63);
        bprev = b;
        pm2 = pm1;
        pm1 = p;
        const int ex = (int)((b >> 52) & 0x7FF);
        if (ex > 1023 + 400 || ex < 1023 - 400) {
            // multiply both carried minors by 2^(1023 - ex): p returns to [1, 2)
            const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
            pm1 *= sc;
            pm2 *= sc;
        }
    }
    return cnt;
}

// deterministic start vector entry in [-1, 1)
__device__ __forceinline__ double start_entry(int i, int r)
{
    unsigned h = (unsigned)(i * 0x9E3779B9u) ^ (unsigned)(r * 0x85EBCA6Bu) ^ 0x27D4EB2Fu;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    return (double)(h & 0xFFFFFF) * (2.0 / 16777216.0) - 1.0;
}

constexpr int EIG_SLOTS = 4;  // warps per CTA that run inverse iteration / back-transformation

__global__ void __launch_bounds__(EIG_THREADS, 1) eigh_cluster_kernel(const EigArgs g)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = g.k, nev = g.nev;
    extern __shared__ double sm[];
    // shared: v[k] w[k] d[k] e2s[k] | 64 scalars | pl[k] | region: this CTA's rows of
    // A during the reduction (when they fit), later the inverse-iteration slots
    double *v = sm, *wv = sm + k, *sd = sm + 2 * k, *se2 = sm + 3 * k, *sc = sm + 4 * k, *pl = sm + 4 * k + 64;
    double *region = sm + 5 * k + 64;
    double *slots = g.slots_in_smem ? region : nullptr;
    double *A = g.A;

    if (g.rows_in_smem) {
        // ---- 1'. Householder tridiagonalisation with the rows in shared memory: the
        // pivot row, the entries of p and the partial sums are read from the owning
        // CTA's shared memory across the cluster
        double *rows = region;
        const int nown = (k - c + C - 1) / C;  // rows c, c + C, ...
        for (long long t = tid; t < (long long)nown * k; t += EIG_THREADS) {
            const int ii = (int)(t / k), col = (int)(t - (long long)ii * k);
            rows[t] = A[(long long)(c + ii * C) * k + col];
        }
        cl.sync();
        for (int j = 0; j + 2 < k; ++j) {
            const int m = k - j - 1;
            const double *prow = cl.map_shared_rank(rows, j % C) + (long long)(j / C) * k;
            for (int l = tid; l < m; l += EIG_THREADS) v[l] = prow[j + 1 + l];
            __syncthreads();
            if (warp == 0) {
                double s2 = 0.0;
                for (int l = 1 + lane; l < m; l += 32) s2 = fma(v[l], v[l], s2);
                s2 = warp_sum(s2);
                if (lane == 0) {
                    const double x0 = v[0];
                    double tau = 0.0, beta = x0, scl = 1.0;
                    if (s2 > 0.0) {
                        const double xn = sqrt(fma(x0, x0, s2));
                        beta = x0 >= 0.0 ? -xn : xn;
                        tau = (beta - x0) / beta;
                        scl = 1.0 / (x0 - beta);
                    }
                    sc[0] = tau;
                    sc[1] = scl;
                    if (c == 0) {
                        g.d[j] = prow[j];
                        g.e[j] = beta;
                        g.tau[j] = tau;
                    }
                }
            }
            __syncthreads();
            const double tau = sc[0], scl = sc[1];
            if (tau == 0.0) {
                cl.sync();
                continue;
            }
            for (int l = 1 + tid; l < m; l += EIG_THREADS) v[l] *= scl;
            if (tid == 0) v[0] = 1.0;
            __syncthreads();
            if (c == 0) {
                double *vh = g.Vh + (long long)j * k + j + 1;
                for (int l = tid; l < m; l += EIG_THREADS) vh[l] = v[l];
            }
            const int i0 = j + 1 + ((c - (j + 1)) % C + C) % C;
            double part = 0.0;
            for (int i = i0 + warp * C; i < k; i += EIG_WARPS * C) {
                const double *ri = rows + (long long)((i - c) / C) * k + j + 1;
                double dot = 0.0;
                for (int l = lane; l < m; l += 32) dot = fma(ri[l], v[l], dot);
                dot = warp_sum(dot) * tau;
                if (lane == 0) {
                    pl[i] = dot;
                    part = fma(dot, v[i - j - 1], part);
                }
            }
            if (lane == 0) sc[8 + warp] = part;
            __syncthreads();
            if (warp == 0) {
                const double t = warp_sum(lane < EIG_WARPS ? sc[8 + lane] : 0.0);
                if (lane == 0) sc[5] = t;
            }
            cl.sync();
            if (warp == 0) {
                const double pv = warp_sum(lane < C ? *cl.map_shared_rank(sc + 5, lane) : 0.0);
                if (lane == 0) sc[2] = 0.5 * tau * pv;
            }
            __syncthreads();
            const double K = sc[2];
            for (int l = tid; l < m; l += EIG_THREADS) {
                const int i = j + 1 + l;
                wv[l] = fma(-K, v[l], *cl.map_shared_rank(pl + i, i % C));
            }
            __syncthreads();
            for (int i = i0 + warp * C; i < k; i += EIG_WARPS * C) {
                double *ri = rows + (long long)((i - c) / C) * k + j + 1;
                const double vi = v[i - j - 1], wi = wv[i - j - 1];
                for (int l = lane; l < m; l += 32) ri[l] = fma(-vi, wv[l], fma(-wi, v[l], ri[l]));
            }
            cl.sync();
        }
        if (c == 0 && tid == 0) {
            if (k >= 2) {
                const double *r2 = cl.map_shared_rank(rows, (k - 2) % C) + (long long)((k - 2) / C) * k;
                g.d[k - 2] = r2[k - 2];
                g.e[k - 2] = r2[k - 1];
                g.tau[k - 2] = 0.0;
            }
            const double *r1 = cl.map_shared_rank(rows, (k - 1) % C) + (long long)((k - 1) / C) * k;
            g.d[k - 1] = r1[k - 1];
            g.tau[k - 1] = 0.0;
        }
        cl.sync();  // every read of the rows is done before the region is reused
    } else {

    // ---- 1. Householder tridiagonalisation
    for (int j = 0; j + 2 < k; ++j) {
        const int m = k - j - 1;
        const double *rowj = A + (long long)j * k + j + 1;
        for (int l = tid; l < m; l += EIG_THREADS) v[l] = __ldcg(rowj + l);
        __syncthreads();
        if (warp == 0) {
            double s = 0.0;
            for (int l = 1 + lane; l < m; l += 32) s = fma(v[l], v[l], s);
            s = warp_sum(s);
            if (lane == 0) {
                const double x0 = v[0];
                double tau = 0.0, beta = x0, scl = 1.0;
                if (s > 0.0) {
                    const double xn = sqrt(fma(x0, x0, s));
                    beta = x0 >= 0.0 ? -xn : xn;
                    tau = (beta - x0) / beta;
                    scl = 1.0 / (x0 - beta);
                }
                sc[0] = tau;
                sc[1] = scl;
                if (c == 0) {
                    g.d[j] = __ldcg(A + (long long)j * k + j);
                    g.e[j] = beta;
                    g.tau[j] = tau;
                }
            }
        }
        __syncthreads();
        const double tau = sc[0], scl = sc[1];
        if (tau == 0.0) {  // nothing below the subdiagonal: no reflection, no update
            cl.sync();
            continue;
        }
        for (int l = 1 + tid; l < m; l += EIG_THREADS) v[l] *= scl;
        if (tid == 0) v[0] = 1.0;
        __syncthreads();
        if (c == 0) {
            double *vh = g.Vh + (long long)j * k + j + 1;
            for (int l = tid; l < m; l += EIG_THREADS) vh[l] = v[l];
        }
        // p_i = tau A[i][j+1:] . v for own rows i > j (one warp per row)
        const int i0 = j + 1 + ((c - (j + 1)) % C + C) % C;
        double part = 0.0;
        for (int i = i0 + warp * C; i < k; i += EIG_WARPS * C) {
            const double *ri = A + (long long)i * k + j + 1;
            double dot = 0.0;
            for (int l = lane; l < m; l += 32) dot = fma(ri[l], v[l], dot);
            dot = warp_sum(dot) * tau;
            if (lane == 0) {
                g.P[i] = dot;
                part = fma(dot, v[i - j - 1], part);
            }
        }
        if (lane == 0) sc[8 + warp] = part;
        __syncthreads();
        if (warp == 0) {
            const double t = warp_sum(lane < EIG_WARPS ? sc[8 + lane] : 0.0);
            if (lane == 0) g.red[c] = t;
        }
        cl.sync();
        if (warp == 0) {
            const double pv = warp_sum(lane < C ? __ldcg(g.red + lane) : 0.0);
            if (lane == 0) sc[2] = 0.5 * tau * pv;
        }
        __syncthreads();
        const double K = sc[2];
        for (int l = tid; l < m; l += EIG_THREADS) wv[l] = fma(-K, v[l], __ldcg(g.P + j + 1 + l));
        __syncthreads();
        for (int i = i0 + warp * C; i < k; i += EIG_WARPS * C) {
            double *ri = A + (long long)i * k + j + 1;
            const double vi = v[i - j - 1], wi = wv[i - j - 1];
            for (int l = lane; l < m; l += 32) ri[l] = fma(-vi, wv[l], fma(-wi, v[l], ri[l]));
        }
        cl.sync();
    }
    if (c == 0 && tid == 0) {
        if (k >= 2) {
            g.d[k - 2] = __ldcg(A + (long long)(k - 2) * k + k - 2);
            g.e[k - 2] = __ldcg(A + (long long)(k - 2) * k + k - 1);
            g.tau[k - 2] = 0.0;
        }
        g.d[k - 1] = __ldcg(A + (long long)(k - 1) * k + k - 1);
        g.tau[k - 1] = 0.0;
    }
    cl.sync();
    }  // rows in global memory

    // ---- 2. lowest nev eigenvalues of T by 32-way multisection (one warp each)
    for (int r = tid; r < k; r += EIG_THREADS) {
        sd[r] = __ldcg(g.d + r);
        const double er = r > 0 ? __ldcg(g.e + r - 1) : 0.0;
        se2[r] = er * er;  // e_{r-1}^2
    }
    __syncthreads();
    if (warp == 0) {
        double lo = INFINITY, hi = -INFINITY;
        for (int r = lane; r < k; r += 32) {
            const double rad = sqrt(se2[r]) + (r + 1 < k ? sqrt(se2[r + 1]) : 0.0);
            lo = fmin(lo, sd[r] - rad);
            hi = fmax(hi, sd[r] + rad);
        }
        lo = -warp_max(-lo);
        hi = warp_max(hi);
        if (lane == 0) {
            sc[3] = lo;
            sc[4] = hi;
        }
    }
    __syncthreads();
    const double tnorm = fmax(fabs(sc[3]), fabs(sc[4]));
    const double eps = 0x1p-52;
    const double lo_b = sc[3] - (4.0 * eps * tnorm + 0x1p-1000), hi_b = sc[4] + (4.0 * eps * tnorm + 0x1p-1000);
    for (int i = c + C * warp; i < nev; i += C * EIG_WARPS) {
        double lo = lo_b, hi = hi_b;
        for (int round = 0; round < 40; ++round) {
            if (hi - lo <= 4.0 * eps * tnorm + 0x1p-1000) break;
            const double x = lo + (hi - lo) * (double)(lane + 1) * (1.0 / 33.0);
            const int cnt = sturm_count(sd, se2, k, x);
            const unsigned above = __ballot_sync(0xffffffffu, cnt >= i + 1);
            const int ls = above ? __ffs(above) - 1 : 32;
            const double nlo = ls == 0 ? lo : lo + (hi - lo) * (double)ls * (1.0 / 33.0);
            const double nhi = ls == 32 ? hi : lo + (hi - lo) * (double)(ls + 1) * (1.0 / 33.0);
            lo = nlo;
            hi = nhi;
        }
        if (lane == 0) g.lam[i] = 0.5 * (lo + hi);
    }
    cl.sync();

    // ---- 3. eigenvectors of T by inverse iteration; eigenvalues closer than
    // 1e-6 |T| form a group handled by one warp (lane 0), groups dealt over the
    // cluster's slot warps
    const double ortol = 1e-6 * tnorm;
    const double pivtol = eps * fmax(tnorm, 1e-300);
    if (warp < EIG_SLOTS) {
        int gidx = 0, i0 = 0;
        while (i0 < nev) {
            int i1 = i0 + 1;
            while (i1 < nev && __ldcg(g.lam + i1) - __ldcg(g.lam + i1 - 1) < ortol) ++i1;
            if (gidx % (C * EIG_SLOTS) == c * EIG_SLOTS + warp) {
                // lane 0 runs the sequential factorisation and substitutions; the
                // whole warp the reductions, scalings and copies
                double lam_prev = 0.0, rq_prev = 0.0;
                for (int i = i0; i < i1; ++i) {
                    double lam = __ldcg(g.lam + i);
                    if (i > i0 && lam <= lam_prev + 10.0 * pivtol) lam = lam_prev + 10.0 * pivtol;
                    lam_prev = lam;
                    double *u0 = slots ? slots + (long long)warp * 6 * k : g.ws + (long long)i * 6 * k;
                    double *u1 = u0 + k, *u2 = u1 + k, *lm = u2 + k, *pv = lm + k, *y = pv + k;
                    double *zout = g.ws + (long long)i * 6 * k + 5 * k;
                    if (lane == 0) {
                        // T - lam I = P L U; u0 holds 1 / (diagonal of U)
                        double dd = sd[0] - lam, du = k > 1 ? __ldcg(g.e) : 0.0;
                        for (int r = 0; r + 1 < k; ++r) {
                            const double er = __ldcg(g.e + r);
                            const double nd = sd[r + 1] - lam;
                            const double ndu = r + 2 < k ? __ldcg(g.e + r + 1) : 0.0;
                            if (fabs(dd) >= fabs(er)) {
                                if (fabs(dd) < pivtol) dd = dd < 0.0 ? -pivtol : pivtol;
                                const double rd = 1.0 / dd;
                                const double mlt = er * rd;
                                u0[r] = rd;
                                u1[r] = du;
                                u2[r] = 0.0;
                                lm[r] = mlt;
                                pv[r] = 0.0;
                                dd = fma(-mlt, du, nd);
                                du = ndu;
                            } else {
                                const double rd = 1.0 / er;
                                const double mlt = dd * rd;
                                u0[r] = rd;
                                u1[r] = nd;
                                u2[r] = ndu;
                                lm[r] = mlt;
                                pv[r] = 1.0;
                                dd = fma(-mlt, nd, du);
                                du = -mlt * ndu;
                            }
                        }
                        if (fabs(dd) < pivtol) dd = dd < 0.0 ? -pivtol : pivtol;
                        u0[k - 1] = 1.0 / dd;
                    }
                    for (int r = lane; r < k; r += 32) y[r] = start_entry(i, r);
                    __syncwarp();
                    // two solves: the shift is accurate to a few ulps of |T|, so the
                    // second solve from the first one's direction is at full precision
                    for (int itn = 0; itn < 2; ++itn) {
                        if (lane == 0) {
                            double cur = y[0];
                            for (int r = 0; r + 1 < k; ++r) {
                                const double nx = y[r + 1];
                                if (pv[r] != 0.0) {
                                    y[r] = nx;
                                    cur = fma(-lm[r], nx, cur);
                                } else {
                                    y[r] = cur;
                                    cur = fma(-lm[r], cur, nx);
                                }
                            }
                            y[k - 1] = cur * u0[k - 1];
                            if (k >= 2) y[k - 2] = (y[k - 2] - u1[k - 2] * y[k - 1]) * u0[k - 2];
                            for (int r = k - 3; r >= 0; --r) y[r] = (y[r] - u1[r] * y[r + 1] - u2[r] * y[r + 2]) * u0[r];
                        }
                        __syncwarp();
                        for (int q = i0; q < i; ++q) {
                            const double *zq = g.ws + (long long)q * 6 * k + 5 * k;
                            double dot = 0.0;
                            for (int r = lane; r < k; r += 32) dot = fma(zq[r], y[r], dot);
                            dot = warp_sum(dot);
                            for (int r = lane; r < k; r += 32) y[r] = fma(-dot, zq[r], y[r]);
                            __syncwarp();
                        }
                        double big = 0.0;
                        for (int r = lane; r < k; r += 32) big = fmax(big, fabs(y[r]));
                        big = warp_max(big);
                        if (big == 0.0) {
                            for (int r = lane; r < k; r += 32) y[r] = start_entry(i + 7919, r);
                            __syncwarp();
                            continue;
                        }
                        const double ib = 1.0 / big;
                        double nrm = 0.0;
                        for (int r = lane; r < k; r += 32) {
                            const double t = y[r] * ib;
                            nrm = fma(t, t, nrm);
                        }
                        nrm = warp_sum(nrm);
                        const double den = big * sqrt(nrm);
                        if (itn == 0) {
                            const double s1 = 1.0 / den;
                            for (int r = lane; r < k; r += 32) y[r] *= s1;
                        } else {
                            for (int r = lane; r < k; r += 32) y[r] /= den;  // exact unit entries survive
                        }
                        __syncwarp();
                    }
                    // eigenvalue: Rayleigh quotient of the unit vector, non-decreasing in the group
                    double rq = 0.0;
                    for (int r = lane; r < k; r += 32) {
                        rq = fma(sd[r] * y[r], y[r], rq);
                        if (r > 0) rq = fma(2.0 * __ldcg(g.e + r - 1) * y[r - 1], y[r], rq);
                    }
                    rq = warp_sum(rq);
                    if (i > i0) rq = fmax(rq, rq_prev);
                    rq_prev = rq;
                    if (lane == 0) g.w[i] = rq;
                    if (zout != y)
                        for (int r = lane; r < k; r += 32) zout[r] = y[r];
                    __syncwarp();
                }
            }
            ++gidx;
            i0 = i1;
        }
    }
    cl.sync();

    // ---- 4. back-transformation z = H_0 ... H_{k-3} y, one vector per slot warp
    if (warp < EIG_SLOTS) {
        for (int i = c + C * warp; i < nev; i += C * EIG_SLOTS) {
            double *zg = g.ws + (long long)i * 6 * k + 5 * k;
            if (slots) {
                double *z = slots + (long long)warp * 6 * k;
                for (int r = lane; r < k; r += 32) z[r] = __ldcg(zg + r);
                __syncwarp();
                // the first 8 x 32 entries of each reflector (and its tau) are loaded one
                // step ahead: they do not depend on z, so their latency overlaps the
                // current step's reduction
                constexpr int PF = 8;
                double cv[PF], nv[PF];
                double ct = 0.0, nt = 0.0;
                auto fetch = [&](int j, double (&v)[PF], double &t) {
                    t = __ldcg(g.tau + j);
                    const int m = k - j - 1;
                    const double *vh = g.Vh + (long long)j * k + j + 1;
#pragma unroll
                    for (int u = 0; u < PF; ++u) {
                        const int l = lane + 32 * u;
                        v[u] = l < m ? __ldcg(vh + l) : 0.0;
                    }
                };
                if (k >= 3) fetch(k - 3, nv, nt);
                for (int j = k - 3; j >= 0; --j) {
#pragma unroll
                    for (int u = 0; u < PF; ++u) cv[u] = nv[u];
                    ct = nt;
                    if (j > 0) fetch(j - 1, nv, nt);
                    if (ct == 0.0) continue;
                    const int m = k - j - 1;
                    const double *vh = g.Vh + (long long)j * k + j + 1;
                    double *zj = z + j + 1;
                    double dot = 0.0;
#pragma unroll
                    for (int u = 0; u < PF; ++u) {
                        const int l = lane + 32 * u;
                        if (l < m) dot = fma(cv[u], zj[l], dot);
                    }
                    for (int l = lane + 32 * PF; l < m; l += 32) dot = fma(__ldcg(vh + l), zj[l], dot);
                    dot = warp_sum(dot) * ct;
#pragma unroll
                    for (int u = 0; u < PF; ++u) {
                        const int l = lane + 32 * u;
                        if (l < m) zj[l] = fma(-dot, cv[u], zj[l]);
                    }
                    for (int l = lane + 32 * PF; l < m; l += 32) zj[l] = fma(-dot, __ldcg(vh + l), zj[l]);
                    __syncwarp();
                }
                for (int r = lane; r < k; r += 32) g.Y[(long long)r * g.ldy + i] = z[r];
            } else {
                // vectors written by other CTAs: every read bypasses L1
                for (int j = k - 3; j >= 0; --j) {
                    const double t = __ldcg(g.tau + j);
                    if (t == 0.0) continue;
                    const int m = k - j - 1;
                    const double *vh = g.Vh + (long long)j * k + j + 1;
                    double dot = 0.0;
                    for (int l = lane; l < m; l += 32) dot = fma(__ldcg(vh + l), __ldcg(zg + j + 1 + l), dot);
                    dot = warp_sum(dot) * t;
                    for (int l = lane; l < m; l += 32) zg[j + 1 + l] = fma(-dot, __ldcg(vh + l), __ldcg(zg + j + 1 + l));
                    __syncwarp();
                }
                for (int r = lane; r < k; r += 32) g.Y[(long long)r * g.ldy + i] = __ldcg(zg + r);
            }
            __syncwarp();
        }
    }
}

}  // namespace

size_t eigh_lowest_scratch(int k, int nev)
{
    return sizeof(double) * ((size_t)k * k + 5 * (size_t)k + 16 + (size_t)nev + 6 * (size_t)nev * k);
}

void eigh_lowest(Prof &prof, cudaStream_t st, double *A, int k, int nev, double *w, double *Y, int ldy,
                 double *scratch, int *flag)
{
    if (k <= 0 || nev <= 0) return;
    nev = std::min(nev, k);
    // cluster size: about 20 rows per CTA, at most 16 (non-portable sizes beyond 8)
    struct Lim {
        int maxc = 8;
        Lim()
        {
            if (cudaFuncSetAttribute(eigh_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = 16;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3(16);
                cfg.blockDim = dim3(EIG_THREADS);
                cfg.dynamicSmemBytes = 48 * 1024;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, eigh_cluster_kernel, &cfg) == cudaSuccess && n >= 1) maxc = 16;
            }
            cudaGetLastError();
        }
    };
    static const Lim lim;
    int C = 1;
    while (C < lim.maxc && C * 20 < k) C *= 2;
    const size_t base = sizeof(double) * (5 * (size_t)k + 64);
    TR_REQUIRE(base <= 200 * 1024, TR_EINVAL, "eigh: subspace too large");
    const size_t slot_bytes = sizeof(double) * EIG_SLOTS * 6 * (size_t)k;
    const size_t row_bytes = sizeof(double) * (size_t)cdiv(k, C) * k;
    const bool slots_in_smem = base + slot_bytes <= 200 * 1024;
    const bool rows_in_smem = base + row_bytes <= 200 * 1024;
    size_t smem = base + std::max(slots_in_smem ? slot_bytes : 0, rows_in_smem ? row_bytes : 0);
    static const cudaError_t sattr =
        cudaFuncSetAttribute(eigh_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    TR_CUDA(sattr);
    EigArgs g;
    g.A = A;
    g.k = k;
    g.nev = nev;
    g.w = w;
    g.Y = Y;
    g.ldy = ldy;
    double *p = scratch;
    g.Vh = p;
    p += (size_t)k * k;
    g.tau = p;
    p += k;
    g.d = p;
    p += k;
    g.e = p;
    p += k;
    g.P = p;
    p += k;
    g.red = p;
    p += 16;
    g.lam = p;
    p += nev;
    g.ws = p;
    g.slots_in_smem = slots_in_smem ? 1 : 0;
    g.rows_in_smem = rows_in_smem ? 1 : 0;
    g.flag = flag;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(EIG_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int tok = prof.begin(st, "subspace_eigh", 4.0 / 3.0 * (double)k * k * k, 0);
    TR_CUDA(cudaLaunchKernelEx(&cfg, eigh_cluster_kernel, g));
    prof.end(st, tok);
}

}  // namespace tr
