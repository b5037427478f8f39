"""Brute-force 3-D quadrature of Gaussian integrals, used to pin the oracle.

Independent of every integral recursion in the repository: the AO functions
are evaluated from their explicit polynomials and the auxiliary function
enters through the closed-form electrostatic potential of a Gaussian charge,
   s:   V(d) = (pi/c)^{3/2} erf(k d) / d,     k = sqrt(c)            (Coulomb)
                                              k = sqrt(c w^2/(c+w^2)) (erf(w r)/r)
   p_x: V = (1/2c) dV_s/dC_x = (1/2c) V_s'(d) (C_x - x)/d,
and the integral over the AO product is done per primitive pair by
Gauss-Hermite quadrature around the product centre.
"""
from __future__ import annotations

import math

import numpy as np

SQ3 = math.sqrt(3.0)


def solid_harmonic(l, m, x, y, z):
    """Explicit real solid harmonics: l=1 x,y,z; l=2 xy, yz, (2zz-xx-yy)/(2 sqrt3), xz, (xx-yy)/2."""
    if l == 0:
        return np.ones_like(x)
    if l == 1:
        return (x, y, z)[m]
    return (x * y, y * z, (2 * z * z - x * x - y * y) / (2 * SQ3), x * z, (x * x - y * y) / 2)[m]


def _erf_over_d(k, d):
    out = np.empty_like(d)
    small = d < 1e-4
    ds = d[small]
    out[small] = 2 * k / math.sqrt(math.pi) * (1 - (k * ds) ** 2 / 3 + (k * ds) ** 4 / 10)
    from scipy.special import erf
    out[~small] = erf(k * d[~small]) / d[~small]
    return out


def _erf_over_d_prime_over_d(k, d):
    """(d/dd [erf(k d)/d]) / d, regular at d = 0."""
    from scipy.special import erf
    out = np.empty_like(d)
    small = d < 1e-3
    ds = d[small]
    out[small] = 2 * k / math.sqrt(math.pi) * (-2 * k * k / 3 + 4 * k ** 4 * ds * ds / 10
                                                - 6 * k ** 6 * ds ** 4 / 42)
    dl = d[~small]
    out[~small] = (2 * k / math.sqrt(math.pi) * np.exp(-(k * dl) ** 2) * dl - erf(k * dl)) / dl ** 3
    return out


def aux_potential(lc, comp, C, c, ka, kb, omega, X, Y, Z):
    """Potential at points (X,Y,Z) of the aux primitive (1 or x,y,z)*exp(-c r_C^2)
    under the operator (ka + kb erf(omega r))/r."""
    dx, dy, dz = X - C[0], Y - C[1], Z - C[2]
    d = np.sqrt(dx * dx + dy * dy + dz * dz)
    pref = (math.pi / c) ** 1.5
    ks = []
    if ka:
        ks.append((ka, math.sqrt(c)))
    if kb and omega > 0:
        ks.append((kb, math.sqrt(c * omega * omega / (c + omega * omega))))
    V = np.zeros_like(d)
    for w, k in ks:
        if lc == 0:
            V += w * pref * _erf_over_d(k, d)
        else:
            # (1/2c) dV_s/dC = (1/2c) V_s'(d) * (-(r - C)/d)
            g = _erf_over_d_prime_over_d(k, d)
            comp_d = (dx, dy, dz)[comp]
            V += w * pref * g * (-comp_d) / (2 * c)
    return V


def gh_grid(n):
    u, w = np.polynomial.hermite.hermgauss(n)
    return u, w


def three_center(A, la, ea, ca, B, lb, eb, cb, C, lc, ec, ka=1.0, kb=0.0, omega=0.0, n=40):
    """out[c][sa][sb] = int chi_a chi_b V_c by Gauss-Hermite quadrature."""
    A, B, C = (np.asarray(v, dtype=float) for v in (A, B, C))
    u, w = gh_grid(n)
    out = np.zeros((2 * lc + 1, 2 * la + 1, 2 * lb + 1))
    for a, cA in zip(ea, ca):
        for b, cB in zip(eb, cb):
            p = a + b
            P = (a * A + b * B) / p
            K = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
            s = 1.0 / math.sqrt(p)
            X = P[0] + s * u[:, None, None]
            Y = P[1] + s * u[None, :, None]
            Z = P[2] + s * u[None, None, :]
            X, Y, Z = np.broadcast_arrays(X, Y, Z)
            W = (w[:, None, None] * w[None, :, None] * w[None, None, :]) * s ** 3
            for cc in range(2 * lc + 1):
                V = aux_potential(lc, cc, C, ec, ka, kb, omega, X, Y, Z)
                for sa in range(2 * la + 1):
                    fa = solid_harmonic(la, sa, X - A[0], Y - A[1], Z - A[2])
                    for sb in range(2 * lb + 1):
                        fb = solid_harmonic(lb, sb, X - B[0], Y - B[1], Z - B[2])
                        out[cc, sa, sb] += cA * cB * K * np.sum(W * fa * fb * V)
    return out


def two_center(A, la, ea, C, lc, ec, ka=1.0, kb=0.0, omega=0.0, n=40):
    """(P|Q) for aux primitives by Gauss-Hermite quadrature of g_P(r) V_Q(r)."""
    A = np.asarray(A, dtype=float)
    u, w = gh_grid(n)
    s = 1.0 / math.sqrt(ea)
    X = A[0] + s * u[:, None, None]
    Y = A[1] + s * u[None, :, None]
    Z = A[2] + s * u[None, None, :]
    X, Y, Z = np.broadcast_arrays(X, Y, Z)
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]) * s ** 3
    out = np.zeros((2 * la + 1, 2 * lc + 1))
    for cc in range(2 * lc + 1):
        V = aux_potential(lc, cc, np.asarray(C, float), ec, ka, kb, omega, X, Y, Z)
        for sa in range(2 * la + 1):
            fa = solid_harmonic(la, sa, X - A[0], Y - A[1], Z - A[2])
            out[sa, cc] = np.sum(W * fa * V)
    return out
