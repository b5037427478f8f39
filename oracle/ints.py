"""Python view of the C oracle integrals -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this.
Wraps oracle/ints.c (Obara-Saika, FP64, no screening).  Auxiliary shells
are passed as (centre, l, exponent) with one uncontracted, unnormalised
primitive each (Sec. 2, Eq. g(r)).
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(_build.build())
        dp = ct.POINTER(ct.c_double)
        ip = ct.POINTER(ct.c_int)
        _lib.orc_boys.argtypes = [ct.c_int, ct.c_double, dp]
        _lib.orc_int3c.argtypes = [ct.c_int, dp, ip, ip, ip, dp, dp, ct.c_int, dp, ip, dp,
                                   ct.c_double, ct.c_double, ct.c_double, dp]
        _lib.orc_int3c_block.argtypes = [dp, ct.c_int, ct.c_int, dp, dp, dp, ct.c_int, ct.c_int,
                                         dp, dp, dp, ct.c_int, ct.c_double, ct.c_double,
                                         ct.c_double, ct.c_double, dp]
        _lib.orc_int2c.argtypes = [ct.c_int, dp, ip, dp, ct.c_double, ct.c_double, ct.c_double, dp]
        _lib.orc_dipole.argtypes = [ct.c_int, dp, ip, ip, ip, dp, dp, dp, dp]
    return _lib


def _d(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _i(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_int))


def boys(mmax: int, T: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    lib().orc_boys(mmax, float(T), _d(out))
    return out


class AuxShells:
    """Auxiliary shells: centres (n,3), l (n,), exponents (n,)."""

    def __init__(self, xyz, l, exps):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.l = np.ascontiguousarray(l, dtype=np.int32)
        self.exps = np.ascontiguousarray(exps, dtype=np.float64)

    @property
    def nfunc(self):
        return int(np.sum(2 * self.l + 1))


def _basis_arrays(xyz_atoms, shells):
    nsh = len(shells)
    sxyz = np.ascontiguousarray([xyz_atoms[s.atom] for s in shells], dtype=np.float64).reshape(nsh, 3)
    sl = np.array([s.l for s in shells], dtype=np.int32)
    snp = np.array([len(s.exps) for s in shells], dtype=np.int32)
    pst = np.zeros(nsh, dtype=np.int32)
    if nsh > 1:
        pst[1:] = np.cumsum(snp)[:-1]
    ex = np.ascontiguousarray(np.concatenate([s.exps for s in shells]), dtype=np.float64)
    cf = np.ascontiguousarray(np.concatenate([s.coefs for s in shells]), dtype=np.float64)
    nao = int(np.sum(2 * sl + 1))
    return nsh, sxyz, sl, snp, pst, ex, cf, nao


def int3c(xyz_atoms, shells, aux: AuxShells, ka=1.0, kb=0.0, omega=0.0) -> np.ndarray:
    """(P|mu nu) for the operator (ka + kb erf(omega r))/r: array [naux][nao][nao]."""
    nsh, sxyz, sl, snp, pst, ex, cf, nao = _basis_arrays(xyz_atoms, shells)
    out = np.zeros((aux.nfunc, nao, nao))
    rc = lib().orc_int3c(nsh, _d(sxyz), _i(sl), _i(snp), _i(pst), _d(ex), _d(cf),
                         len(aux.l), _d(aux.xyz), _i(aux.l), _d(aux.exps),
                         float(ka), float(kb), float(omega), _d(out))
    if rc != 0:
        raise ValueError("orc_int3c rejected its input")
    return out


def dipole(xyz_atoms, shells, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """<mu| r - origin |nu> of the AO functions: array [3][nao][nao] (x, y, z)."""
    nsh, sxyz, sl, snp, pst, ex, cf, nao = _basis_arrays(xyz_atoms, shells)
    out = np.zeros((3, nao, nao))
    O = np.ascontiguousarray(origin, dtype=np.float64)
    rc = lib().orc_dipole(nsh, _d(sxyz), _i(sl), _i(snp), _i(pst), _d(ex), _d(cf), _d(O), _d(out))
    if rc != 0:
        raise ValueError("orc_dipole rejected its input")
    return out


def int3c_block(A, la, ea, ca, B, lb, eb, cb, C, lc, ec, ka=1.0, kb=0.0, omega=0.0):
    """One block out[c][sa][sb] for AO shells (A,la) and (B,lb) and aux shell (C,lc)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    ea = np.ascontiguousarray(ea, dtype=np.float64)
    ca = np.ascontiguousarray(ca, dtype=np.float64)
    eb = np.ascontiguousarray(eb, dtype=np.float64)
    cb = np.ascontiguousarray(cb, dtype=np.float64)
    out = np.zeros((2 * lc + 1, 2 * la + 1, 2 * lb + 1))
    rc = lib().orc_int3c_block(_d(A), la, len(ea), _d(ea), _d(ca), _d(B), lb, len(eb), _d(eb),
                               _d(cb), _d(C), lc, float(ec), float(ka), float(kb), float(omega),
                               _d(out))
    if rc != 0:
        raise ValueError("orc_int3c_block rejected its input")
    return out


def int2c(aux: AuxShells, ka=1.0, kb=0.0, omega=0.0) -> np.ndarray:
    """(P|Q) for the operator (ka + kb erf(omega r))/r."""
    n = aux.nfunc
    out = np.zeros((n, n))
    rc = lib().orc_int2c(len(aux.l), _d(aux.xyz), _i(aux.l), _d(aux.exps),
                         float(ka), float(kb), float(omega), _d(out))
    if rc != 0:
        raise ValueError("orc_int2c rejected its input")
    return out
