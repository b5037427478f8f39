"""Thin Python binding of libtdarisp (argument marshalling only).

Every computation happens in the CUDA library behind include/tdarisp.h.
PyTorch is used only to hold device buffers and to name the CUDA stream.
If the compiled library is missing this module raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdarisp.so")

TR_OK, TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_ENOCONV, TR_ENOTPD = 0, -1, -2, -3, -4, -5

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


class Shell(ct.Structure):
    _fields_ = [("atom", ct.c_int), ("l", ct.c_int), ("nprim", ct.c_int),
                ("exp", _dp), ("coef", _dp)]


class Options(ct.Structure):
    _fields_ = [("cx", ct.c_double), ("k_alpha", ct.c_double), ("k_beta", ct.c_double),
                ("omega", ct.c_double), ("window_ev", ct.c_double), ("aux_on_h", ct.c_int),
                ("nstates", ct.c_int), ("block", ct.c_int), ("max_space", ct.c_int),
                ("max_iter", ct.c_int), ("tol", ct.c_double), ("precision", ct.c_int),
                ("screen", ct.c_double), ("hbm_budget", ct.c_size_t),
                ("aux_chunk_bytes", ct.c_size_t), ("host_budget", ct.c_size_t),
                ("dav_dev_rows", ct.c_int)]


class Dims(ct.Structure):
    _fields_ = [(n, ct.c_int) for n in ("nao", "nmo", "nocc", "nvir", "naux_j", "naux_k",
                                        "occ_k0", "nocc_k", "nvir_k", "npair", "ntotal_pair")]


class SolveInfo(ct.Structure):
    _fields_ = [("niter", ct.c_int), ("nmatvec", ct.c_int), ("nrestart", ct.c_int),
                ("converged", ct.c_int), ("t_matvec_ms", ct.c_double), ("t_ortho_ms", ct.c_double),
                ("t_eigh_ms", ct.c_double), ("t_other_ms", ct.c_double), ("max_space", ct.c_int),
                ("dev_rows", ct.c_int), ("host_bytes_moved", ct.c_longlong)]


class ProfEntry(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_long), ("total_ms", ct.c_double),
                ("flops", ct.c_double), ("bytes", ct.c_double)]


# name -> (restype, argtypes); the full C ABI of include/tdarisp.h
SIGNATURES = {
    "tr_version": (ct.c_int, []),
    "tr_options_default": (None, [ct.POINTER(Options)]),
    "tr_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.POINTER(Options), ct.c_void_p]),
    "tr_destroy": (None, [ct.c_void_p]),
    "tr_last_error": (ct.c_char_p, [ct.c_void_p]),
    "tr_set_options": (ct.c_int, [ct.c_void_p, ct.POINTER(Options)]),
    "tr_set_molecule": (ct.c_int, [ct.c_void_p, ct.c_int, _ip, _dp, _dp, ct.c_int, ct.POINTER(Shell)]),
    "tr_set_orbitals": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "tr_get_dims": (ct.c_int, [ct.c_void_p, ct.POINTER(Dims)]),
    "tr_build": (ct.c_int, [ct.c_void_p]),
    "tr_int3c": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p]),
    "tr_int2c": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p]),
    "tr_get_tensor": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int]),
    "tr_matvec": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "tr_matvec_noalloc": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "tr_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                            ct.POINTER(SolveInfo)]),
    "tr_solve_batch": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.POINTER(ct.c_void_p),
                                  ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_void_p), ct.c_int,
                                  ct.POINTER(SolveInfo), ct.c_int]),
    "tr_profile": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "tr_profile_get": (ct.c_int, [ct.c_void_p, ct.POINTER(ProfEntry), ct.c_int]),
    "tr_launch_count": (ct.c_long, [ct.c_void_p]),
}

_lib = None


def lib():
    """Load libtdarisp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtdarisp.so is not built; run __graft_entry__.build() or "
                               "python -m paper_2603_29257_gb300.build")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def solve_batch(contexts, autotune=True):
    """Lockstep Davidson solves of several built contexts (tr_solve_batch).
    Returns a list of (omega, X, resid, info) with host arrays."""
    n = len(contexts)
    hs = (ct.c_void_p * n)(*[c._h for c in contexts])
    oms, Xs, rss = [], [], []
    for c in contexts:
        d = c.dims()
        k = min(c.options.nstates, d.nocc * d.nvir)
        oms.append(np.zeros(k))
        Xs.append(np.zeros((k, d.nocc, d.nvir)))
        rss.append(np.zeros(k))
    P = ct.c_void_p * n
    op = P(*[a.ctypes.data for a in oms])
    xp = P(*[a.ctypes.data for a in Xs])
    rp = P(*[a.ctypes.data for a in rss])
    infos = (SolveInfo * n)()
    rc = lib().tr_solve_batch(hs, n, op, xp, rp, 0, infos, 1 if autotune else 0)
    if rc not in (TR_OK, TR_ENOCONV):
        raise TDARispError(rc, "tr_solve_batch: " + lib().tr_last_error(contexts[0]._h).decode())
    return [(oms[i], Xs[i], rss[i], infos[i]) for i in range(n)]


class TDARispError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


def default_options(**kw) -> Options:
    o = Options()
    lib().tr_options_default(ct.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Context:
    """One TDA-risp problem on the current CUDA device."""

    def __init__(self, stream=None, **options):
        self._opts = default_options(**options)
        h = ct.c_void_p()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available() and torch.cuda.is_initialized():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        rc = lib().tr_create(ct.byref(h), ct.byref(self._opts), ct.c_void_p(stream or 0))
        if rc != TR_OK:
            raise TDARispError(rc, "tr_create failed")
        self._h = h
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            lib().tr_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what):
        if rc not in (TR_OK,):
            msg = lib().tr_last_error(self._h).decode()
            raise TDARispError(rc, "%s: %s" % (what, msg))
        return rc

    @property
    def options(self) -> Options:
        return self._opts

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self._opts, k, v)
        self._check(lib().tr_set_options(self._h, ct.byref(self._opts)), "tr_set_options")

    def set_molecule(self, Z, xyz, aux_exp, shells):
        """shells: sequence of objects with atom, l, exps, coefs."""
        Zc = np.ascontiguousarray(Z, dtype=np.int32)
        X = _f64(xyz).reshape(-1, 3)
        ae = _f64(aux_exp)
        arr = (Shell * len(shells))()
        keep = []
        for k, s in enumerate(shells):
            e, c = _f64(s.exps), _f64(s.coefs)
            keep += [e, c]
            arr[k] = Shell(int(s.atom), int(s.l), len(e), _ptr(e), _ptr(c))
        rc = lib().tr_set_molecule(self._h, len(Zc), Zc.ctypes.data_as(_ip), _ptr(X), _ptr(ae),
                                   len(shells), arr)
        self._check(rc, "tr_set_molecule")

    def set_orbitals(self, C, eps, nocc):
        if _is_torch(C) and C.is_cuda:
            nao, nmo = C.shape
            rc = lib().tr_set_orbitals(self._h, nao, nmo, nocc, ct.c_void_p(C.data_ptr()),
                                       ct.c_void_p(eps.data_ptr()), 1)
        else:
            Cn, en = _f64(C), _f64(eps)
            nao, nmo = Cn.shape
            rc = lib().tr_set_orbitals(self._h, nao, nmo, nocc, Cn.ctypes.data_as(ct.c_void_p),
                                       en.ctypes.data_as(ct.c_void_p), 0)
        self._check(rc, "tr_set_orbitals")

    def set_molecule_from(self, mol):
        """Convenience: a molecule object with Z, xyz, aux_exp, shells, C, eps, nocc."""
        self.set_molecule(mol.Z, mol.xyz, mol.aux_exp, mol.shells)
        self.set_orbitals(mol.C, mol.eps, mol.nocc)

    def dims(self) -> Dims:
        d = Dims()
        self._check(lib().tr_get_dims(self._h, ct.byref(d)), "tr_get_dims")
        return d

    def build(self):
        self._check(lib().tr_build(self._h), "tr_build")

    def int3c(self, which, p0, np_, out):
        """Raw AO integrals into a CUDA tensor out[np][nao][nao] (float64)."""
        self._check(lib().tr_int3c(self._h, which, p0, np_, ct.c_void_p(out.data_ptr())), "tr_int3c")
        return out

    def int2c(self, which, out):
        self._check(lib().tr_int2c(self._h, which, ct.c_void_p(out.data_ptr())), "tr_int2c")
        return out

    def tensor(self, which) -> np.ndarray:
        d = self.dims()
        shapes = {0: (d.naux_j, d.nocc, d.nvir), 1: (d.naux_k, d.nocc_k, d.nocc_k),
                  2: (d.naux_k, d.nvir_k, d.nvir_k), 3: (d.nocc, d.nvir)}
        out = np.zeros(shapes[which])
        self._check(lib().tr_get_tensor(self._h, which, out.ctypes.data_as(ct.c_void_p), 0),
                    "tr_get_tensor")
        return out

    def matvec(self, X, out=None):
        """A X for X[m][nocc][nvir]: numpy in -> numpy out (host path, synchronous);
        CUDA tensor in -> CUDA tensor out (asynchronous on the context stream)."""
        if _is_torch(X) and X.is_cuda:
            import torch
            X = X.contiguous()
            m = X.shape[0]
            if out is None:
                out = torch.empty_like(X)
            rc = lib().tr_matvec(self._h, m, ct.c_void_p(X.data_ptr()), ct.c_void_p(out.data_ptr()), 1)
            self._check(rc, "tr_matvec")
            return out
        Xn = _f64(X)
        m = Xn.shape[0]
        AX = np.empty_like(Xn)
        rc = lib().tr_matvec(self._h, m, Xn.ctypes.data_as(ct.c_void_p), AX.ctypes.data_as(ct.c_void_p), 0)
        self._check(rc, "tr_matvec")
        return AX

    def matvec_noalloc(self, X, out):
        """A X into out (CUDA tensors) without any device allocation (static scratch)."""
        rc = lib().tr_matvec_noalloc(self._h, X.shape[0], ct.c_void_p(X.data_ptr()), ct.c_void_p(out.data_ptr()))
        self._check(rc, "tr_matvec_noalloc")
        return out

    def solve(self, want_x=True, device=False):
        """Davidson (Sec. 3.3).  Returns (omega, X, resid, info); X is None unless want_x.
        device=True returns CUDA tensors for omega and X."""
        d = self.dims()
        n = min(self._opts.nstates, d.nocc * d.nvir)
        info = SolveInfo()
        if device:
            import torch
            om = torch.empty(n, dtype=torch.float64, device="cuda")
            X = torch.empty((n, d.nocc, d.nvir), dtype=torch.float64, device="cuda") if want_x else None
            rs = torch.empty(n, dtype=torch.float64, device="cuda")
            rc = lib().tr_solve(self._h, ct.c_void_p(om.data_ptr()),
                                ct.c_void_p(X.data_ptr()) if want_x else None,
                                ct.c_void_p(rs.data_ptr()), 1, ct.byref(info))
        else:
            om = np.zeros(n)
            X = np.zeros((n, d.nocc, d.nvir)) if want_x else None
            rs = np.zeros(n)
            rc = lib().tr_solve(self._h, om.ctypes.data_as(ct.c_void_p),
                                X.ctypes.data_as(ct.c_void_p) if want_x else None,
                                rs.ctypes.data_as(ct.c_void_p), 0, ct.byref(info))
        if rc not in (TR_OK, TR_ENOCONV):
            self._check(rc, "tr_solve")
        return om, X, rs, info

    def profile(self, enable=True):
        self._check(lib().tr_profile(self._h, 1 if enable else 0), "tr_profile")

    def profile_get(self):
        arr = (ProfEntry * 128)()
        n = lib().tr_profile_get(self._h, arr, 128)
        if n < 0:
            self._check(n, "tr_profile_get")
        return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].total_ms,
                                           flops=arr[i].flops, bytes=arr[i].bytes)
                for i in range(n)}

    def launch_count(self) -> int:
        return int(lib().tr_launch_count(self._h))
