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

TR_OK, TR_EINVAL, TR_ENOMEM, TR_ECUDA, TR_ENOCONV, TR_ENOTPD, TR_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6

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
                ("dav_dev_rows", ct.c_int), ("matvec_ws_bytes", ct.c_size_t),
                ("xform_slices", ct.c_int), ("j_ao", ct.c_int), ("tddft", ct.c_int),
                ("wait_cycles", ct.c_longlong), ("wait_test", ct.c_int)]


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


class ServerOptions(ct.Structure):
    _fields_ = [("max_active", ct.c_int), ("hbm_budget", ct.c_size_t), ("autotune_tiles", ct.c_int),
                ("build_threads", ct.c_int)]


class Request(ct.Structure):
    _fields_ = [("natm", ct.c_int), ("Z", _ip), ("xyz", _dp), ("aux_exp", _dp), ("nshell", ct.c_int),
                ("shells", ct.POINTER(Shell)), ("nao", ct.c_int), ("nmo", ct.c_int), ("nocc", ct.c_int),
                ("C", _dp), ("eps", _dp), ("opt", Options), ("want_x", ct.c_int)]


class Result(ct.Structure):
    _fields_ = [("id", ct.c_longlong), ("status", ct.c_int), ("nstates", ct.c_int),
                ("omega", ct.c_double * 64), ("resid", ct.c_double * 64), ("X", _dp),
                ("t_submit", ct.c_double), ("t_admit", ct.c_double), ("t_built", ct.c_double),
                ("t_done", ct.c_double), ("niter", ct.c_int), ("nmatvec", ct.c_int),
                ("error", ct.c_char * 160), ("j_ao", ct.c_int)]


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
    "tr_transition_dipoles": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "tr_oscillator_strengths": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "tr_matvec": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "tr_matvec_noalloc": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "tr_matvec_tddft": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "tr_solve_tddft": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                                  ct.POINTER(SolveInfo)]),
    "tr_solve": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                            ct.POINTER(SolveInfo)]),
    "tr_build_batch": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.c_int]),
    "tr_solve_batch": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, ct.POINTER(ct.c_void_p),
                                  ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_void_p), ct.c_int,
                                  ct.POINTER(SolveInfo), ct.c_int]),
    "tr_server_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.POINTER(ServerOptions)]),
    "tr_server_submit": (ct.c_int, [ct.c_void_p, ct.POINTER(Request), ct.POINTER(ct.c_longlong)]),
    "tr_server_poll": (ct.c_int, [ct.c_void_p, ct.POINTER(Result), ct.c_int, ct.c_int]),
    "tr_server_outstanding": (ct.c_int, [ct.c_void_p]),
    "tr_server_clock": (ct.c_double, [ct.c_void_p]),
    "tr_server_destroy": (None, [ct.c_void_p]),
    "tr_free": (None, [ct.c_void_p]),
    "tr_profile": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "tr_profile_get": (ct.c_int, [ct.c_void_p, ct.POINTER(ProfEntry), ct.c_int]),
    "tr_launch_count": (ct.c_long, [ct.c_void_p]),
    "tr_subspace_eigh": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p,
                                    ct.c_int]),
    "tr_memory": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t),
                             ct.POINTER(ct.c_size_t)]),
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


def build_batch(contexts, nthreads=8):
    """tr_build of several contexts concurrently (tr_build_batch)."""
    n = len(contexts)
    hs = (ct.c_void_p * n)(*[c._h for c in contexts])
    rc = lib().tr_build_batch(hs, n, nthreads)
    if rc != TR_OK:
        msgs = [lib().tr_last_error(c._h).decode() for c in contexts]
        raise TDARispError(rc, "tr_build_batch: " + "; ".join(m for m in msgs if m))


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
                  2: (d.naux_k, d.nvir_k, d.nvir_k), 3: (d.nocc, d.nvir),
                  4: (d.naux_k, d.nocc_k, d.nvir_k)}
        out = np.zeros(shapes[which])
        self._check(lib().tr_get_tensor(self._h, which, out.ctypes.data_as(ct.c_void_p), 0),
                    "tr_get_tensor")
        return out

    def _device_block(self, X, what):
        """X as a contiguous float64 CUDA tensor of shape (m, nocc, nvir); raises
        TDARispError before any pointer reaches the library otherwise."""
        import torch
        if not (_is_torch(X) and X.is_cuda):
            raise TDARispError(TR_EINVAL, "%s: X must be a CUDA tensor" % what)
        if X.dtype != torch.float64:
            raise TDARispError(TR_EINVAL, "%s: X must be float64, got %s" % (what, X.dtype))
        d = self.dims()
        if X.dim() != 3 or tuple(X.shape[1:]) != (d.nocc, d.nvir):
            raise TDARispError(TR_EINVAL, "%s: X must have shape (m, %d, %d), got %s"
                               % (what, d.nocc, d.nvir, tuple(X.shape)))
        return X.contiguous()

    def _host_block(self, X, what):
        """X as a contiguous float64 host array of shape (m, nocc, nvir)."""
        Xn = _f64(X)
        d = self.dims()
        if Xn.ndim == 2 and Xn.shape[1] == d.nocc * d.nvir:
            Xn = Xn.reshape(-1, d.nocc, d.nvir)
        if Xn.ndim != 3 or Xn.shape[1:] != (d.nocc, d.nvir):
            raise TDARispError(TR_EINVAL, "%s: X must have shape (m, %d, %d), got %s"
                               % (what, d.nocc, d.nvir, Xn.shape))
        return Xn

    @staticmethod
    def _check_out(out, X, what):
        """out must be a contiguous CUDA float64 tensor shaped like X."""
        if not (_is_torch(out) and out.is_cuda and out.dtype == X.dtype and out.shape == X.shape
                and out.is_contiguous() and out.device == X.device):
            raise TDARispError(TR_EINVAL, "%s: out must be a contiguous CUDA float64 tensor of shape %s "
                                          "on the device of X" % (what, tuple(X.shape)))

    def matvec(self, X, out=None):
        """A X for X[m][nocc][nvir]: numpy in -> numpy out (host path, synchronous);
        CUDA tensor in -> CUDA tensor out (asynchronous on the context stream)."""
        if _is_torch(X) and X.is_cuda:
            import torch
            X = self._device_block(X, "matvec")
            m = X.shape[0]
            if out is None:
                out = torch.empty_like(X)
            self._check_out(out, X, "matvec")
            rc = lib().tr_matvec(self._h, m, ct.c_void_p(X.data_ptr()), ct.c_void_p(out.data_ptr()), 1)
            self._check(rc, "tr_matvec")
            return out
        Xn = self._host_block(X, "matvec")
        m = Xn.shape[0]
        AX = np.empty_like(Xn)
        rc = lib().tr_matvec(self._h, m, Xn.ctypes.data_as(ct.c_void_p), AX.ctypes.data_as(ct.c_void_p), 0)
        self._check(rc, "tr_matvec")
        return AX

    def matvec_tddft(self, X):
        """((A + B) X, (A - B) X) of full TDDFT-risp (Sec. 2, Eq. hessian; tddft = 1):
        numpy in -> numpy out, CUDA tensor in -> CUDA tensors out (asynchronous)."""
        if _is_torch(X) and X.is_cuda:
            import torch
            X = self._device_block(X, "matvec_tddft")
            P, M = torch.empty_like(X), torch.empty_like(X)
            rc = lib().tr_matvec_tddft(self._h, X.shape[0], ct.c_void_p(X.data_ptr()), ct.c_void_p(P.data_ptr()),
                                       ct.c_void_p(M.data_ptr()), 1)
            self._check(rc, "tr_matvec_tddft")
            return P, M
        Xn = self._host_block(X, "matvec_tddft")
        P, M = np.empty_like(Xn), np.empty_like(Xn)
        rc = lib().tr_matvec_tddft(self._h, Xn.shape[0], Xn.ctypes.data_as(ct.c_void_p),
                                   P.ctypes.data_as(ct.c_void_p), M.ctypes.data_as(ct.c_void_p), 0)
        self._check(rc, "tr_matvec_tddft")
        return P, M

    def solve_tddft(self):
        """Full TDDFT-risp Davidson (tddft = 1).  Returns (omega, X+Y, X-Y, resid, info)
        as numpy arrays, (X+Y).(X-Y) = 1 per state."""
        d = self.dims()
        n = min(self._opts.nstates, d.nocc * d.nvir)
        info = SolveInfo()
        om, rs = np.zeros(n), np.zeros(n)
        P, M = np.zeros((n, d.nocc, d.nvir)), np.zeros((n, d.nocc, d.nvir))
        rc = lib().tr_solve_tddft(self._h, om.ctypes.data_as(ct.c_void_p), P.ctypes.data_as(ct.c_void_p),
                                  M.ctypes.data_as(ct.c_void_p), rs.ctypes.data_as(ct.c_void_p), 0, ct.byref(info))
        if rc not in (TR_OK, TR_ENOCONV):
            self._check(rc, "tr_solve_tddft")
        return om, P, M, rs, info

    def matvec_noalloc(self, X, out):
        """A X into out (CUDA tensors) without any device allocation (static scratch).
        X and out: float64 CUDA tensors of shape (m, nocc, nvir); out contiguous."""
        X = self._device_block(X, "matvec_noalloc")
        self._check_out(out, X, "matvec_noalloc")
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

    def transition_dipoles(self, X, origin=None):
        """mu[k][d] = sqrt(2) sum_ia <i|r_d - O_d|a> X[k][i][a] (Sec. 2, Eq. transition,
        Y = 0): numpy in -> numpy out, CUDA tensor in -> CUDA tensor out."""
        O = None if origin is None else _f64(origin)
        Op = None if O is None else O.ctypes.data_as(ct.c_void_p)
        if _is_torch(X) and X.is_cuda:
            import torch
            X = X.contiguous()
            mu = torch.empty((X.shape[0], 3), dtype=torch.float64, device=X.device)
            self._check(lib().tr_transition_dipoles(self._h, X.shape[0], ct.c_void_p(X.data_ptr()), Op,
                                                    ct.c_void_p(mu.data_ptr()), 1), "tr_transition_dipoles")
            return mu
        Xn = _f64(X)
        mu = np.zeros((Xn.shape[0], 3))
        self._check(lib().tr_transition_dipoles(self._h, Xn.shape[0], Xn.ctypes.data_as(ct.c_void_p), Op,
                                                mu.ctypes.data_as(ct.c_void_p), 0), "tr_transition_dipoles")
        return mu

    def oscillator_strengths(self, omega, X):
        """f_k = 2/3 omega_k |mu_k|^2 (Sec. 2, Eq. oscillator_strength)."""
        if _is_torch(X) and X.is_cuda:
            import torch
            X = X.contiguous()
            om = omega.contiguous()
            f = torch.empty(X.shape[0], dtype=torch.float64, device=X.device)
            self._check(lib().tr_oscillator_strengths(self._h, X.shape[0], ct.c_void_p(om.data_ptr()),
                                                      ct.c_void_p(X.data_ptr()), ct.c_void_p(f.data_ptr()), 1),
                        "tr_oscillator_strengths")
            return f
        Xn, om = _f64(X), _f64(omega)
        f = np.zeros(Xn.shape[0])
        self._check(lib().tr_oscillator_strengths(self._h, Xn.shape[0], om.ctypes.data_as(ct.c_void_p),
                                                  Xn.ctypes.data_as(ct.c_void_p), f.ctypes.data_as(ct.c_void_p), 0),
                    "tr_oscillator_strengths")
        return f

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

    def subspace_eigh(self, H, nev):
        """Lowest nev eigenpairs of the symmetric matrix H (host arrays) with the
        device eigensolver of the Davidson driver: (w[nev], Y[k][nev])."""
        Hn = _f64(H)
        k = Hn.shape[0]
        w = np.empty(nev)
        Y = np.empty((k, nev))
        self._check(lib().tr_subspace_eigh(self._h, k, Hn.ctypes.data_as(ct.c_void_p), nev,
                                           w.ctypes.data_as(ct.c_void_p), Y.ctypes.data_as(ct.c_void_p), 0),
                    "tr_subspace_eigh")
        return w, Y

    def memory(self):
        """(bytes held, peak bytes, estimated peak of build + solve)."""
        u, p, e = ct.c_size_t(), ct.c_size_t(), ct.c_size_t()
        self._check(lib().tr_memory(self._h, ct.byref(u), ct.byref(p), ct.byref(e)), "tr_memory")
        return u.value, p.value, e.value

    def launch_count(self) -> int:
        return int(lib().tr_launch_count(self._h))


class Server:
    """Continuous-batching server (tr_server_*): submit molecules as they arrive,
    poll results.  Each result is a dict with omega, resid, X (if requested),
    status, times on the server clock, niter and nmatvec."""

    def __init__(self, max_active=64, hbm_budget=0, autotune=True, build_threads=4):
        o = ServerOptions(max_active, hbm_budget, 1 if autotune else 0, build_threads)
        h = ct.c_void_p()
        rc = lib().tr_server_create(ct.byref(h), ct.byref(o))
        if rc != TR_OK:
            raise TDARispError(rc, "tr_server_create failed")
        self._h = h
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().tr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def clock(self):
        return lib().tr_server_clock(self._h)

    def submit(self, mol, want_x=False, **options):
        """Queue a molecule (Z, xyz, aux_exp, shells, C, eps, nocc); returns its id."""
        Zc = np.ascontiguousarray(mol.Z, dtype=np.int32)
        X = _f64(mol.xyz).reshape(-1, 3)
        ae = _f64(mol.aux_exp)
        arr = (Shell * len(mol.shells))()
        keep = [Zc, X, ae]
        for k, sh in enumerate(mol.shells):
            e, c = _f64(sh.exps), _f64(sh.coefs)
            keep += [e, c]
            arr[k] = Shell(int(sh.atom), int(sh.l), len(e), _ptr(e), _ptr(c))
        C, eps = _f64(mol.C), _f64(mol.eps)
        keep += [C, eps]
        q = Request(len(Zc), Zc.ctypes.data_as(_ip), _ptr(X), _ptr(ae), len(mol.shells), arr,
                    C.shape[0], C.shape[1], int(mol.nocc), _ptr(C), _ptr(eps),
                    default_options(**options), 1 if want_x else 0)
        rid = ct.c_longlong()
        rc = lib().tr_server_submit(self._h, ct.byref(q), ct.byref(rid))
        if rc != TR_OK:
            raise TDARispError(rc, "tr_server_submit failed")
        self._shapes[rid.value] = (int(mol.nocc), C.shape[1] - int(mol.nocc))
        return rid.value

    def poll(self, max_results=64, timeout_ms=-1):
        buf = (Result * max_results)()
        n = lib().tr_server_poll(self._h, buf, max_results, timeout_ms)
        if n < 0:
            raise TDARispError(n, "tr_server_poll failed")
        out = []
        for i in range(n):
            r = buf[i]
            k = r.nstates
            d = dict(id=r.id, status=r.status, nstates=k, omega=np.array(r.omega[:k]),
                     resid=np.array(r.resid[:k]), t_submit=r.t_submit, t_admit=r.t_admit,
                     t_built=r.t_built, t_done=r.t_done, niter=r.niter, nmatvec=r.nmatvec,
                     error=r.error.decode(errors="replace"), X=None, j_ao=r.j_ao)
            if r.X:
                nocc, nvir = self._shapes.get(r.id, (0, 0))
                d["X"] = np.ctypeslib.as_array(r.X, shape=(k * nocc * nvir,)).copy().reshape(k, nocc, nvir)
                lib().tr_free(ct.cast(r.X, ct.c_void_p))
            out.append(d)
        return out

    def outstanding(self):
        return lib().tr_server_outstanding(self._h)

    def drain(self, timeout_ms=-1):
        """Results of everything outstanding."""
        out = []
        while self.outstanding() > 0:
            got = self.poll(timeout_ms=timeout_ms)
            if not got and timeout_ms >= 0:
                break
            out += got
        return out
