"""TDA-risp CPU oracle in plain NumPy FP64 -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this module; the product path never imports it.  It shares no code with the
CUDA library.  Every function follows the paper's definitions directly:

  A_{ia,jb} = (e_a - e_i) d_ij d_ab + 2 (ia|jb) - c_x (ij|ab)     Sec. 2, Eq. TDA-risp
  (pq|rs)   ~ sum_PQ (pq|P) (P|Q)^-1 (Q|rs)                       Sec. 2, Eq. RI
  aux basis: one s and one p primitive per non-hydrogen atom for J,
             the s primitive only for K, none on hydrogen          Sec. 3.2
  K window:  occupied e_i > -W and virtual e_a < W (W = 40 eV),
             K restricted to that block                           Sec. 3.2
  T_ij^P = sum_Q (ij|Q) (Q|P)^-1,  T_ab^P = (ab|P),
  K_mia  = sum_P sum_j T_ij^P sum_b T_ab^P X_mjb                  Sec. 3.2, Eq. K_mia ff.
  range-separated exchange: every K integral and the K metric use
  (alpha + beta erf(omega r))/r                                   Sec. 3.2, Eqs. RSH, K_mia_RSH
  Davidson: standard block Davidson with restart that keeps the current
  Ritz vectors and recomputes A V                                 Sec. 3.3
  full TDDFT-risp: (A + B) = D + 4 (ia|jb) - c_x [(ib|ja) + (ij|ab)],
  (A - B) = D + c_x [(ib|ja) - (ij|ab)], (ib|ja) from T_ia^P' on the
  window with the K operator, and (A - B)(A + B)|X+Y> = Omega^2 |X+Y>   Sec. 2, Eqs. tddft, hessian; Sec. 3.2

The reading of (ab|Q) in the paper's T_ab definition (a dangling sum over Q)
is T_ab^P = (ab|P), which makes sum_P T_ij^P T_ab^P the RI value of (ij|ab).
The Coulomb coefficient of A + B is read as 4 (the printed Eq. hessian has 2):
with B = 2 (ia|jb) - c_x (ib|ja), the half sum of A + B and A - B is then the
A of Eq. TDA-risp, as the TDA limit requires.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import ints

HARTREE_TO_EV = 27.211386245988


def aux_shells(Z, xyz, aux_exp, kind: str, include_h: bool = False) -> ints.AuxShells:
    """Auxiliary shells of Sec. 3.2: 'J' gives s then p on every atom that
    carries an auxiliary exponent (hydrogen excluded unless include_h), 'K'
    gives the s shells only."""
    cen, ls, ex = [], [], []
    for a, z in enumerate(Z):
        if aux_exp[a] <= 0.0 or (z == 1 and not include_h):
            continue
        cen.append(xyz[a])
        ls.append(0)
        ex.append(aux_exp[a])
        if kind == "J":
            cen.append(xyz[a])
            ls.append(1)
            ex.append(aux_exp[a])
    return ints.AuxShells(np.asarray(cen).reshape(-1, 3), ls, ex)


def window(eps, nocc, window_ev):
    """Exchange window of Sec. 3.2: occupied orbitals with e > -W and virtual
    orbitals with e < W (Hartree).  window_ev <= 0 keeps every orbital."""
    eps = np.asarray(eps)
    occ = np.arange(nocc)
    vir = np.arange(len(eps) - nocc)
    if window_ev <= 0:
        return occ, vir
    w = window_ev / HARTREE_TO_EV
    return occ[eps[:nocc] > -w], vir[eps[nocc:] < w]


@dataclasses.dataclass
class Factors:
    nocc: int
    nvir: int
    D: np.ndarray        # (nocc, nvir) e_a - e_i
    Y: np.ndarray        # (NJ, nocc, nvir) (P|ia), Coulomb
    GJ: np.ndarray       # (NJ, NJ) (P|Q), Coulomb
    Tij: np.ndarray      # (NK, o', o') sum_Q (ij|Q)(Q|P)^-1 with the K operator
    Tab: np.ndarray      # (NK, v', v') (ab|P) with the K operator
    GK: np.ndarray       # (NK, NK) K-operator metric
    occK: np.ndarray     # occupied window indices
    virK: np.ndarray     # virtual window indices (relative to nocc)
    cx: float
    Tia: np.ndarray | None = None  # (NK, o', v') (ia|P) with the K operator (full TDDFT only)


def build(Z, xyz, shells, aux_exp, C, eps, nocc, cx, ka=1.0, kb=0.0, omega=0.0,
          window_ev=40.0, include_h=False, chunk=16, tddft=False) -> Factors:
    """Three-centre integrals, metrics and MO-basis tensors of Secs. 2 and 3.2.

    The K operator is (ka + kb erf(omega r))/r; for a global hybrid ka=1, kb=0.
    J always uses the Coulomb operator.  tddft: also (ia|P) on the window with
    the K operator, the tensor that only the full TDDFT exchange needs (Sec. 3.2)."""
    C = np.asarray(C, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    nmo = C.shape[1]
    nvir = nmo - nocc
    Co, Cv = C[:, :nocc], C[:, nocc:]
    occK, virK = window(eps, nocc, window_ev)
    CoK, CvK = Co[:, occK], Cv[:, virK]
    D = eps[nocc:][None, :] - eps[:nocc][:, None]

    auxJ = aux_shells(Z, xyz, aux_exp, "J", include_h)
    auxK = aux_shells(Z, xyz, aux_exp, "K", include_h)

    def mo_blocks(aux, ka_, kb_, om_, pairs):
        out = [[] for _ in pairs]
        for s0 in range(0, len(aux.l), chunk):
            sub = ints.AuxShells(aux.xyz[s0:s0 + chunk], aux.l[s0:s0 + chunk], aux.exps[s0:s0 + chunk])
            I = ints.int3c(xyz, shells, sub, ka_, kb_, om_)
            for k, (L, R) in enumerate(pairs):
                out[k].append(np.einsum("mp,Pmn,nq->Ppq", L, I, R, optimize=True))
        return [np.concatenate(o, axis=0) if o else np.zeros((0, L.shape[1], R.shape[1]))
                for o, (L, R) in zip(out, pairs)]

    (Y,) = mo_blocks(auxJ, 1.0, 0.0, 0.0, [(Co, Cv)])
    GJ = ints.int2c(auxJ)
    kpairs = [(CoK, CoK), (CvK, CvK)] + ([(CoK, CvK)] if tddft else [])
    Iij, Iab, *Iia = mo_blocks(auxK, ka, kb, omega, kpairs)
    GK = ints.int2c(auxK, ka, kb, omega)
    NK = GK.shape[0]
    if NK:
        # T_ij^P = sum_Q (ij|Q) [(Q|P)^-1]
        Tij = np.einsum("Qij,QP->Pij", Iij, np.linalg.inv(GK))
    else:
        Tij = Iij
    return Factors(nocc=nocc, nvir=nvir, D=D, Y=Y, GJ=GJ, Tij=Tij, Tab=Iab, GK=GK,
                   occK=occK, virK=virK, cx=float(cx), Tia=Iia[0] if tddft else None)


def coulomb_ri(f: Factors) -> np.ndarray:
    """(ia|jb) = sum_PQ (ia|P) (P|Q)^-1 (Q|jb) as an (nov, nov) matrix."""
    n = f.nocc * f.nvir
    if f.Y.shape[0] == 0:
        return np.zeros((n, n))
    Y = f.Y.reshape(f.Y.shape[0], n)
    return Y.T @ np.linalg.solve(f.GJ, Y)


def exchange_ri(f: Factors) -> np.ndarray:
    """(ij|ab) RI value on the window, embedded as an (nov, nov) matrix with
    rows (i,a) and columns (j,b); zero outside the window."""
    K = np.zeros((f.nocc, f.nvir, f.nocc, f.nvir))
    if f.Tij.shape[0]:
        blk = np.einsum("Pij,Pab->iajb", f.Tij, f.Tab, optimize=True)
        K[np.ix_(f.occK, f.virK, f.occK, f.virK)] = blk
    n = f.nocc * f.nvir
    return K.reshape(n, n)


def exchange_ri_B(f: Factors) -> np.ndarray:
    """(ib|ja) RI value, sum_PQ (ib|P) (P|Q)^-1 (Q|ja) with the K operator, on the
    window, embedded as an (nov, nov) matrix with rows (i,a) and columns (j,b);
    zero outside the window (Sec. 2, Eq. hessian; Sec. 3.2)."""
    K = np.zeros((f.nocc, f.nvir, f.nocc, f.nvir))
    if f.Tia is None:
        raise ValueError("exchange_ri_B: factors built without tddft=True")
    NK = f.Tia.shape[0]
    if NK:
        W = np.linalg.solve(f.GK, f.Tia.reshape(NK, -1)).reshape(f.Tia.shape)
        blk = np.einsum("Pib,Pja->iajb", f.Tia, W, optimize=True)
        K[np.ix_(f.occK, f.virK, f.occK, f.virK)] = blk
    n = f.nocc * f.nvir
    return K.reshape(n, n)


def explicit_A(f: Factors) -> np.ndarray:
    """Explicit TDA-risp matrix (Sec. 2, Eq. TDA-risp) for small problems."""
    A = 2.0 * coulomb_ri(f) - f.cx * exchange_ri(f)
    A[np.diag_indices_from(A)] += f.D.reshape(-1)
    return A


def explicit_ApB(f: Factors) -> np.ndarray:
    """A + B of Sec. 2, Eq. hessian (no XC kernel), Coulomb coefficient 4."""
    M = 4.0 * coulomb_ri(f) - f.cx * (exchange_ri_B(f) + exchange_ri(f))
    M[np.diag_indices_from(M)] += f.D.reshape(-1)
    return M


def explicit_AmB(f: Factors) -> np.ndarray:
    """A - B of Sec. 2, Eq. hessian."""
    M = f.cx * (exchange_ri_B(f) - exchange_ri(f))
    M[np.diag_indices_from(M)] += f.D.reshape(-1)
    return M


def matvec(f: Factors, X: np.ndarray) -> np.ndarray:
    """A X for a block X[m][nocc][nvir] without forming A (Sec. 3.2 order for K)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, f.nocc, f.nvir)
    AX = f.D[None] * X
    if f.Y.shape[0]:
        Z = np.einsum("Pia,mia->Pm", f.Y, X, optimize=True)
        Z = np.linalg.solve(f.GJ, Z)
        AX += 2.0 * np.einsum("Pia,Pm->mia", f.Y, Z, optimize=True)
    if f.Tij.shape[0] and len(f.occK) and len(f.virK):
        Xw = X[:, f.occK][:, :, f.virK]
        M = np.einsum("Pab,mjb->Pmja", f.Tab, Xw, optimize=True)
        K = np.einsum("Pij,Pmja->mia", f.Tij, M, optimize=True)
        AX[np.ix_(np.arange(X.shape[0]), f.occK, f.virK)] -= f.cx * K
    return AX


def matvec_B(f: Factors, X: np.ndarray) -> np.ndarray:
    """B X = 2 J X - c_x sum_jb (ib|ja) X_jb without forming B: with
    W^P = sum_Q (P|Q)^-1 (Q|ja), E^P_mij = sum_b (ib|P) X_mjb and the exchange
    part sum_P sum_j E^P_mij W^P_ja on the window."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, f.nocc, f.nvir)
    BX = np.zeros_like(X)
    if f.Y.shape[0]:
        Z = np.linalg.solve(f.GJ, np.einsum("Pia,mia->Pm", f.Y, X, optimize=True))
        BX += 2.0 * np.einsum("Pia,Pm->mia", f.Y, Z, optimize=True)
    if f.Tia is None:
        raise ValueError("matvec_B: factors built without tddft=True")
    NK = f.Tia.shape[0]
    if NK and len(f.occK) and len(f.virK):
        W = np.linalg.solve(f.GK, f.Tia.reshape(NK, -1)).reshape(f.Tia.shape)
        Xw = X[:, f.occK][:, :, f.virK]
        E = np.einsum("Pib,mjb->Pmij", f.Tia, Xw, optimize=True)
        K = np.einsum("Pmij,Pja->mia", E, W, optimize=True)
        BX[np.ix_(np.arange(X.shape[0]), f.occK, f.virK)] -= f.cx * K
    return BX


def matvec_pm(f: Factors, X: np.ndarray):
    """(A + B) X and (A - B) X from A X and B X."""
    AX, BX = matvec(f, X), matvec_B(f, X)
    return AX + BX, AX - BX


def tddft_dense(f: Factors, nstates: int):
    """Lowest nstates of the full TDDFT-risp problem (Sec. 2, Eqs. tddft and
    hessian) by dense algebra: with M = (A - B)^(1/2) (A - B positive definite),
    M (A + B) M t = Omega^2 t; X+Y = M t / sqrt(Omega) and X-Y = (A + B)(X+Y) / Omega,
    so that (X+Y).(X-Y) = 1.  Returns omega, X+Y and X-Y as [n][nocc][nvir], the
    largest-magnitude component of each X+Y positive (X-Y takes the same sign)."""
    P, Mm = explicit_ApB(f), explicit_AmB(f)
    lam, U = np.linalg.eigh(Mm)
    if lam.min() <= 0.0:
        raise ValueError("tddft_dense: A - B is not positive definite")
    Mh = (U * np.sqrt(lam)) @ U.T
    w2, T = np.linalg.eigh(Mh @ P @ Mh)
    w2, T = w2[:nstates], T[:, :nstates]
    if w2.min() <= 0.0:
        raise ValueError("tddft_dense: non-positive Omega^2")
    om = np.sqrt(w2)
    XpY = (Mh @ T / np.sqrt(om)).T
    XmY = (P @ XpY.T / om).T
    idx = np.argmax(np.abs(XpY), axis=1)
    s = np.sign(XpY[np.arange(len(om)), idx])
    s[s == 0] = 1.0
    shape = (len(om), f.nocc, f.nvir)
    return om, (XpY * s[:, None]).reshape(shape), (XmY * s[:, None]).reshape(shape)


# --------------------------------------------------------------------------
# Davidson (Sec. 3.3: standard procedure; restart keeps the Ritz vectors and
# recomputes A V).  The paper leaves guess, preconditioner and norms open;
# this oracle uses: unit-vector guess on the `block` smallest diagonal
# entries (ties to the lower index), diagonal preconditioner with the
# denominator floored at 1e-8 in magnitude, two passes of classical
# Gram-Schmidt, new vectors dropped below norm 1e-8, convergence when every
# one of the nstates residual 2-norms is below tol.

@dataclasses.dataclass
class DavidsonResult:
    omega: np.ndarray
    X: np.ndarray
    resid: np.ndarray
    niter: int
    nmatvec: int
    nrestart: int
    converged: bool


def _orth_new(V, T, drop=1e-8):
    keep = []
    for t in T:
        t = t / np.linalg.norm(t)
        for _ in range(2):
            if V.shape[0]:
                t = t - V.T @ (V @ t)
            if keep:
                Q = np.asarray(keep)
                t = t - Q.T @ (Q @ t)
        n = np.linalg.norm(t)
        if n < drop:
            continue
        keep.append(t / n)
    return np.asarray(keep).reshape(-1, V.shape[1])


def davidson(apply_A, D, nstates, block=None, tol=1e-6, max_space=None, max_iter=200,
             floor=1e-8) -> DavidsonResult:
    D = np.asarray(D, dtype=np.float64).reshape(-1)
    n = D.size
    nstates = min(nstates, n)
    block = min(n, block if block else 2 * nstates)
    block = max(block, nstates)
    max_space = max_space if max_space else 20 * nstates
    max_space = max(max_space, block + nstates)
    order = np.argsort(D, kind="stable")[:block]
    V = np.zeros((block, n))
    V[np.arange(block), order] = 1.0
    W = apply_A(V)
    nmv = block
    nrestart = 0
    theta = Xr = rn = None
    for it in range(1, max_iter + 1):
        H = V @ W.T
        H = 0.5 * (H + H.T)
        w, y = np.linalg.eigh(H)
        theta = w[:nstates]
        Y = y[:, :nstates]
        Xr = Y.T @ V
        R = Y.T @ W - theta[:, None] * Xr
        rn = np.linalg.norm(R, axis=1)
        if np.all(rn < tol):
            return DavidsonResult(theta, Xr, rn, it, nmv, nrestart, True)
        T = []
        for k in np.nonzero(rn >= tol)[0]:
            den = theta[k] - D
            small = np.abs(den) < floor
            den[small] = np.where(den[small] < 0, -floor, floor)
            T.append(R[k] / den)
        T = np.asarray(T)
        if V.shape[0] + T.shape[0] > max_space:
            V = _orth_new(np.zeros((0, n)), Xr)
            W = apply_A(V)
            nmv += V.shape[0]
            nrestart += 1
            continue
        Tn = _orth_new(V, T)
        if Tn.shape[0] == 0:
            break
        V = np.vstack([V, Tn])
        W = np.vstack([W, apply_A(Tn)])
        nmv += Tn.shape[0]
    return DavidsonResult(theta, Xr, rn, it, nmv, nrestart, False)


def solve(f: Factors, nstates, block=None, tol=1e-6, max_space=None, max_iter=200):
    """Lowest nstates of the TDA-risp problem by the Davidson procedure above."""
    nov = f.nocc * f.nvir

    def apply_A(V):
        return matvec(f, V.reshape(-1, f.nocc, f.nvir)).reshape(-1, nov)

    return davidson(apply_A, f.D, nstates, block, tol, max_space, max_iter)


def fix_sign(X):
    """Sign convention: the largest-magnitude component of each vector is positive."""
    X = np.array(X, dtype=np.float64, copy=True).reshape(X.shape[0], -1)
    idx = np.argmax(np.abs(X), axis=1)
    s = np.sign(X[np.arange(X.shape[0]), idx])
    s[s == 0] = 1.0
    return X * s[:, None]


def transition_dipoles(xyz, shells, C, nocc, X, origin=(0.0, 0.0, 0.0)):
    """Electric transition dipoles in the dipole length form with Y = 0 (Sec. 2,
    Eq. transition): mu[k][d] = sqrt(2) sum_ia r^d_ia X[k][i][a] with
    r^d_ia = sum_mn C_mi <m| r_d - O_d |n> C_na; the sqrt(2) is the singlet spin
    adaptation for unit-norm X.  For full TDDFT the same sum over X+Y with
    (X+Y).(X-Y) = 1 (Eq. transition)."""
    C = np.asarray(C, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    M = ints.dipole(xyz, shells, origin)
    r = np.einsum("mi,dmn,na->dia", C[:, :nocc], M, C[:, nocc:])
    return np.sqrt(2.0) * np.einsum("dia,kia->kd", r, X.reshape(X.shape[0], nocc, -1))


def oscillator_strengths(omega, mu):
    """f_k = 2/3 omega_k |mu_k|^2 (Sec. 2, Eq. oscillator_strength)."""
    return 2.0 / 3.0 * np.asarray(omega, dtype=np.float64) * np.sum(np.asarray(mu) ** 2, axis=1)
