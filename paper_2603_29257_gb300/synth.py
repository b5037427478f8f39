"""Seeded synthetic molecules for TDA-risp workloads.

This module produces inputs only: geometry, AO basis, auxiliary exponents,
MO coefficients and orbital energies.  It holds none of the TDA-risp
arithmetic (no electron-repulsion integrals, no response matrix), so that the
CUDA library and the CPU oracle can both consume its output without sharing
any of the method's code.

The paper's molecules (PDB/CCDC structures, SCF orbitals) are not available;
these seeded stand-ins have the same shape: organic-like chains of C/N/O with
hydrogens, a def2-SVP-shaped spherical AO basis (heavy 3s2p1d, H 2s1p), the
minimal auxiliary basis of one s and one p shell per non-hydrogen atom with a
fixed exponent per element (the exponent theta/R_A^2 of the paper's Eq. for g(r)
with theta = 0.2 and a synthetic radius), and orthonormal MOs C = S^-1/2 Q.

Conventions shared as data with every consumer:
  * units: bohr and Hartree;
  * a contracted AO function is  chi(r) = sum_k coef_k * Y(r - A) * exp(-exp_k |r - A|^2)
    with the coefficients taken literally (normalisation already folded in);
  * Y for l=0 is 1; for l=1 the order is x, y, z; for l=2 the order is
    xy, yz, (2zz - xx - yy)/(2 sqrt 3), xz, (xx - yy)/2  (real solid harmonics
    m = -2..2, every one with the norm of xy);
  * auxiliary functions are the bare primitives 1 and x, y, z times
    exp(-alpha |r - A|^2), unnormalised.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ANGSTROM_TO_BOHR = 1.0 / 0.529177210903
HARTREE_TO_EV = 27.211386245988

# Synthetic auxiliary exponents (bohr^-2): theta / R^2 with theta = 0.2 and radii
# R_C = 0.7071, R_N = 0.6325, R_O = 0.5774 bohr.  These radii are chosen for the
# synthetic workload; the paper does not print its semi-empirical radii.
AUX_EXPONENT = {6: 0.40, 7: 0.50, 8: 0.60}

# Angular momenta of the AO shells per element class (def2-SVP shape).
HEAVY_SHELLS = (0, 0, 0, 1, 1, 2)
HYDROGEN_SHELLS = (0, 0, 1)
NFUNC = {0: 1, 1: 3, 2: 5}

# d-shell Cartesian order used by the cart -> spherical map below.
CART_D = ((2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2))


@dataclasses.dataclass
class Shell:
    atom: int
    l: int
    exps: np.ndarray   # (nprim,)
    coefs: np.ndarray  # (nprim,) literal coefficients of the raw primitives


@dataclasses.dataclass
class Molecule:
    Z: np.ndarray          # (natm,) int
    xyz: np.ndarray        # (natm, 3) bohr
    shells: list           # list[Shell]
    aux_exp: np.ndarray    # (natm,) exponent of the aux s/p primitive, 0 = none (H)
    nao: int
    nocc: int
    C: np.ndarray          # (nao, nmo) MO coefficients, nmo = nao
    eps: np.ndarray        # (nmo,) ascending orbital energies, Hartree
    seed: int

    @property
    def natm(self) -> int:
        return len(self.Z)

    @property
    def nvir(self) -> int:
        return self.C.shape[1] - self.nocc

    def ao_offsets(self) -> np.ndarray:
        off = np.zeros(len(self.shells) + 1, dtype=np.int64)
        for k, sh in enumerate(self.shells):
            off[k + 1] = off[k] + NFUNC[sh.l]
        return off


# --------------------------------------------------------------------------
# geometry

def _place(a, b, c, bond, angle, dihedral):
    """Position of a new atom d bonded to c with angle b-c-d and dihedral a-b-c-d."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    nn = np.linalg.norm(n)
    if nn < 1e-12:
        n = np.cross(bc, np.array([0.0, 0.0, 1.0]))
        if np.linalg.norm(n) < 1e-12:
            n = np.cross(bc, np.array([0.0, 1.0, 0.0]))
        nn = np.linalg.norm(n)
    n /= nn
    m = np.cross(n, bc)
    d2 = np.array([-bond * math.cos(angle),
                   bond * math.sin(angle) * math.cos(dihedral),
                   bond * math.sin(angle) * math.sin(dihedral)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


def chain_geometry(rng, n_heavy, n_h, max_tries=2000):
    """Heavy-atom chain (bonds 1.40 +- 0.05 A, angles U[105,125] deg, random
    dihedral; non-bonded heavy pairs >= 2.0 A) with hydrogens attached
    round-robin at 1.09 +- 0.03 A (>= 1.5 A from other heavy atoms, >= 1.4 A
    from other hydrogens).  Returns (Z, xyz in Angstrom)."""
    Zh = rng.choice(np.array([6, 7, 8]), size=n_heavy, p=[0.6, 0.2, 0.2])
    pos = [np.zeros(3)]
    if n_heavy > 1:
        pos.append(np.array([rng.uniform(1.35, 1.45), 0.0, 0.0]))
    if n_heavy > 2:
        bond = rng.uniform(1.35, 1.45)
        ang = math.radians(rng.uniform(105.0, 125.0))
        pos.append(pos[1] + bond * np.array([-math.cos(ang), math.sin(ang), 0.0]))
    k, stuck = 3, 0
    while k < n_heavy:
        for _ in range(max_tries):
            bond = rng.uniform(1.35, 1.45)
            ang = math.radians(rng.uniform(105.0, 125.0))
            dih = rng.uniform(-math.pi, math.pi)
            p = _place(pos[k - 3], pos[k - 2], pos[k - 1], bond, ang, dih)
            d = np.linalg.norm(np.asarray(pos[: k - 1]) - p, axis=1)
            if d.min() >= 2.0:
                break
        else:
            # the chain end is trapped (long chains): regrow its last few atoms
            stuck += 1
            if stuck > 1000 or k <= 3:
                raise RuntimeError("chain placement failed")
            back = min(k - 3, 4)
            del pos[k - back:]
            k -= back
            continue
        pos.append(p)
        k += 1
    heavy = np.asarray(pos)
    hpos = []
    for h in range(n_h):
        parent = h % n_heavy
        for _ in range(max_tries):
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            p = heavy[parent] + rng.uniform(1.06, 1.12) * v
            dh = np.linalg.norm(heavy - p, axis=1)
            dh[parent] = np.inf
            if dh.min() < 1.5:
                continue
            if hpos and np.linalg.norm(np.asarray(hpos) - p, axis=1).min() < 1.4:
                continue
            break
        else:
            raise RuntimeError("hydrogen placement failed")
        hpos.append(p)
    Z = np.concatenate([Zh, np.ones(n_h, dtype=Zh.dtype)]).astype(np.int32)
    xyz = np.concatenate([heavy, np.asarray(hpos).reshape(-1, 3)])
    return Z, xyz


# --------------------------------------------------------------------------
# basis

def _double_factorial(n):
    return 1 if n <= 0 else n * _double_factorial(n - 2)


def _draw_shell(rng, atom, l):
    nprim = int(rng.integers(1, 6))
    exps = np.sort(np.exp(rng.uniform(math.log(0.1), math.log(2000.0), size=nprim)))[::-1].copy()
    raw = rng.uniform(0.1, 1.0, size=nprim)
    # norm of the reference component (1, x or xy) of one-centre primitives:
    # int x^2..  exp(-p r^2) = (pi/p)^{3/2} / (2p)^l
    p = exps[:, None] + exps[None, :]
    ov = (math.pi / p) ** 1.5 / (2.0 * p) ** l
    norm = raw @ ov @ raw
    return Shell(atom=atom, l=l, exps=exps, coefs=raw / math.sqrt(norm))


def _cart_list(l):
    if l == 0:
        return [(0, 0, 0)]
    if l == 1:
        return [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    return list(CART_D)


def _cart2sph(l):
    if l < 2:
        return np.eye(NFUNC[l])
    s3 = math.sqrt(3.0)
    # rows: spherical m=-2..2, cols: CART_D
    return np.array([
        [0, 1, 0, 0, 0, 0],
        [0, 0, 0, 0, 1, 0],
        [-0.5 / s3, 0, 0, -0.5 / s3, 0, 1.0 / s3],
        [0, 0, 1, 0, 0, 0],
        [0.5, 0, 0, -0.5, 0, 0],
    ])


class _NumpyOps:
    """Array operations of the overlap code on the host (numpy)."""
    zeros = staticmethod(lambda shape: np.zeros(shape))
    sqrt = staticmethod(np.sqrt)
    exp = staticmethod(np.exp)
    einsum = staticmethod(np.einsum)
    asarray = staticmethod(lambda a: np.asarray(a, dtype=np.float64))
    index = staticmethod(lambda a: np.asarray(a))
    sum23 = staticmethod(lambda a: a.sum(axis=(2, 3)))
    swap12 = staticmethod(lambda a: a.transpose(0, 2, 1, 3))
    empty = staticmethod(lambda shape: np.empty(shape))


class _TorchOps:
    """The same operations with torch on a device (large molecules)."""

    def __init__(self, device):
        import torch
        self.t, self.dev = torch, device

    def zeros(self, shape):
        return self.t.zeros(shape, dtype=self.t.float64, device=self.dev)

    def empty(self, shape):
        return self.t.empty(shape, dtype=self.t.float64, device=self.dev)

    def sqrt(self, a):
        return self.t.sqrt(a) if self.t.is_tensor(a) else math.sqrt(a)

    def exp(self, a):
        return self.t.exp(a)

    def einsum(self, eq, *ops):
        return self.t.einsum(eq, *[o if self.t.is_tensor(o) else self.asarray(o) for o in ops])

    def asarray(self, a):
        return self.t.as_tensor(np.asarray(a, dtype=np.float64), device=self.dev)

    def index(self, a):
        return self.t.as_tensor(np.asarray(a), device=self.dev)

    @staticmethod
    def sum23(a):
        return a.sum(dim=(2, 3))

    @staticmethod
    def swap12(a):
        return a.permute(0, 2, 1, 3)


def _overlap_1d(la, lb, xa, xb, a, b, ops=_NumpyOps):
    """1-D overlap table S[i, j] for i<=la, j<=lb, vectorised over leading dims."""
    p = a + b
    xp = (a * xa + b * xb) / p
    pa, pb = xp - xa, xp - xb
    shape = tuple(np.broadcast_shapes(tuple(a.shape), tuple(b.shape), tuple(xa.shape), tuple(xb.shape)))
    s = ops.zeros(shape + (la + 1, lb + 1))
    s[..., 0, 0] = ops.sqrt(math.pi / p) * ops.exp(-a * b / p * (xa - xb) ** 2)
    inv2p = 0.5 / p
    for i in range(la + 1):
        for j in range(lb + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                v = pa * s[..., i - 1, j]
                if i > 1:
                    v = v + (i - 1) * inv2p * s[..., i - 2, j]
                if j > 0:
                    v = v + j * inv2p * s[..., i - 1, j - 1]
            else:
                v = pb * s[..., i, j - 1]
                if j > 1:
                    v = v + (j - 1) * inv2p * s[..., i, j - 2]
            s[..., i, j] = v
    return s


def overlap_matrix(xyz, shells, device=None):
    """AO overlap matrix in the spherical convention of this module (used to
    build orthonormal synthetic MOs; not part of TDA-risp).  device: None runs
    numpy on the host; a torch device name runs the same arithmetic with torch
    there (large molecules) and returns a torch tensor."""
    ops = _NumpyOps if device is None else _TorchOps(device)
    rows_chunk = 16 if device is None else 256
    off = np.zeros(len(shells) + 1, dtype=np.int64)
    for k, sh in enumerate(shells):
        off[k + 1] = off[k] + NFUNC[sh.l]
    nao = int(off[-1])
    S = ops.zeros((nao, nao))
    groups = {}
    for k, sh in enumerate(shells):
        groups.setdefault(sh.l, []).append(k)
    packed = {}
    for l, idx in groups.items():
        npmax = max(len(shells[k].exps) for k in idx)
        ex = np.ones((len(idx), npmax))
        cf = np.zeros((len(idx), npmax))
        for r, k in enumerate(idx):
            n = len(shells[k].exps)
            ex[r, :n] = shells[k].exps
            cf[r, :n] = shells[k].coefs
        cen = np.asarray([xyz[shells[k].atom] for k in idx])
        packed[l] = (np.asarray(idx), ops.asarray(ex), ops.asarray(cf), ops.asarray(cen))
    for la, (ia_all, exa_all, cfa_all, cena_all) in packed.items():
        for lb, (ib, exb, cfb, cenb) in packed.items():
            ca, cb = _cart_list(la), _cart_list(lb)
            na, nb = NFUNC[la], NFUNC[lb]
            cols = ops.index((off[ib][:, None] + np.arange(nb)[None, :]).reshape(-1))
            for r0 in range(0, len(ia_all), rows_chunk):
                ia = ia_all[r0:r0 + rows_chunk]
                exa, cfa, cena = exa_all[r0:r0 + rows_chunk], cfa_all[r0:r0 + rows_chunk], cena_all[r0:r0 + rows_chunk]
                # dims: [sa, sb, pa, pb]
                a = exa[:, None, :, None]
                b = exb[None, :, None, :]
                cc = cfa[:, None, :, None] * cfb[None, :, None, :]
                tabs = []
                for d in range(3):
                    xa = cena[:, None, None, None, d]
                    xb = cenb[None, :, None, None, d]
                    tabs.append(_overlap_1d(la, lb, xa, xb, a, b, ops))
                blk = ops.empty((len(ia), len(ib), len(ca), len(cb)))
                for u, (ax, ay, az) in enumerate(ca):
                    for v, (bx, by, bz) in enumerate(cb):
                        prim = tabs[0][..., ax, bx] * tabs[1][..., ay, by] * tabs[2][..., az, bz]
                        blk[:, :, u, v] = ops.sum23(prim * cc)
                blk = ops.einsum("mu,abuv,nv->abmn", _cart2sph(la), blk, _cart2sph(lb))
                rows = ops.index((off[ia][:, None] + np.arange(na)[None, :]).reshape(-1))
                S[rows[:, None], cols[None, :]] = ops.swap12(blk).reshape(len(ia) * na, len(ib) * nb)
    return S


def build_basis(rng, Z, xyz_bohr, min_eig=1e-7, max_redraw=200, device=None):
    shells = []
    for a, z in enumerate(Z):
        for l in (HYDROGEN_SHELLS if z == 1 else HEAVY_SHELLS):
            shells.append(_draw_shell(rng, a, l))
    for _ in range(max_redraw):
        S = overlap_matrix(xyz_bohr, shells, device)
        if device is None:
            w, v = np.linalg.eigh(S)
            soft = v[:, 0]
        else:
            import torch
            w, v = torch.linalg.eigh(S)
            soft = v[:, 0].cpu().numpy()
        if float(w[0]) > min_eig:
            return shells, S, w, v
        # redraw the shell carrying the largest weight of the softest direction
        off = np.zeros(len(shells) + 1, dtype=np.int64)
        for k, sh in enumerate(shells):
            off[k + 1] = off[k] + NFUNC[sh.l]
        wt = np.add.reduceat(soft ** 2, off[:-1])
        k = int(np.argmax(wt))
        shells[k] = _draw_shell(rng, shells[k].atom, shells[k].l)
    raise RuntimeError("could not draw a well-conditioned basis")


# --------------------------------------------------------------------------
# molecules

# molecules with more atoms than this are built with the dense linear algebra
# (overlap, its eigendecomposition, QR, products) on a CUDA device when one is
# available: the same formulas and random numbers, rounded differently
LARGE_ATOMS = 300


def make_molecule(seed: int, n_heavy: int, n_h: int, nocc: int | None = None, device=None) -> Molecule:
    """Seeded organic-like molecule with orthonormal synthetic MOs.

    nocc defaults to round(0.2 * nao) (42 of 210 for the 24-atom case).
    device: None computes everything with numpy; a torch device name ("cuda")
    runs the overlap, eigendecomposition, QR and products there."""
    rng = np.random.default_rng(seed)
    Z, xyz_ang = chain_geometry(rng, n_heavy, n_h)
    xyz = xyz_ang * ANGSTROM_TO_BOHR
    shells, S, w, v = build_basis(rng, Z, xyz, device=device)
    nao = S.shape[0]
    if nocc is None:
        nocc = int(round(nao * 42 / 210))
    g = rng.normal(size=(nao, nao))
    if device is None:
        q, r = np.linalg.qr(g)
        q = q * np.sign(np.diag(r))[None, :]
        s_inv_half = (v * (1.0 / np.sqrt(w))[None, :]) @ v.T
        C = s_inv_half @ q
    else:
        import torch
        q, r = torch.linalg.qr(torch.as_tensor(g, device=device))
        del g
        q = q * torch.sign(torch.diagonal(r))[None, :]
        del r
        s_inv_half = (v * (1.0 / torch.sqrt(w))[None, :]) @ v.T
        del v, S
        C = (s_inv_half @ q).cpu().numpy()
        del q, s_inv_half
    eps = np.concatenate([np.sort(rng.uniform(-1.2, -0.25, size=nocc)),
                          np.sort(rng.uniform(0.02, 4.0, size=nao - nocc))])
    aux = np.array([0.0 if z == 1 else AUX_EXPONENT[int(z)] for z in Z])
    return Molecule(Z=Z, xyz=xyz, shells=shells, aux_exp=aux, nao=nao, nocc=nocc,
                    C=np.ascontiguousarray(C), eps=eps, seed=seed)


def molecule_24():
    """24-atom case: 10 heavy + 14 H, nao = 210, nocc = 42, seed 1."""
    return make_molecule(1, 10, 14, nocc=42)


def molecule_200():
    """200-atom case: 100 heavy + 100 H, nao = 1900, nocc = 380, seed 2."""
    return make_molecule(2, 100, 100)


def molecule_by_atoms(seed: int, natoms: int, device=None) -> Molecule:
    """Molecule of natoms atoms, half of them (rounded) heavy.  device as in
    make_molecule ("auto": a CUDA device above LARGE_ATOMS atoms when torch sees one)."""
    n_heavy = max(1, int(round(natoms / 2)))
    if device == "auto":
        device = None
        if natoms > LARGE_ATOMS:
            try:
                import torch
                if torch.cuda.is_available():
                    device = "cuda"
            except ImportError:
                pass
    return make_molecule(seed, n_heavy, natoms - n_heavy, device=device)


def random_trial_block(seed: int, m: int, nocc: int, nvir: int) -> np.ndarray:
    """Seeded block of m trial vectors X[m][nocc][nvir] (unit norm each)."""
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(m, nocc, nvir))
    x /= np.linalg.norm(x.reshape(m, -1), axis=1)[:, None, None]
    return x
