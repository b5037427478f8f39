"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, brute-force quadrature, textbook identities, invariants and
dense linear algebra."""
from __future__ import annotations

import math

import numpy as np
import pytest
import scipy.linalg
from scipy.special import erf

import quadrature as quad
from oracle import ints, tda
from paper_2603_29257_gb300 import synth


@pytest.fixture(scope="module")
def small_mol():
    return synth.make_molecule(seed=7, n_heavy=3, n_h=3)


# ---------------------------------------------------------------- Boys function

def _boys_quad(m, T, n=200):
    hi = min(1.0, 12 / math.sqrt(T)) if T > 0 else 1.0
    x, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * hi * (x + 1)
    return float(np.sum(0.5 * hi * w * t ** (2 * m) * np.exp(-T * t * t)))


@pytest.mark.parametrize("T", [0.0, 1e-3, 0.5, 5.0, 30.0, 59.9, 60.1, 100.0, 500.0])
def test_boys_against_quadrature(T):
    F = ints.boys(8, T)
    for m in range(9):
        assert abs(F[m] - _boys_quad(m, T)) <= 1e-13 * F[m]


def test_boys_special_values():
    F = ints.boys(8, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(9)], rtol=1e-15, atol=0)
    for T in (0.01, 2.0, 17.0, 80.0):
        assert abs(ints.boys(0, T)[0] - 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))) < 1e-15


# ---------------------------------------------------------------- integrals vs quadrature

OPS = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.3), (0.222, 0.778, 0.2)]


@pytest.mark.parametrize("la,lb,lc", [(0, 0, 0), (1, 0, 0), (0, 1, 1), (1, 1, 0), (2, 0, 1),
                                      (2, 1, 0), (1, 2, 1), (2, 2, 0), (2, 2, 1)])
@pytest.mark.parametrize("op", OPS)
def test_int3c_against_quadrature(la, lb, lc, op):
    rng = np.random.default_rng(100 * la + 10 * lb + lc)
    A = rng.normal(size=3)
    B = A + 0.8 * rng.normal(size=3)
    C = A + rng.normal(size=3)
    ea, ca = np.array([1.3, 0.4]), np.array([0.7, 0.5])
    eb, cb = np.array([0.9, 0.25]), np.array([1.1, -0.3])
    o = ints.int3c_block(A, la, ea, ca, B, lb, eb, cb, C, lc, 0.5, *op)
    q = quad.three_center(A, la, ea, ca, B, lb, eb, cb, C, lc, 0.5, *op, n=36)
    assert np.abs(o - q).max() <= 1e-11 * max(1.0, np.abs(q).max())


@pytest.mark.parametrize("la,lc", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("op", OPS)
def test_int2c_against_quadrature(la, lc, op):
    rng = np.random.default_rng(7 * la + lc)
    A = rng.normal(size=3)
    C = A + 1.5 * rng.normal(size=3)
    aux = ints.AuxShells(np.vstack([A, C]), [la, lc], [0.45, 0.6])
    G = ints.int2c(aux, *op)
    na = 2 * la + 1
    q = quad.two_center(A, la, 0.45, C, lc, 0.6, *op, n=40)
    assert np.abs(G[:na, na:] - q).max() <= 1e-11 * max(1.0, np.abs(q).max())
    # symmetry of the metric
    assert np.abs(G - G.T).max() <= 1e-14 * np.abs(G).max()


def test_p_aux_is_centre_derivative_of_s_aux():
    """(mu nu|p_x) = (1/2c) d/dC_x (mu nu|s): Richardson finite difference."""
    rng = np.random.default_rng(3)
    A, B = rng.normal(size=3), rng.normal(size=3)
    C = rng.normal(size=3)
    ea, ca, eb, cb, c = [0.8, 2.0], [0.6, 0.4], [0.5], [1.0], 0.45
    for op in OPS:
        p = ints.int3c_block(A, 2, ea, ca, B, 1, eb, cb, C, 1, c, *op)
        for d in range(3):
            def s_at(h):
                Cd = C.copy()
                Cd[d] += h
                return ints.int3c_block(A, 2, ea, ca, B, 1, eb, cb, Cd, 0, c, *op)[0]
            h = 1e-3
            d1 = (s_at(h) - s_at(-h)) / (2 * h)
            d2 = (s_at(h / 2) - s_at(-h / 2)) / h
            deriv = (4 * d2 - d1) / 3
            assert np.abs(p[d] - deriv / (2 * c)).max() < 1e-9


def test_erf_operator_limits():
    """omega -> infinity recovers Coulomb; omega -> 0 vanishes; linear in (ka, kb)."""
    rng = np.random.default_rng(5)
    A, B, C = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
    args = (A, 1, [0.9], [1.0], B, 2, [0.6, 1.7], [0.3, 0.8], C, 1, 0.5)
    coul = ints.int3c_block(*args, 1.0, 0.0, 0.0)
    big = ints.int3c_block(*args, 0.0, 1.0, 1e4)
    tiny = ints.int3c_block(*args, 0.0, 1.0, 1e-6)
    assert np.abs(big - coul).max() < 1e-7 * np.abs(coul).max()
    assert np.abs(tiny).max() < 1e-12
    e = ints.int3c_block(*args, 0.0, 1.0, 0.3)
    mix = ints.int3c_block(*args, 0.4, 0.7, 0.3)
    assert np.abs(mix - (0.4 * coul + 0.7 * e)).max() < 1e-14 * np.abs(coul).max()


def test_contracted_ao_normalisation(small_mol):
    """Generator coefficients give unit-norm AO functions (quadrature of chi^2)."""
    u, w = np.polynomial.hermite.hermgauss(30)
    for sh in small_mol.shells[:9]:
        for m in range(2 * sh.l + 1):
            tot = 0.0
            for a, ca in zip(sh.exps, sh.coefs):
                for b, cb in zip(sh.exps, sh.coefs):
                    s = 1 / math.sqrt(a + b)
                    X, Y, Z = np.meshgrid(s * u, s * u, s * u, indexing="ij")
                    W = np.einsum("i,j,k->ijk", w, w, w) * s ** 3
                    f = quad.solid_harmonic(sh.l, m, X, Y, Z)
                    tot += ca * cb * np.sum(W * f * f)
            assert abs(tot - 1.0) < 1e-12


# ---------------------------------------------------------------- RI exactness

def _coulomb_gaussians(p, q, R2, omega=None):
    """Textbook two-Gaussian repulsion int int e^{-p r1_A^2} e^{-q r2_B^2} op(r12)."""
    rho = p * q / (p + q)
    pref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q))
    if omega is None:
        T = rho * R2
        return pref * (0.5 * math.sqrt(math.pi / T) * erf(math.sqrt(T)) if T > 0 else 1.0)
    s = omega * omega / (omega * omega + rho)
    T = s * rho * R2
    f0 = 0.5 * math.sqrt(math.pi / T) * erf(math.sqrt(T)) if T > 0 else 1.0
    return pref * math.sqrt(s) * f0


@pytest.mark.parametrize("omega", [None, 0.4])
def test_ri_exact_when_densities_are_aux_functions(omega):
    """Worked example: s AO exponent a_k on atom k and aux s exponent 2 a_k on
    the same atom.  Diagonal densities then lie in the aux span and the RI value
    (mu mu|P)(P|Q)^-1(Q|nu nu) equals the exact four-centre integral."""
    A = np.array([0.0, 0.0, 0.0])
    B = np.array([0.3, -1.1, 1.7])
    a1, a2 = 0.7, 1.9
    Z = np.array([6, 6])
    xyz = np.vstack([A, B])
    c1 = (2 * a1 / math.pi) ** 0.75
    c2 = (2 * a2 / math.pi) ** 0.75
    shells = [synth.Shell(0, 0, np.array([a1]), np.array([c1])),
              synth.Shell(1, 0, np.array([a2]), np.array([c2]))]
    aux = ints.AuxShells(xyz, [0, 0], [2 * a1, 2 * a2])
    ka, kb, om = (1.0, 0.0, 0.0) if omega is None else (0.0, 1.0, omega)
    I = ints.int3c(xyz, shells, aux, ka, kb, om)
    G = ints.int2c(aux, ka, kb, om)
    ri = np.einsum("Pmn,PQ,Qkl->mnkl", I, np.linalg.inv(G), I)
    R2 = float(np.sum((A - B) ** 2))
    exact_11_22 = c1 ** 2 * c2 ** 2 * _coulomb_gaussians(2 * a1, 2 * a2, R2, omega)
    exact_11_11 = c1 ** 4 * _coulomb_gaussians(2 * a1, 2 * a1, 0.0, omega)
    assert abs(ri[0, 0, 1, 1] - exact_11_22) < 1e-13 * exact_11_22
    assert abs(ri[0, 0, 0, 0] - exact_11_11) < 1e-13 * exact_11_11


def test_one_by_one_response_matrix_by_hand():
    """Worked example: one atom, two s AO functions on it, one s aux function.
    With nocc = nvir = 1 the 1x1 TDA-risp matrix is
    e_a - e_i + 2 (ia|P)^2/(P|P) - c_x (ii|P)(aa|P)/(P|P), with the same-centre
    closed form (mu nu|P) = c_mu c_nu 2 pi^{5/2} / (p c sqrt(p + c))."""
    a = np.array([0.5, 2.0])
    cn = (2 * a / math.pi) ** 0.75
    c_aux = 0.6
    shells = [synth.Shell(0, 0, a[:1], cn[:1]), synth.Shell(0, 0, a[1:], cn[1:])]
    xyz = np.zeros((1, 3))
    S01 = cn[0] * cn[1] * (math.pi / (a[0] + a[1])) ** 1.5
    S = np.array([[1.0, S01], [S01, 1.0]])
    w, v = np.linalg.eigh(S)
    C = v @ np.diag(w ** -0.5) @ v.T
    eps = np.array([-0.5, 0.3])
    cx = 0.25
    f = tda.build(np.array([6]), xyz, shells, np.array([c_aux]), C, eps, 1, cx, window_ev=0)
    # The J aux basis of a heavy atom also has a p shell, which has zero overlap with
    # same-centre s densities; only the s function contributes.
    mn = np.array([[cn[i] * cn[j] * 2 * math.pi ** 2.5 / ((a[i] + a[j]) * c_aux * math.sqrt(a[i] + a[j] + c_aux))
                    for j in range(2)] for i in range(2)])
    PP = 2 * math.pi ** 2.5 / (c_aux * c_aux * math.sqrt(2 * c_aux))
    ia = C[:, 0] @ mn @ C[:, 1]
    ii = C[:, 0] @ mn @ C[:, 0]
    aa = C[:, 1] @ mn @ C[:, 1]
    expect = eps[1] - eps[0] + 2 * ia * ia / PP - cx * ii * aa / PP
    A = tda.explicit_A(f)
    assert A.shape == (1, 1)
    assert abs(A[0, 0] - expect) < 1e-14 * abs(expect)


# ---------------------------------------------------------------- response matrix

@pytest.fixture(scope="module")
def small_factors(small_mol):
    m = small_mol
    return tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, cx=0.25)


@pytest.fixture(scope="module")
def small_factors_rsh(small_mol):
    m = small_mol
    return tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, cx=1.0,
                     ka=0.222, kb=0.778, omega=0.2)


def test_aux_basis_excludes_hydrogen(small_mol):
    m = small_mol
    nheavy = int(np.sum(m.Z > 1))
    J = tda.aux_shells(m.Z, m.xyz, m.aux_exp, "J")
    K = tda.aux_shells(m.Z, m.xyz, m.aux_exp, "K")
    assert J.nfunc == 4 * nheavy and K.nfunc == nheavy
    assert set(J.l.tolist()) == {0, 1} and set(K.l.tolist()) == {0}


def test_window_indices():
    eps = np.array([-2.0, -1.48, -1.46, -0.3, 0.1, 1.46, 1.48, 3.0])
    occ, vir = tda.window(eps, 4, 40.0)
    assert occ.tolist() == [2, 3] and vir.tolist() == [0, 1]
    occ, vir = tda.window(eps, 4, 0.0)
    assert occ.tolist() == [0, 1, 2, 3] and vir.tolist() == [0, 1, 2, 3]


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_A_symmetric_and_columns(which, small_factors, small_factors_rsh):
    f = small_factors if which == "hyb" else small_factors_rsh
    A = tda.explicit_A(f)
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    n = A.shape[0]
    rng = np.random.default_rng(1)
    cols = rng.choice(n, 6, replace=False)
    E = np.zeros((len(cols), n))
    E[np.arange(len(cols)), cols] = 1.0
    AX = tda.matvec(f, E.reshape(len(cols), f.nocc, f.nvir)).reshape(len(cols), n)
    assert np.abs(AX - A[:, cols].T).max() < 1e-13 * np.abs(A).max()


def test_zero_coupling_gives_orbital_energy_differences(small_factors):
    f = small_factors
    z = tda.Factors(**{**f.__dict__, "Y": np.zeros_like(f.Y), "Tij": np.zeros_like(f.Tij), "cx": 0.0})
    w = np.linalg.eigvalsh(tda.explicit_A(z))
    assert np.abs(np.sort(f.D.reshape(-1)) - w).max() <= 1e-15
    f0 = tda.Factors(**{**f.__dict__, "cx": 0.0})
    assert np.abs(tda.explicit_A(f0) - np.diag(f.D.reshape(-1)) - 2 * tda.coulomb_ri(f)).max() < 1e-13


def test_coulomb_only_interlacing(small_factors):
    """J part is PSD with rank <= N_auxJ: lambda_k(D) <= lambda_k(A) <= lambda_{k+NJ}(D)."""
    f = tda.Factors(**{**small_factors.__dict__, "cx": 0.0})
    d = np.sort(f.D.reshape(-1))
    w = np.linalg.eigvalsh(tda.explicit_A(f))
    NJ = f.Y.shape[0]
    assert np.all(w >= d - 1e-12)
    assert np.all(w[: len(d) - NJ] <= d[NJ:] + 1e-12)
    Jm = tda.coulomb_ri(f)
    assert np.linalg.matrix_rank(Jm, tol=1e-10 * np.abs(Jm).max()) <= NJ


def test_translation_invariance(small_mol):
    m = small_mol
    shift = np.array([3.7, -12.1, 0.45])
    f1 = tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, 0.25)
    f2 = tda.build(m.Z, m.xyz + shift, m.shells, m.aux_exp, m.C, m.eps, m.nocc, 0.25)
    A1, A2 = tda.explicit_A(f1), tda.explicit_A(f2)
    assert np.abs(A1 - A2).max() < 1e-11 * np.abs(A1).max()


def _rot_ao(R, shells, nao):
    """AO transformation for a rotation r' = R r of the molecule: chi'(r) = chi(R^T r)."""
    T = np.zeros((nao, nao))
    rng = np.random.default_rng(0)
    pts = rng.normal(size=(40, 3))
    off = 0
    for sh in shells:
        n = 2 * sh.l + 1
        # solid harmonics of rotated points are linear combinations of the originals
        F = np.array([quad.solid_harmonic(sh.l, k, *pts.T) for k in range(n)]).T      # at r
        Fr = np.array([quad.solid_harmonic(sh.l, k, *(pts @ R).T) for k in range(n)]).T  # at R^T r
        M, *_ = np.linalg.lstsq(F, Fr, rcond=None)   # Fr = F M
        T[off:off + n, off:off + n] = M
        off += n
    return T


def test_rotation_invariance(small_mol):
    """Rotating the molecule (and the AO coefficients with it) leaves A unchanged."""
    m = small_mol
    ang = 0.7
    R = np.array([[math.cos(ang), -math.sin(ang), 0], [math.sin(ang), math.cos(ang), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)], [0, math.sin(0.4), math.cos(0.4)]])
    T = _rot_ao(R, m.shells, m.nao)
    # chi_mu(R^T r) = sum_nu chi'_nu(r) T[nu, mu] with chi' the AO functions of the
    # rotated molecule, so the rotated MOs have coefficients C' = T C
    C2 = T @ m.C
    f1 = tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, 1.0, 0.222, 0.778, 0.2)
    f2 = tda.build(m.Z, m.xyz @ R.T, m.shells, m.aux_exp, C2, m.eps, m.nocc, 1.0, 0.222, 0.778, 0.2)
    A1, A2 = tda.explicit_A(f1), tda.explicit_A(f2)
    assert np.abs(A1 - A2).max() < 1e-10 * np.abs(A1).max()


def test_generator_orbitals_orthonormal(small_mol):
    m = small_mol
    S = synth.overlap_matrix(m.xyz, m.shells)
    assert np.abs(m.C.T @ S @ m.C - np.eye(m.nao)).max() < 1e-12


# ---------------------------------------------------------------- Davidson

@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_davidson_matches_dense_eigh(which, small_factors, small_factors_rsh):
    f = small_factors if which == "hyb" else small_factors_rsh
    A = tda.explicit_A(f)
    w, v = np.linalg.eigh(A)
    r = tda.solve(f, 6, tol=1e-7)
    assert r.converged
    assert np.abs(r.omega - w[:6]).max() < 1e-10
    ov = np.abs(np.einsum("kn,nk->k", r.X, v[:, :6]))
    assert np.all(ov > 1 - 1e-8)
    assert np.all(r.resid < 1e-7)


def test_davidson_restart_path(small_factors):
    """A tiny max_space forces restarts; the converged result must not change."""
    f = small_factors
    w = np.linalg.eigvalsh(tda.explicit_A(f))
    r = tda.solve(f, 4, block=4, tol=1e-7, max_space=9, max_iter=400)
    assert r.converged and r.nrestart > 0
    assert np.abs(r.omega - w[:4]).max() < 1e-10


@pytest.mark.slow
def test_davidson_24_atom_case_matches_dense():
    m = synth.molecule_24()
    f = tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, 0.25)
    A = tda.explicit_A(f)
    w = scipy.linalg.eigh(A, eigvals_only=True, subset_by_index=[0, 4], driver="evr")
    r = tda.solve(f, 5, tol=1e-6)
    assert r.converged
    assert np.abs(r.omega - w).max() < 1e-9


# ---------------------------------------------------------------- dipole integrals (Sec. 2, Eq. transition)

def _shell(atom, l, a, c=1.0):
    return synth.Shell(atom=atom, l=l, exps=np.array([a]), coefs=np.array([c]))


def test_dipole_of_two_s_primitives_closed_form():
    """<a| x - O_x |b> = (P_x - O_x) (pi/p)^{3/2} exp(-ab/p |AB|^2) for s primitives."""
    xyz = np.array([[0.1, -0.4, 0.7], [1.3, 0.2, -0.5]])
    a, b = 0.8, 1.7
    O = np.array([0.25, -0.6, 0.9])
    M = ints.dipole(xyz, [_shell(0, 0, a), _shell(1, 0, b)], O)
    p = a + b
    P = (a * xyz[0] + b * xyz[1]) / p
    S = (math.pi / p) ** 1.5 * math.exp(-a * b / p * np.sum((xyz[0] - xyz[1]) ** 2))
    for d in range(3):
        assert abs(M[d, 0, 1] - (P[d] - O[d]) * S) < 1e-14
        assert abs(M[d, 1, 0] - M[d, 0, 1]) < 1e-15
        assert abs(M[d, 0, 0] - (xyz[0, d] - O[d]) * (math.pi / (2 * a)) ** 1.5) < 1e-14


def test_dipole_of_p_and_d_against_gauss_hermite_quadrature():
    """<p_x(A)| y - O_y |d_xy(B)> and <p_z(A)| z - O_z |d_z2(B)> by a product
    Gauss-Hermite rule about the Gaussian product centre (exact for these degrees)."""
    xyz = np.array([[0.0, 0.3, -0.2], [0.9, -0.5, 0.4]])
    a, b = 0.6, 1.1
    O = np.array([0.2, 0.1, -0.3])
    M = ints.dipole(xyz, [_shell(0, 1, a), _shell(1, 2, b)], O)
    p = a + b
    P = (a * xyz[0] + b * xyz[1]) / p
    pref = math.exp(-a * b / p * np.sum((xyz[0] - xyz[1]) ** 2))
    t, w = np.polynomial.hermite.hermgauss(8)
    g = [P[d] + t / math.sqrt(p) for d in range(3)]          # nodes per direction
    W = np.einsum("i,j,k->ijk", w, w, w) / p ** 1.5
    X, Y, Z = np.meshgrid(g[0], g[1], g[2], indexing="ij")
    A, B = xyz[0], xyz[1]
    px, pz = X - A[0], Z - A[2]
    dxy = (X - B[0]) * (Y - B[1])
    dz2 = (2 * (Z - B[2]) ** 2 - (X - B[0]) ** 2 - (Y - B[1]) ** 2) / (2 * math.sqrt(3))
    # AO order: p_x, p_y, p_z (0..2) then d: xy, yz, z2, xz, x2-y2 (3..7)
    ref1 = pref * np.sum(W * px * (Y - O[1]) * dxy)
    ref2 = pref * np.sum(W * pz * (Z - O[2]) * dz2)
    assert abs(M[1, 0, 3] - ref1) < 1e-13 * max(1.0, abs(ref1))
    assert abs(M[2, 2, 5] - ref2) < 1e-13 * max(1.0, abs(ref2))


def test_dipole_origin_shift_gives_the_overlap_of_the_orbitals(small_mol):
    """M(O) = M(0) - O_d S: the three shifted differences agree, and that overlap
    makes the synthetic orbitals (built from the input generator's own overlap)
    orthonormal, C^T S C = I."""
    m = small_mol
    O = np.array([0.3, -0.7, 1.1])
    D0 = ints.dipole(m.xyz, m.shells)
    D1 = ints.dipole(m.xyz, m.shells, O)
    S = [(D0[d] - D1[d]) / O[d] for d in range(3)]
    assert np.abs(S[0] - S[1]).max() < 1e-12 and np.abs(S[0] - S[2]).max() < 1e-12
    assert np.abs(m.C.T @ S[0] @ m.C - np.eye(m.C.shape[1])).max() < 1e-10


def test_transition_dipoles_do_not_depend_on_the_origin(small_mol):
    m = small_mol
    X = synth.random_trial_block(3, 4, m.nocc, m.nvir)
    mu0 = tda.transition_dipoles(m.xyz, m.shells, m.C, m.nocc, X)
    mu1 = tda.transition_dipoles(m.xyz, m.shells, m.C, m.nocc, X, origin=(2.0, -1.0, 0.5))
    assert np.abs(mu0 - mu1).max() < 1e-11 * max(1.0, np.abs(mu0).max())


def test_ri_invariant_under_auxiliary_rescaling(small_mol):
    """Rescaling auxiliary function P by s_P multiplies (P|mn) by s_P and (P|Q) by
    s_P s_Q; every RI quantity, and so A, A + B and A - B, is unchanged (a metric
    applied the wrong way round or left out breaks this)."""
    m = small_mol
    f = tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, cx=1.0, ka=0.222, kb=0.778, omega=0.2,
                  tddft=True)
    rng = np.random.default_rng(5)
    sJ = rng.uniform(0.2, 5.0, f.GJ.shape[0])
    sK = rng.uniform(0.2, 5.0, f.GK.shape[0])
    g = tda.Factors(**{**f.__dict__,
                       "Y": sJ[:, None, None] * f.Y, "GJ": np.outer(sJ, sJ) * f.GJ,
                       # T_ij^P = sum_Q (ij|Q) [(Q|P)^-1] carries 1/s_P; T_ab^P = (ab|P) carries s_P
                       "Tij": f.Tij / sK[:, None, None], "Tab": sK[:, None, None] * f.Tab,
                       "GK": np.outer(sK, sK) * f.GK, "Tia": sK[:, None, None] * f.Tia})
    for fn in (tda.explicit_A, tda.explicit_ApB, tda.explicit_AmB):
        a, b = fn(f), fn(g)
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("op", [(1.0, 0.0, 0.0), (0.222, 0.778, 0.2), (0.0, 1.0, 0.4)])
def test_metrics_symmetric_positive_definite(small_mol, op):
    """(P|Q) with the Coulomb, range-separated and pure long-range operators:
    symmetric, positive definite, and its Cholesky factor reproduces it."""
    m = small_mol
    for kind in ("J", "K"):
        G = ints.int2c(tda.aux_shells(m.Z, m.xyz, m.aux_exp, kind), *op)
        assert np.abs(G - G.T).max() <= 1e-15 * np.abs(G).max()
        assert np.linalg.eigvalsh(G).min() > 0.0
        L = np.linalg.cholesky(G)
        assert np.abs(L @ L.T - G).max() < 1e-13 * np.abs(G).max()
