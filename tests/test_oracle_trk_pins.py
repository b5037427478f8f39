"""Thomas-Reiche-Kuhn pins of the oracle's transition dipoles and oscillator
strengths (Sec. 2, Eqs. oscillator_strength and transition).

The model: closed-shell "traps", each an isotropic harmonic oscillator
V = omega^2 r^2 / 2 holding two electrons, placed far apart.  Per trap the AO
basis is one s and one p primitive of exponent omega/2: these are the exact
oscillator eigenfunctions (energies 3/2 omega and 5/2 omega), and x times the
ground state lies in the span of the p function, so the one-electron sum rule
sum_a (e_a - e_i) |<i|x|a>|^2 = 1/2 holds exactly in this basis.

What fixes the constants, independently of the formulas under test:
- <s|x|p_x> = 1/sqrt(2 omega), the oscillator's ladder-operator matrix element;
- the TRK sum rule: the oscillator strengths of all states sum to the number
  of electrons.  For uncoupled excitations this is the one-electron rule above
  times two electrons per trap; with Coulomb coupling and no exchange (c_x = 0)
  the full TDDFT (RPA) solution keeps the energy-weighted sum of the uncoupled
  problem (Thouless), for any coupling strength.
A dropped singlet factor sqrt(2) halves the sum, a wrong 2/3 scales it, and
X+Y normalised other than (X+Y).(X-Y) = 1 changes it once the states couple.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import tda
from paper_2603_29257_gb300 import synth


def _traps(omegas, spacing=24.0, aux=0.0):
    """Traps on the x axis `spacing` bohr apart.  Returns (Z, xyz, shells,
    aux_exp, C, eps, nocc): orbitals are the AO functions themselves (exact
    oscillator states, normalised by hand), sorted by energy."""
    n = len(omegas)
    Z = np.full(n, 6)
    xyz = np.zeros((n, 3))
    xyz[:, 0] = spacing * np.arange(n)
    shells, energies = [], []
    for t, w in enumerate(omegas):
        a = 0.5 * w
        ns = (2.0 * a / math.pi) ** 0.75            # int (N e^{-a r^2})^2 = 1
        npx = ns * 2.0 * math.sqrt(a)                # int (N x e^{-a r^2})^2 = 1
        shells.append(synth.Shell(t, 0, np.array([a]), np.array([ns])))
        shells.append(synth.Shell(t, 1, np.array([a]), np.array([npx])))
        energies += [1.5 * w] + [2.5 * w] * 3
    energies = np.array(energies)
    order = np.argsort(energies, kind="stable")
    nao = 4 * n
    C = np.zeros((nao, nao))
    C[order, np.arange(nao)] = 1.0
    return Z, xyz, shells, np.full(n, aux), C, energies[order], n


OMEGAS = [1.0, 0.8]


def test_trap_orbitals_are_orthonormal_and_dipole_is_the_ladder_element():
    Z, xyz, shells, aux, C, eps, nocc = _traps(OMEGAS)
    S = synth.overlap_matrix(xyz, shells)
    assert np.abs(C.T @ S @ C - np.eye(len(eps))).max() < 1e-14
    # one trap, one occupied (s) and one virtual (p_x) orbital: |<s|x|p_x>| = 1/sqrt(2 omega)
    # and the closed-shell singlet excitation s -> p_x (Y = 0, unit X) has
    # mu = sqrt(2) <s|x|p_x>, f = 2/3 * omega * 2 / (2 omega) = 2/3
    Z1, xyz1, sh1, _, C1, eps1, nocc1 = _traps([0.7])
    X = np.zeros((1, 1, 3))
    X[0, 0, 0] = 1.0
    mu = tda.transition_dipoles(xyz1, sh1, C1, nocc1, X)
    assert abs(abs(mu[0, 0]) - math.sqrt(2.0) / math.sqrt(2 * 0.7)) < 1e-14
    assert np.abs(mu[0, 1:]).max() < 1e-15
    f = tda.oscillator_strengths([0.7], mu)
    assert abs(f[0] - 2.0 / 3.0) < 1e-14


def test_tda_without_coupling_obeys_the_trk_sum_rule():
    Z, xyz, shells, aux, C, eps, nocc = _traps(OMEGAS)
    fac = tda.build(Z, xyz, shells, aux, C, eps, nocc, cx=0.0, window_ev=0.0)
    A = tda.explicit_A(fac)
    w, V = np.linalg.eigh(A)
    X = V.T.reshape(len(w), fac.nocc, fac.nvir)
    f = tda.oscillator_strengths(w, tda.transition_dipoles(xyz, shells, C, nocc, X))
    assert abs(f.sum() - 2.0 * len(OMEGAS)) < 1e-12       # N electrons
    # every in-trap excitation (energy omega of its trap) carries 2/3; the
    # excitations between traps carry nothing
    for om in OMEGAS:
        sel = np.abs(w - om) < 1e-12
        assert sel.sum() == 3
        assert np.allclose(f[sel], 2.0 / 3.0, atol=1e-12)
    assert np.abs(f[~np.isin(np.round(w, 12), np.round(OMEGAS, 12))]).max() < 1e-12


@pytest.mark.parametrize("aux", [0.35, 0.9])
def test_coupled_full_tddft_keeps_the_trk_sum(aux):
    Z, xyz, shells, auxe, C, eps, nocc = _traps(OMEGAS, aux=aux)
    fac = tda.build(Z, xyz, shells, auxe, C, eps, nocc, cx=0.0, window_ev=0.0, tddft=True)
    n = fac.nocc * fac.nvir
    om, XpY, XmY = tda.tddft_dense(fac, n)
    bare = np.sort(fac.D.reshape(-1))
    assert np.abs(om - bare).max() > 1e-3                # the Coulomb coupling really shifts the roots
    f = tda.oscillator_strengths(om, tda.transition_dipoles(xyz, shells, C, nocc, XpY))
    assert abs(f.sum() - 2.0 * len(OMEGAS)) < 1e-10
    # individual strengths move with the coupling; only their sum is fixed
    assert np.abs(f[f > 1e-6] - 2.0 / 3.0).max() > 1e-4


@pytest.mark.parametrize("a,b,centre,origin", [(0.3, 1.7, (1.5, -0.4, 2.0), (0.0, 0.0, 0.0)),
                                               (2.2, 0.45, (-3.0, 0.7, 0.1), (0.9, 1.1, -2.0))])
def test_s_to_p_dipole_of_unequal_exponents_by_hand(a, b, centre, origin):
    """One centre A, an occupied s primitive of exponent a and a virtual p_x
    primitive of exponent b (orthogonal by parity, so C is the diagonal of their
    norms).  By hand: <s|x - O_x|p_x> = N_s N_p int (x - A_x)^2 e^{-(a+b)|r-A|^2}
    = N_s N_p (pi/(a+b))^{3/2} / (2(a+b)); the A_x - O_x part multiplies <s|p_x> = 0.
    The singlet excitation with unit X then has mu_x = sqrt(2) r and
    f = 2/3 Omega 2 r^2 for any Omega."""
    ns = (2.0 * a / math.pi) ** 0.75
    npx = (2.0 * b / math.pi) ** 0.75 * 2.0 * math.sqrt(b)
    shells = [synth.Shell(0, 0, np.array([a]), np.array([1.0])),
              synth.Shell(0, 1, np.array([b]), np.array([1.0]))]
    xyz = np.array([centre])
    C = np.diag([ns, npx, npx, npx])
    r = ns * npx * (math.pi / (a + b)) ** 1.5 / (2.0 * (a + b))
    X = np.zeros((1, 1, 3))
    X[0, 0, 0] = 1.0
    mu = tda.transition_dipoles(xyz, shells, C, 1, X, origin=origin)
    assert abs(mu[0, 0] - math.sqrt(2.0) * r) < 1e-14 * r
    assert np.abs(mu[0, 1:]).max() < 1e-15
    Om = 0.37
    f = tda.oscillator_strengths([Om], mu)
    assert abs(f[0] - 2.0 / 3.0 * Om * 2.0 * r * r) < 1e-14
