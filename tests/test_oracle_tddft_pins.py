"""Pins of the full TDDFT-risp oracle (Sec. 2, Eqs. tddft and hessian; the
(ib|ja) exchange through T_ia^P' on the window, Sec. 3.2), each against
something other than the oracle's own formulas:

- the four-index RI tensor over all window orbitals, indexed by brute force;
- the non-Hermitian 2n x 2n response matrix of Eq. tddft, diagonalised by a
  general eigensolver;
- the eigenvector relations of Eq. tddft itself;
- the pure-functional special case, where the problem reduces to Casida's
  symmetric form D^2 + 4 D^1/2 J D^1/2;
- the TDA limit (the half sum of A + B and A - B is the A of Eq. TDA-risp)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ints, tda
from paper_2603_29257_gb300 import synth

RSH = dict(cx=1.0, ka=0.222, kb=0.778, omega=0.2)
HYB = dict(cx=0.25, ka=1.0, kb=0.0, omega=0.0)


@pytest.fixture(scope="module")
def mol():
    return synth.make_molecule(seed=7, n_heavy=3, n_h=3)


def _factors(m, op, window_ev=40.0):
    return tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, op["cx"], op["ka"], op["kb"],
                     op["omega"], window_ev=window_ev, tddft=True)


@pytest.fixture(scope="module")
def fac(mol):
    return {"rsh": _factors(mol, RSH), "hyb": _factors(mol, HYB)}


@pytest.mark.parametrize("which", ["rsh", "hyb"])
def test_exchange_terms_from_one_four_index_tensor(mol, which):
    """(ib|ja) and (ij|ab) picked by index from sum_PQ (pq|P)(P|Q)^-1(Q|rs) over
    every window orbital pair, with a window that cuts both spaces."""
    op = RSH if which == "rsh" else HYB
    m = mol
    f = _factors(m, op, window_ev=25.0)
    assert 0 < len(f.occK) < f.nocc and 0 < len(f.virK) < f.nvir
    auxK = tda.aux_shells(m.Z, m.xyz, m.aux_exp, "K")
    I = ints.int3c(m.xyz, m.shells, auxK, op["ka"], op["kb"], op["omega"])
    G = ints.int2c(auxK, op["ka"], op["kb"], op["omega"])
    mo = np.concatenate([f.occK, m.nocc + f.virK])
    Cw = m.C[:, mo]
    Ipq = np.einsum("mp,Pmn,nq->Ppq", Cw, I, Cw)
    eri = np.einsum("Ppq,PQ,Qrs->pqrs", Ipq, np.linalg.inv(G), Ipq)
    no, nv = len(f.occK), len(f.virK)
    o, v = np.arange(no), no + np.arange(nv)
    ibja = eri[np.ix_(o, v, o, v)].transpose(0, 3, 2, 1)      # [i][a][j][b] = (ib|ja)
    ijab = eri[np.ix_(o, o, v, v)].transpose(0, 2, 1, 3)      # [i][a][j][b] = (ij|ab)
    KB = tda.exchange_ri_B(f).reshape(f.nocc, f.nvir, f.nocc, f.nvir)
    KA = tda.exchange_ri(f).reshape(f.nocc, f.nvir, f.nocc, f.nvir)
    sel = np.ix_(f.occK, f.virK, f.occK, f.virK)
    sc = np.abs(ibja).max()
    assert np.abs(KB[sel] - ibja).max() < 1e-12 * sc
    assert np.abs(KA[sel] - ijab).max() < 1e-12 * sc
    # nothing outside the window
    mask = np.ones_like(KB, dtype=bool)
    mask[sel] = False
    assert not KB[mask].any()


def test_a_plus_b_and_a_minus_b_halves_give_the_tda_matrix(fac):
    for f in fac.values():
        P, M = tda.explicit_ApB(f), tda.explicit_AmB(f)
        A = tda.explicit_A(f)
        assert np.abs(0.5 * (P + M) - A).max() < 1e-13 * np.abs(A).max()
        assert np.abs(P - P.T).max() < 1e-13 * np.abs(P).max()
        assert np.abs(M - M.T).max() < 1e-13 * np.abs(M).max()


@pytest.mark.parametrize("which", ["rsh", "hyb"])
def test_dense_solve_against_the_non_hermitian_response_matrix(fac, which):
    f = fac[which]
    A = tda.explicit_A(f)
    B = 0.5 * (tda.explicit_ApB(f) - tda.explicit_AmB(f))
    L = np.block([[A, B], [-B, -A]])
    ev = np.linalg.eigvals(L)
    assert np.abs(ev.imag).max() < 1e-8 * np.abs(ev).max()
    pos = np.sort(ev.real[ev.real > 0])
    om, XpY, XmY = tda.tddft_dense(f, 6)
    assert np.abs(om - pos[:6]).max() < 1e-11 * pos[5]


@pytest.mark.parametrize("which", ["rsh", "hyb"])
def test_dense_vectors_satisfy_the_response_equations(fac, which):
    """[[A, B], [B, A]] (X, Y) = Omega (X, -Y) with X^2 - Y^2 = 1 (Eq. tddft)."""
    f = fac[which]
    A = tda.explicit_A(f)
    B = 0.5 * (tda.explicit_ApB(f) - tda.explicit_AmB(f))
    om, XpY, XmY = tda.tddft_dense(f, 5)
    n = f.nocc * f.nvir
    for k in range(5):
        p, q = XpY[k].reshape(n), XmY[k].reshape(n)
        X, Y = 0.5 * (p + q), 0.5 * (p - q)
        sc = om[k] * np.abs(X).max()
        assert np.abs(A @ X + B @ Y - om[k] * X).max() < 1e-11 * sc
        assert np.abs(B @ X + A @ Y + om[k] * Y).max() < 1e-11 * sc
        assert abs(X @ X - Y @ Y - 1.0) < 1e-12
    # Y is small next to X for these states, but not zero: the full problem differs from TDA
    assert np.abs(XpY - XmY).max() > 1e-6


def test_pure_functional_is_casida_form(mol):
    """c_x = 0: A - B = D and Omega^2 are the eigenvalues of D^2 + 4 D^1/2 J D^1/2."""
    f = _factors(mol, dict(cx=0.0, ka=1.0, kb=0.0, omega=0.0))
    d = f.D.reshape(-1)
    J = tda.coulomb_ri(f)
    S = np.diag(d * d) + 4.0 * np.sqrt(d)[:, None] * J * np.sqrt(d)[None, :]
    w = np.sqrt(np.linalg.eigvalsh(S))
    om, _, _ = tda.tddft_dense(f, 6)
    assert np.abs(om - w[:6]).max() < 1e-12 * w[5]


@pytest.mark.parametrize("which", ["rsh", "hyb"])
def test_factored_products_match_the_explicit_matrices(fac, which):
    f = fac[which]
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, f.nocc, f.nvir))
    P, M = tda.matvec_pm(f, X)
    n = f.nocc * f.nvir
    Pe = (tda.explicit_ApB(f) @ X.reshape(4, n).T).T
    Me = (tda.explicit_AmB(f) @ X.reshape(4, n).T).T
    sc = np.abs(Pe).max()
    assert np.abs(P.reshape(4, n) - Pe).max() < 1e-12 * sc
    assert np.abs(M.reshape(4, n) - Me).max() < 1e-12 * sc


def test_tddft_energies_lie_below_tda(fac):
    """Thouless' variational principle for a stable ground state: the lowest root
    is the minimum over (X, Y) of (X, Y)^T [[A, B], [B, A]] (X, Y) / (X^2 - Y^2);
    Y = 0 gives the TDA Rayleigh quotient, so the lowest TDDFT root lies at or
    below the lowest TDA root."""
    for f in fac.values():
        om, _, _ = tda.tddft_dense(f, 1)
        w = np.linalg.eigvalsh(tda.explicit_A(f))[0]
        assert om[0] <= w + 1e-12
