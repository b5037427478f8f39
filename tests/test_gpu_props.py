"""Transition properties (Sec. 2, Eqs. oscillator_strength and transition, Y = 0):
GPU dipole integrals (McMurchie-Davidson), their MO transform and the
transition dipoles and oscillator strengths, against the oracle (Obara-Saika
integrals, plain einsum) on the same vectors."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from oracle import tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    return tdarisp


@pytest.fixture(scope="module")
def mol():
    return synth.make_molecule(seed=41, n_heavy=6, n_h=5)


def _ctx(mol, **kw):
    c = _lib().Context(cx=0.25, **kw)
    c.set_molecule_from(mol)
    return c


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n", [1, 6, 33])
def test_transition_dipoles_against_oracle(mol, n):
    c = _ctx(mol)   # no tr_build needed
    X = synth.random_trial_block(900 + n, n, mol.nocc, mol.nvir)
    mu = c.transition_dipoles(X)
    ref = tda.transition_dipoles(mol.xyz, mol.shells, mol.C, mol.nocc, X)
    assert mu.shape == (n, 3)
    assert _rel(mu, ref) < 1e-12


def test_origin_and_device_path(mol):
    c = _ctx(mol)
    X = synth.random_trial_block(17, 4, mol.nocc, mol.nvir)
    mu_h = c.transition_dipoles(X)
    mu_d = c.transition_dipoles(torch.from_numpy(X).cuda(), origin=(1.5, -2.0, 0.75)).cpu().numpy()
    # orthonormal orbitals: <i|a> = 0, so the origin drops out
    assert np.abs(mu_d - mu_h).max() < 1e-11 * max(1.0, np.abs(mu_h).max())


def test_oscillator_strengths_of_solved_states(mol):
    c = _ctx(mol, nstates=5, tol=1e-7)
    c.build()
    om, X, rs, info = c.solve()
    f = c.oscillator_strengths(om, X)
    ref = tda.oscillator_strengths(om, tda.transition_dipoles(mol.xyz, mol.shells, mol.C, mol.nocc, X))
    assert np.all(f >= 0)
    assert _rel(f, ref) < 1e-12
    fd = c.oscillator_strengths(torch.from_numpy(om).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    assert _rel(fd, ref) < 1e-12


@pytest.mark.parametrize("case", ["hybrid", "rsh"])
@pytest.mark.parametrize("tddft", [0, 1])
def test_24atom_oscillator_strengths_against_golden(case, tddft):
    """Solve on the GPU (TDA, or full TDDFT with X+Y), then f on the GPU, against
    the oracle's dense solution stored by tests/golden/make_golden.py."""
    here = os.path.dirname(os.path.abspath(__file__))
    gold = json.load(open(os.path.join(here, "golden", "oscillator_24atom.json")))["cases"][case]
    op = gold["options"]
    c = _lib().Context(cx=op["cx"], k_alpha=op["ka"], k_beta=op["kb"], omega=op["omega"], tddft=tddft,
                       nstates=5, tol=1e-10)
    c.set_molecule_from(synth.molecule_24())
    c.build()
    if tddft:
        om, X, _, rs, info = c.solve_tddft()
        ref_om, ref_f = gold["omega_tddft"], gold["f_tddft"]
    else:
        om, X, rs, info = c.solve()
        ref_om, ref_f = gold["omega_tda"], gold["f_tda"]
    assert info.converged
    assert np.abs(om - np.array(ref_om)).max() < 1e-9
    f = c.oscillator_strengths(om, X)
    ref = np.array(ref_f)
    assert np.all(np.abs(f - ref) <= 1e-4 * ref + 1e-9), (f, ref)
