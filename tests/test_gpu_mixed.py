"""Reduced-precision form (TR_MIXED: FP32 MO tensors, FP32 J contractions, K on
the tensor cores as 3xTF32) against the FP64 oracle: 1e-5 Ha per state."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from oracle import tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RSH = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)
HYB = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0)
MIXED = 1


def _ctx(mol, **opts):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(precision=MIXED, **opts)
    c.set_molecule_from(mol)
    c.build()
    return c


@pytest.fixture(scope="module")
def mid():
    # 68 atoms: window 129 occupied (two 128-row tiles, the second one row high)
    # x ~190 virtual (two 128-column tiles), 34 aux functions for K
    mol = synth.make_molecule(seed=41, n_heavy=34, n_h=34)
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, RSH["cx"],
                  RSH["k_alpha"], RSH["k_beta"], RSH["omega"])
    return mol, f


@pytest.mark.parametrize("m", [1, 13, 40])
def test_mixed_matvec_against_oracle(mid, m):
    mol, f = mid
    c = _ctx(mol, **RSH)
    d = c.dims()
    assert d.nocc_k > 128 and d.nvir_k > 128
    X = synth.random_trial_block(200 + m, m, mol.nocc, mol.nvir)
    AX = c.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = tda.matvec(f, X)
    err = np.abs(AX - ref).max() / np.abs(ref).max()
    print("mixed matvec relative error", err)
    assert err < 1e-5


def test_mixed_solve_against_dense_eigh():
    mol = synth.make_molecule(seed=7, n_heavy=3, n_h=3)
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, HYB["cx"])
    w = np.linalg.eigvalsh(tda.explicit_A(f))[:6]
    c = _ctx(mol, nstates=6, tol=1e-6, **HYB)
    om, X, rs, info = c.solve()
    err = np.abs(om - w)
    print("per-state |dOmega| (Ha), mixed:", err)
    assert info.converged and np.all(err < 1e-5)


@pytest.mark.parametrize("case", ["hybrid", "rsh"])
def test_mixed_24atom_against_golden(case):
    gold = json.load(open(os.path.join(HERE, "golden", "omega_24atom.json")))
    ref = np.array(gold["cases"][case]["omega"])
    op = HYB if case == "hybrid" else RSH
    c = _ctx(synth.molecule_24(), nstates=5, tol=1e-6, **op)
    om, X, rs, info = c.solve()
    err = np.abs(om - ref)
    print("per-state |dOmega| (Ha), mixed 24-atom %s:" % case, err)
    assert info.converged and np.all(err < 1e-5), err


def test_mixed_tensors_against_oracle(mid):
    """MO tensors (built in FP64, kept in FP32) against the FP64 oracle."""
    mol, f = mid
    c = _ctx(mol, **RSH)
    for which, ref in ((0, f.Y), (1, f.Tij), (2, f.Tab)):
        got = c.tensor(which)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print("tensor", which, "relative error", err)
        assert err < 1e-6
