"""FP64 form on the tensor cores (precision TR_FP64_TC = 2): MO transforms and
the J and K contractions as 7-slice Ozaki products on tcgen05 bf16.  Results
must meet the FP64 bar: matvec element by element against the oracle at the
FP64 tolerance, excitation energies against the golden values to 1e-8 Ha."""
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
TC = 2


def _ctx(mol, **opts):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(**opts)
    c.set_molecule_from(mol)
    c.build()
    return c


@pytest.fixture(scope="module")
def mid():
    mol = synth.make_molecule(seed=41, n_heavy=34, n_h=34)
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, RSH["cx"],
                  RSH["k_alpha"], RSH["k_beta"], RSH["omega"])
    return mol, f


@pytest.mark.parametrize("m", [1, 13, 40])
def test_matvec_against_oracle(mid, m):
    mol, f = mid
    c = _ctx(mol, precision=TC, **RSH)
    X = synth.random_trial_block(300 + m, m, mol.nocc, mol.nvir)
    AX = c.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    ref = tda.matvec(f, X)
    err = np.abs(AX - ref).max() / np.abs(ref).max()
    print("FP64-TC matvec relative error", err)
    assert err < 1e-12


def test_chunked_exchange_equals_single_chunk(mid):
    """A small matvec workspace forces several P chunks (T_ij sliced at K-block
    offsets); the result equals the one-chunk product."""
    mol, _ = mid
    X = torch.from_numpy(synth.random_trial_block(77, 9, mol.nocc, mol.nvir)).cuda()
    a = _ctx(mol, precision=TC, **RSH).matvec(X).cpu().numpy()
    b = _ctx(mol, precision=TC, matvec_ws_bytes=1 << 20, **RSH).matvec(X).cpu().numpy()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("case", ["hybrid", "rsh"])
def test_24atom_against_golden(case):
    gold = json.load(open(os.path.join(HERE, "golden", "omega_24atom.json")))
    ref = np.array(gold["cases"][case]["omega"])
    op = HYB if case == "hybrid" else RSH
    c = _ctx(synth.molecule_24(), precision=TC, nstates=5, tol=1e-6, **op)
    om, X, rs, info = c.solve()
    err = np.abs(om - ref)
    print("per-state |dOmega| (Ha), FP64-TC %s:" % case, err)
    assert info.converged and np.all(err < 1e-8), err


def test_no_exchange_and_no_aux():
    """c_x = 0 (no K stages) and a molecule without auxiliary functions (no J)."""
    mol = synth.make_molecule(seed=8, n_heavy=4, n_h=4)
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, 0.0)
    c = _ctx(mol, precision=TC, cx=0.0)
    X = synth.random_trial_block(5, 3, mol.nocc, mol.nvir)
    assert np.abs(c.matvec(X) - tda.matvec(f, X)).max() < 1e-12 * np.abs(tda.matvec(f, X)).max()
    mol.aux_exp = np.zeros_like(mol.aux_exp)
    c = _ctx(mol, precision=TC, nstates=3, tol=1e-10, **HYB)
    om, X, rs, info = c.solve()
    D = np.sort((mol.eps[mol.nocc:][None, :] - mol.eps[:mol.nocc][:, None]).reshape(-1))
    # the tensor-core products accumulate in double-FP32 pairs (about 48 bits):
    # FP64-level, not bit-exact (the FP64-pipe form returns these bits exactly)
    assert np.all(np.abs(om - D[:3]) <= 4e-15 * np.abs(D[:3])), np.abs(om - D[:3]) / np.abs(D[:3])
