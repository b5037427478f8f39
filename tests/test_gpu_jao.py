"""Coulomb term on the fly in the AO basis (j_ao = 1, Sec. 3.1): the same RI
operator as the stored (P|ia) route, formed from AO transition densities with
the three-centre integrals generated per auxiliary chunk.  Checked element by
element against the oracle, against the stored route, across chunkings, in
every precision, through the Davidson solve, and for the memory estimate."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HYB = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0)
RSH = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    return tdarisp


def _ctx(mol, **opts):
    c = _lib().Context(**opts)
    c.set_molecule_from(mol)
    return c


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def mol():
    # 5 heavy atoms: 20 J auxiliary functions, several GEMM tiles and a ragged tail
    return synth.make_molecule(seed=31, n_heavy=5, n_h=4)


@pytest.fixture(scope="module")
def refs(mol):
    out = {}
    for name, op in (("hyb", HYB), ("rsh", RSH)):
        out[name] = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc,
                              op["cx"], op["k_alpha"], op["k_beta"], op["omega"])
    return out


@pytest.mark.parametrize("which", ["hyb", "rsh"])
@pytest.mark.parametrize("m", [1, 13, 40])
def test_matvec_against_oracle(mol, refs, which, m):
    op = HYB if which == "hyb" else RSH
    c = _ctx(mol, j_ao=1, **op)
    c.build()
    X = synth.random_trial_block(500 + m, m, mol.nocc, mol.nvir)
    AX = c.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    assert _rel(AX, tda.matvec(refs[which], X)) < 1e-12


def test_same_operator_as_the_stored_route(mol):
    X = torch.from_numpy(synth.random_trial_block(77, 9, mol.nocc, mol.nvir)).cuda()
    out = []
    for j_ao in (0, 1):
        c = _ctx(mol, j_ao=j_ao, **RSH)
        c.build()
        out.append(c.matvec(X).cpu().numpy())
    assert _rel(out[1], out[0]) < 1e-13


def test_chunked_integrals_equal_one_chunk(mol):
    """Auxiliary chunks of one atom (4 functions): the integrals are generated in
    two passes per block instead of once."""
    X = torch.from_numpy(synth.random_trial_block(78, 5, mol.nocc, mol.nvir)).cuda()
    res = []
    d = None
    for chunk in (0, 1):
        c = _ctx(mol, j_ao=1, **HYB)
        if chunk:
            c.set_options(aux_chunk_bytes=4 * 8 * d.nao * d.nao)
        c.build()
        d = c.dims()
        res.append(c.matvec(X).cpu().numpy())
    assert _rel(res[1], res[0]) < 1e-13


@pytest.mark.parametrize("precision,tol", [(1, 2e-5), (2, 1e-12)])
def test_other_precisions(mol, refs, precision, tol):
    c = _ctx(mol, j_ao=1, precision=precision, **RSH)
    c.build()
    X = synth.random_trial_block(81, 7, mol.nocc, mol.nvir)
    AX = c.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    assert _rel(AX, tda.matvec(refs["rsh"], X)) < tol


def test_solve_matches_dense_eigh(mol, refs):
    w = np.linalg.eigvalsh(tda.explicit_A(refs["hyb"]))
    c = _ctx(mol, j_ao=1, nstates=5, tol=1e-8, **HYB)
    c.build()
    om, X, rs, info = c.solve()
    assert info.converged
    assert np.abs(om - w[:5]).max() < 1e-8


def test_no_stored_coulomb_tensor_and_memory_estimate(mol):
    tdarisp = _lib()
    c = _ctx(mol, j_ao=1, nstates=4, tol=1e-7, **HYB)
    est = c.memory()[2]
    c.build()
    with pytest.raises(tdarisp.TDARispError):
        c.tensor(0)
    c.solve()
    assert c.memory()[1] <= est, (c.memory(), est)   # the estimate bounds the real peak
