"""Davidson vectors spilled to pinned host memory (Sec. 3.3): forced by capping the
device rows and the host budget on the host side; the results must not change."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPTS = dict(cx=0.25, nstates=5, tol=1e-9, block=8)


@pytest.fixture(scope="module")
def mol():
    return synth.make_molecule(seed=21, n_heavy=4, n_h=4)


@pytest.fixture(scope="module")
def exact(mol):
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, 0.25)
    return np.linalg.eigvalsh(tda.explicit_A(f))[:5]


def _solve(mol, **kw):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    with tdarisp.Context(**{**OPTS, **kw}) as c:
        c.set_molecule_from(mol)
        c.build()
        return c.solve()


def test_no_spill_reference(mol, exact):
    om, X, rs, info = _solve(mol)
    assert info.converged and info.dev_rows == info.max_space and info.host_bytes_moved == 0
    assert np.abs(om - exact).max() < 1e-9


@pytest.mark.parametrize("dev_rows", [1, 3, 11])
def test_spilled_rows_give_the_same_result(mol, exact, dev_rows):
    om0, X0, _, info0 = _solve(mol)
    om, X, rs, info = _solve(mol, dav_dev_rows=dev_rows)
    assert info.converged
    assert info.dev_rows < info.max_space and info.host_bytes_moved > 0
    assert info.niter == info0.niter and info.nmatvec == info0.nmatvec
    assert np.abs(om - om0).max() < 1e-12
    ov = np.abs(np.einsum("kia,kia->k", X, X0))
    assert np.all(ov > 1 - 1e-10)
    assert np.abs(om - exact).max() < 1e-9


def test_host_budget_triggers_restarts(mol, exact):
    d = None
    nov = mol.nocc * mol.nvir
    # room for 20 spilled V/W rows in pinned memory beyond 4 device rows
    om, X, rs, info = _solve(mol, dav_dev_rows=4, host_budget=20 * 2 * nov * 8, max_iter=400)
    assert info.converged and info.max_space == 24 and info.nrestart > 0
    assert np.abs(om - exact).max() < 1e-9
