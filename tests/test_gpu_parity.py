"""GPU path (through the C ABI) against the CPU oracle, element by element."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ints, tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HYB = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0)
RSH = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)


def _ctx(mol, **opts):
    from paper_2603_29257_gb300 import tdarisp
    import __graft_entry__
    __graft_entry__.build()
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(**opts)
    c.set_molecule_from(mol)
    return c


def _oracle(mol, op, window_ev=40.0, include_h=False):
    return tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc,
                     op["cx"], op["k_alpha"], op["k_beta"], op["omega"], window_ev=window_ev,
                     include_h=include_h)


@pytest.fixture(scope="module")
def small():
    return synth.make_molecule(seed=7, n_heavy=3, n_h=3)


@pytest.fixture(scope="module")
def small_ref(small):
    return {"hyb": _oracle(small, HYB), "rsh": _oracle(small, RSH)}


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_int2c_metric(small, which):
    op = HYB if which == "hyb" else RSH
    c = _ctx(small, **op)
    d = c.dims()
    for w, aux_kind, args in ((0, "J", (1.0, 0.0, 0.0)), (1, "K", (op["k_alpha"], op["k_beta"], op["omega"]))):
        aux = tda.aux_shells(small.Z, small.xyz, small.aux_exp, aux_kind)
        ref = ints.int2c(aux, *args)
        n = d.naux_j if w == 0 else d.naux_k
        out = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        c.int2c(w, out)
        assert _rel(out.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_int3c_all_blocks(small, which):
    op = HYB if which == "hyb" else RSH
    c = _ctx(small, **op)
    d = c.dims()
    for w, aux_kind, args in ((0, "J", (1.0, 0.0, 0.0)), (1, "K", (op["k_alpha"], op["k_beta"], op["omega"]))):
        aux = tda.aux_shells(small.Z, small.xyz, small.aux_exp, aux_kind)
        ref = ints.int3c(small.xyz, small.shells, aux, *args)
        n = d.naux_j if w == 0 else d.naux_k
        out = torch.zeros((n, d.nao, d.nao), dtype=torch.float64, device="cuda")
        c.int3c(w, 0, n, out)
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
        # a ragged chunk [1, n-1)
        part = torch.zeros((n - 2, d.nao, d.nao), dtype=torch.float64, device="cuda")
        c.int3c(w, 1, n - 2, part)
        assert np.abs(part.cpu().numpy() - ref[1:n - 1]).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_built_tensors(small, small_ref, which):
    op = HYB if which == "hyb" else RSH
    f = small_ref[which]
    c = _ctx(small, **op)
    c.build()
    d = c.dims()
    assert (d.nocc_k, d.nvir_k) == (len(f.occK), len(f.virK))
    assert d.occ_k0 == f.occK[0]
    assert _rel(c.tensor(0), f.Y) < 1e-12
    assert _rel(c.tensor(1), f.Tij) < 1e-11
    assert _rel(c.tensor(2), f.Tab) < 1e-12
    assert np.array_equal(c.tensor(3), f.D)


@pytest.mark.parametrize("which", ["hyb", "rsh"])
@pytest.mark.parametrize("m", [1, 7, 40])
def test_matvec_device(small, small_ref, which, m):
    op = HYB if which == "hyb" else RSH
    f = small_ref[which]
    c = _ctx(small, **op)
    c.build()
    X = synth.random_trial_block(100 + m, m, small.nocc, small.nvir)
    AX = c.matvec(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    ref = tda.matvec(f, X)
    assert _rel(AX.cpu().numpy(), ref) < 1e-12


def test_matvec_host_path_and_empty(small, small_ref):
    c = _ctx(small, **HYB)
    c.build()
    X = synth.random_trial_block(5, 3, small.nocc, small.nvir)
    assert _rel(c.matvec(X), tda.matvec(small_ref["hyb"], X)) < 1e-12
    assert c.matvec(np.zeros((0, small.nocc, small.nvir))).shape[0] == 0


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_solve_matches_dense_eigh(small, small_ref, which):
    op = HYB if which == "hyb" else RSH
    f = small_ref[which]
    A = tda.explicit_A(f)
    w, v = np.linalg.eigh(A)
    c = _ctx(small, nstates=6, tol=1e-8, **op)
    c.build()
    om, X, rs, info = c.solve()
    assert info.converged
    err = np.abs(om - w[:6])
    assert err.max() < 1e-8, err
    ov = np.abs(np.einsum("kn,nk->k", X.reshape(6, -1), v[:, :6]))
    assert np.all(ov > 1 - 1e-8)
    # sign convention and normalisation
    Xf = X.reshape(6, -1)
    assert np.allclose(np.linalg.norm(Xf, axis=1), 1.0, atol=1e-12)
    assert np.all(Xf[np.arange(6), np.argmax(np.abs(Xf), axis=1)] > 0)
    assert np.all(rs < 1e-8)


def test_solve_restart_path(small, small_ref):
    f = small_ref["hyb"]
    w = np.linalg.eigvalsh(tda.explicit_A(f))
    c = _ctx(small, nstates=4, block=4, max_space=9, max_iter=400, tol=1e-8, **HYB)
    c.build()
    om, X, rs, info = c.solve()
    assert info.converged and info.nrestart > 0
    assert np.abs(om - w[:4]).max() < 1e-9


@pytest.mark.parametrize("opts", [dict(window_ev=0.0), dict(cx=0.0), dict(window_ev=12.0)])
def test_variants(small, opts):
    op = dict(HYB)
    op.update({k: v for k, v in opts.items() if k in op})
    wev = opts.get("window_ev", 40.0)
    f = _oracle(small, op, window_ev=wev)
    c = _ctx(small, **{**HYB, **opts})
    c.build()
    X = synth.random_trial_block(9, 4, small.nocc, small.nvir)
    assert _rel(c.matvec(X), tda.matvec(f, X)) < 1e-12


def test_hydrogen_in_aux_basis(small):
    mol = synth.make_molecule(seed=7, n_heavy=3, n_h=3)
    mol.aux_exp = np.where(mol.Z == 1, 0.3, mol.aux_exp)
    f = _oracle(mol, HYB, include_h=True)
    c = _ctx(mol, aux_on_h=1, **HYB)
    c.build()
    assert c.dims().naux_j == 4 * len(mol.Z)
    X = synth.random_trial_block(2, 3, mol.nocc, mol.nvir)
    assert _rel(c.matvec(X), tda.matvec(f, X)) < 1e-12
    c2 = _ctx(mol, aux_on_h=0, **HYB)
    assert c2.dims().naux_j == 4 * int(np.sum(mol.Z > 1))
