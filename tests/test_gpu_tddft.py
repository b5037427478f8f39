"""Full TDDFT-risp on the GPU (tddft = 1; Sec. 2, Eqs. tddft and hessian; T_ia^P'
on the exchange window, Sec. 3.2): the window tensor, the (A + B) and (A - B)
products and the symplectic Davidson, element by element against the oracle,
plus properties at the 200-atom size where the oracle cannot follow."""
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


def _oracle(mol, op, window_ev=40.0):
    return tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, op["cx"], op["k_alpha"],
                     op["k_beta"], op["omega"], window_ev=window_ev, tddft=True)


@pytest.fixture(scope="module")
def mol():
    # 5 heavy atoms: 5 K and 20 J auxiliary functions, several GEMM tiles and a ragged tail
    return synth.make_molecule(seed=31, n_heavy=5, n_h=4)


@pytest.fixture(scope="module")
def refs(mol):
    return {"hyb": _oracle(mol, HYB), "rsh": _oracle(mol, RSH), "rsh_cut": _oracle(mol, RSH, 25.0)}


def test_window_tensor_gives_the_ib_ja_exchange(mol, refs):
    c = _ctx(mol, tddft=1, **RSH)
    c.build()
    t = c.tensor(4)
    f = refs["rsh"]
    blk = np.einsum("Pib,Pja->iajb", t, t)
    K = tda.exchange_ri_B(f).reshape(f.nocc, f.nvir, f.nocc, f.nvir)[np.ix_(f.occK, f.virK, f.occK, f.virK)]
    assert _rel(blk, K) < 1e-12


@pytest.mark.parametrize("which", ["hyb", "rsh", "rsh_cut"])
@pytest.mark.parametrize("m", [1, 13, 40])
@pytest.mark.parametrize("j_ao", [0, 1])
def test_products_against_oracle(mol, refs, which, m, j_ao):
    op = HYB if which == "hyb" else RSH
    win = 25.0 if which == "rsh_cut" else 40.0
    c = _ctx(mol, tddft=1, j_ao=j_ao, window_ev=win, **op)
    c.build()
    f = refs[which]
    if which == "rsh_cut":
        d = c.dims()
        assert d.nocc_k < d.nocc and d.nvir_k < d.nvir   # the window cuts both spaces
    X = synth.random_trial_block(900 + m, m, mol.nocc, mol.nvir)
    P, M = c.matvec_tddft(X)
    Pr, Mr = tda.matvec_pm(f, X)
    assert _rel(P, Pr) < 1e-12
    assert _rel(M, Mr) < 1e-12
    # A X on the same context is still the TDA product
    assert _rel(c.matvec(X), tda.matvec(f, X)) < 1e-12


@pytest.mark.parametrize("which", ["rsh", "rsh_cut"])
@pytest.mark.parametrize("j_ao", [0, 1])
def test_tensor_core_products_against_oracle(mol, refs, which, j_ao):
    """precision = TR_FP64_TC: the (ib|ja) stages as 7-slice tensor-core products
    (and the MO transforms, J and the TDA stages as in that form)."""
    win = 25.0 if which == "rsh_cut" else 40.0
    c = _ctx(mol, tddft=1, precision=2, j_ao=j_ao, window_ev=win, **RSH)
    c.build()
    X = synth.random_trial_block(700, 37, mol.nocc, mol.nvir)
    P, M = c.matvec_tddft(X)
    Pr, Mr = tda.matvec_pm(refs[which], X)
    assert _rel(P, Pr) < 1e-12
    assert _rel(M, Mr) < 1e-12


def test_tensor_core_solve_matches_dense_solve(mol, refs):
    c = _ctx(mol, tddft=1, precision=2, nstates=5, tol=1e-8, **RSH)
    c.build()
    om, XpY, XmY, rs, info = c.solve_tddft()
    assert info.converged
    _check_solution(refs["rsh"], om, XpY, XmY, rs, 1e-8)


def test_device_products_equal_host_products(mol):
    c = _ctx(mol, tddft=1, **RSH)
    c.build()
    X = synth.random_trial_block(5, 6, mol.nocc, mol.nvir)
    P, M = c.matvec_tddft(X)
    Pd, Md = c.matvec_tddft(torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(Pd.cpu().numpy(), P) and np.array_equal(Md.cpu().numpy(), M)


def _check_solution(f, om, XpY, XmY, rs, tol):
    w, Pd, Md = tda.tddft_dense(f, len(om))
    assert np.abs(om - w).max() < 1e-9
    n = f.nocc * f.nvir
    ApB, AmB = tda.explicit_ApB(f), tda.explicit_AmB(f)
    for k in range(len(om)):
        p, q = XpY[k].reshape(n), XmY[k].reshape(n)
        assert abs(p @ q - 1.0) < 1e-10
        r = np.sqrt(np.sum((ApB @ p - om[k] * q) ** 2) + np.sum((AmB @ q - om[k] * p) ** 2))
        assert r < 1.01 * tol and abs(r - rs[k]) < 1e-9
        # the same state as the dense solve (non-degenerate roots here)
        assert np.abs(p - Pd[k].reshape(n)).max() < 1e-5
        assert np.abs(q - Md[k].reshape(n)).max() < 1e-5


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_solve_matches_dense_solve(mol, refs, which):
    op = HYB if which == "hyb" else RSH
    c = _ctx(mol, tddft=1, nstates=5, tol=1e-8, **op)
    c.build()
    om, XpY, XmY, rs, info = c.solve_tddft()
    assert info.converged
    _check_solution(refs[which], om, XpY, XmY, rs, 1e-8)
    # tr_solve on the same context returns X+Y
    om2, X2, _, _ = c.solve()
    assert np.abs(om2 - om).max() < 1e-12 and np.abs(X2 - XpY).max() < 1e-10


def test_solve_with_restarts_and_spilled_rows(mol, refs):
    """Subspace capped at the smallest size (a restart basis plus one step) and
    only 10 rows of V, (A+B)V and (A-B)V on the device: restarts and host spill."""
    n = 3
    c = _ctx(mol, tddft=1, nstates=n, tol=1e-8, block=2 * n, max_space=4 * n, dav_dev_rows=10, **RSH)
    c.build()
    om, XpY, XmY, rs, info = c.solve_tddft()
    assert info.converged and info.nrestart >= 1 and info.dev_rows == 10 and info.host_bytes_moved > 0
    _check_solution(refs["rsh"], om, XpY, XmY, rs, 1e-8)


@pytest.mark.parametrize("case", ["hybrid", "rsh"])
@pytest.mark.parametrize("precision", [0, 2])
def test_24atom_against_golden(case, precision):
    """24-atom molecule (nov 7056): the five lowest roots against the oracle's dense
    solve stored by tests/golden/make_golden.py."""
    gold = json.load(open(os.path.join(HERE, "golden", "omega_tddft_24atom.json")))
    ref = np.array(gold["cases"][case]["omega"])
    op = HYB if case == "hybrid" else RSH
    c = _ctx(synth.molecule_24(), tddft=1, precision=precision, nstates=5, tol=1e-6, **op)
    c.build()
    om, XpY, XmY, rs, info = c.solve_tddft()
    err = np.abs(om - ref)
    assert info.converged and np.all(err < 1e-8), err


def test_oscillator_strengths_of_full_tddft_states(mol, refs):
    c = _ctx(mol, tddft=1, nstates=4, tol=1e-9, **RSH)
    c.build()
    om, XpY, XmY, rs, info = c.solve_tddft()
    f_gpu = c.oscillator_strengths(om, XpY)
    w, Pd, _ = tda.tddft_dense(refs["rsh"], 4)
    mu = tda.transition_dipoles(mol.xyz, mol.shells, mol.C, mol.nocc, Pd)
    f_ref = tda.oscillator_strengths(w, mu)
    assert np.abs(f_gpu - f_ref).max() < 1e-8 * max(1.0, np.abs(f_ref).max())


@pytest.mark.parametrize("precision", [0, 2])
def test_degenerate_cases(mol, precision):
    """No exchange (c_x = 0: A - B = D, A + B = D + 4 J), a window with no virtual
    orbital (no K term at all), no auxiliary functions (B = 0, Omega = e_a - e_i),
    and an empty block."""
    X = synth.random_trial_block(44, 5, mol.nocc, mol.nvir)
    for op, win in ((dict(RSH, cx=0.0), 40.0), (RSH, 1e-3)):
        f = _oracle(mol, op, win)
        c = _ctx(mol, tddft=1, precision=precision, window_ev=win, **op)
        c.build()
        P, M = c.matvec_tddft(X)
        Pr, Mr = tda.matvec_pm(f, X)
        assert _rel(P, Pr) < 1e-12 and _rel(M, Mr) < 1e-12
        if op["cx"] == 0.0:
            D = f.D.reshape(1, f.nocc, f.nvir)
            assert _rel(M, D * X) < 1e-13
        assert c.matvec_tddft(np.zeros((0, mol.nocc, mol.nvir)))[0].shape[0] == 0
    m0 = synth.make_molecule(seed=31, n_heavy=5, n_h=4)
    m0.aux_exp = np.zeros_like(m0.aux_exp)
    c = _ctx(m0, tddft=1, precision=precision, nstates=3, tol=1e-10, **RSH)
    c.build()
    om, XpY, XmY, rs, info = c.solve_tddft()
    D = np.sort((m0.eps[m0.nocc:][None, :] - m0.eps[:m0.nocc][:, None]).reshape(-1))
    assert info.converged and np.all(np.abs(om - D[:3]) <= 4e-15 * D[:3])


def test_invalid_uses_are_rejected(mol):
    tdarisp = _lib()
    with pytest.raises(tdarisp.TDARispError):
        tdarisp.Context(tddft=1, precision=1)
    c = _ctx(mol, **RSH)
    c.build()
    X = synth.random_trial_block(1, 2, mol.nocc, mol.nvir)
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_tddft(X)
    with pytest.raises(tdarisp.TDARispError):
        c.tensor(4)
    with pytest.raises(tdarisp.TDARispError):
        c.solve_tddft()
    t = _ctx(mol, tddft=1, nstates=2, **RSH)
    t.build()
    with pytest.raises(tdarisp.TDARispError):
        tdarisp.solve_batch([t])


def test_operator_properties_at_200_atoms():
    """The 200-atom RSH case (nov 577,600, window 380 x 567, 100 K auxiliary
    functions), FP64 pipe and tensor-core forms: (A + B) and (A - B) are symmetric
    on a random block, their half sum is the TDA product of the same context, and
    the two forms agree."""
    mol = synth.molecule_200()
    out = []
    for precision in (0, 2):
        c = _ctx(mol, tddft=1, precision=precision, **RSH)
        c.build()
        d = c.dims()
        X = torch.from_numpy(synth.random_trial_block(11, 4, d.nocc, d.nvir)).cuda()
        P, M = c.matvec_tddft(X)
        A = c.matvec(X)
        torch.cuda.synchronize()
        x, p, m, a = (t.reshape(4, -1) for t in (X, P, M, A))
        assert (0.5 * (p + m) - a).abs().max().item() < 1e-12 * a.abs().max().item()
        for S in (p, m, p - m):
            G = x @ S.T          # G[i][j] = x_i . (S x_j)
            assert (G - G.T).abs().max().item() < 1e-11 * G.abs().max().item()
        out.append((p.cpu(), m.cpu()))
        del c
    # the tensor-core form agrees with the FP64 pipe at this size
    for u, v in zip(out[0], out[1]):
        assert (u - v).abs().max().item() < 1e-12 * u.abs().max().item()
