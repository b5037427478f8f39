"""MO transforms on the bf16 tensor cores by the Ozaki splitting scheme
(xform_slices = S): the FP64 tensors (P|ia), T_ij, T_ab against the FP64
oracle for several S, the error falling with S as 2^(-8S); with 7 slices the
FP64 form still meets the FP64 bar on the golden excitation energies."""
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


def bound(S):
    """Relative error bound (to the tensor's largest element) for S slices.
    Each operand element keeps its row's leading 7 + 8 (S-1) bits, an error of
    at most 2^(-8S) of the row's largest element; through the two products and
    the cancellation in the AO-to-MO sums this was observed as ~2^(14-8S) on
    these molecules.  Bound: 4x that, plus FP64 rounding of the reference."""
    return 2.0 ** (16 - 8 * S) + 2e-12


def _ctx(mol, precision=0, **opts):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(precision=precision, **opts)
    c.set_molecule_from(mol)
    c.build()
    return c


@pytest.fixture(scope="module")
def mid():
    # 68 atoms, nao 646: 21 K blocks of 32 with a ragged tail (several exact
    # chunks for every S), 129 window occupied rows (two M tiles), 11 N tiles
    mol = synth.make_molecule(seed=41, n_heavy=34, n_h=34)
    f = tda.build(mol.Z, mol.xyz, mol.shells, mol.aux_exp, mol.C, mol.eps, mol.nocc, RSH["cx"],
                  RSH["k_alpha"], RSH["k_beta"], RSH["omega"])
    return mol, f


def test_sliced_tensors_against_oracle(mid):
    mol, f = mid
    errs = {}
    for S in (3, 4, 5, 7):
        c = _ctx(mol, xform_slices=S, **RSH)
        e = []
        for which, ref in ((0, f.Y), (1, f.Tij), (2, f.Tab)):
            got = c.tensor(which)
            assert got.shape == ref.shape
            e.append(np.abs(got - ref).max() / np.abs(ref).max())
        errs[S] = max(e)
        print("slices", S, "relative errors (P|ia), T_ij, T_ab:", e)
        c.close()
    for S, e in errs.items():
        assert e < bound(S), (S, e)
    assert errs[7] < errs[5] < errs[3]


def test_fp64_pipe_and_sliced_agree(mid):
    """xform_slices = -1 (FP64 pipe) against 7 slices, element by element."""
    mol, _ = mid
    a = _ctx(mol, xform_slices=-1, **HYB)
    b = _ctx(mol, xform_slices=7, **HYB)
    for which in (0, 1, 2):
        ta, tb = a.tensor(which), b.tensor(which)
        assert np.abs(ta - tb).max() < 1e-12 * np.abs(ta).max()


@pytest.mark.parametrize("case", ["hybrid", "rsh"])
def test_fp64_form_with_7_slices_meets_golden(case):
    gold = json.load(open(os.path.join(HERE, "golden", "omega_24atom.json")))
    ref = np.array(gold["cases"][case]["omega"])
    op = HYB if case == "hybrid" else RSH
    c = _ctx(synth.molecule_24(), nstates=5, tol=1e-6, xform_slices=7, **op)
    om, X, rs, info = c.solve()
    err = np.abs(om - ref)
    print("per-state |dOmega| (Ha), FP64 form, 7 slices, %s:" % case, err)
    assert info.converged and np.all(err < 1e-8), err


def test_mixed_default_uses_slices_and_meets_bar(mid):
    """The reduced-precision form builds its tensors on the tensor cores (no
    FP64-pipe transform kernels) and stays within 1e-5 Ha of the FP64 form."""
    mol, _ = mid
    c = _ctx(mol, precision=1, nstates=4, tol=1e-6, **RSH)
    c.profile(True)
    c.build()
    names = set(c.profile_get())
    assert "xform_J1_oz" in names and "xform_J1" not in names, names
    om, X, rs, info = c.solve()
    ref = _ctx(mol, precision=0, nstates=4, tol=1e-6, **RSH)
    om0, X0, rs0, info0 = ref.solve()
    assert info.converged and info0.converged
    err = np.abs(om - om0)
    print("per-state |dOmega| (Ha), mixed with sliced transforms vs FP64 form:", err)
    assert np.all(err < 1e-5), err
