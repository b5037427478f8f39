"""The timed 200-atom case against the oracle, per state and element by element.

tests/golden/omega_200atom_rsh.json holds, from the CPU oracle alone
(tests/golden/make_golden.py cfg2): the 15 lowest excitation energies of the
200-atom range-separated case (Sec. 2 Eq. TDA-risp with Sec. 3.2 Eqs. RSH and
K_mia_RSH) from the oracle's block Davidson (Sec. 3.3) at residual 1e-7, and
its A X for two seeded trial vectors on one whole occupied row each plus 128
seeded (i, a) entries.  The GPU runs the configuration bench.py times (15
states, block 30) in each form: the FP64 pipe, FP64 on the tensor cores
(7-slice products) and the reduced-precision form.  Bars: FP64 forms 1e-8 Ha
per state and 1e-12 of the largest |A X| per entry; reduced precision 1e-5 Ha
per state and 1e-5 of the largest |A X| per entry.
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RSH = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)
# precision -> (per-state Omega bar in Ha, A X bar relative to max |A X|, solver residual)
FORMS = {0: (1e-8, 1e-12, 1e-7), 2: (1e-8, 1e-12, 1e-7), 1: (1e-5, 1e-5, 1e-5)}


@pytest.fixture(scope="module")
def gold():
    with open(os.path.join(HERE, "golden", "omega_200atom_rsh.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def mol():
    return synth.molecule_200()


def _ctx(mol, **opts):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(**opts)
    c.set_molecule_from(mol)
    return c


def _sample_positions(nocc, nvir, gold):
    ii, aa = np.array(gold["ax"]["samples"]["i"]), np.array(gold["ax"]["samples"]["a"])
    assert ii.max() < nocc and aa.max() < nvir
    return ii, aa


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_200atom_matvec_against_oracle_samples(mol, gold, precision):
    """A X of the two seeded vectors: one whole occupied row and 128 seeded
    entries per vector, against the oracle's matrix-free product."""
    _, bar, _ = FORMS[precision]
    ax = gold["ax"]
    X = synth.random_trial_block(ax["x_seed"], ax["m"], mol.nocc, mol.nvir)
    with _ctx(mol, nstates=15, block=30, precision=precision, **RSH) as c:
        c.build()
        AX = c.matvec(torch.from_numpy(X).cuda()).cpu().numpy()
    ii, aa = _sample_positions(mol.nocc, mol.nvir, gold)
    worst = 0.0
    for k in range(ax["m"]):
        scale = ax["max_abs"][k]
        row = ax["rows"][k]
        assert row["vector"] == k
        e_row = np.abs(AX[k, row["i"]] - np.array(row["values"])).max() / scale
        e_smp = np.abs(AX[k, ii, aa] - np.array(ax["samples"]["values"][k])).max() / scale
        # the largest element itself is a property of the whole product
        e_max = abs(np.abs(AX[k]).max() - scale) / scale
        worst = max(worst, e_row, e_smp, e_max)
    print("precision %d: A X relative error against the oracle %.2e" % (precision, worst))
    assert worst < bar, worst


@pytest.mark.parametrize("precision", [0, 2, 1])
def test_200atom_omega_against_oracle(mol, gold, precision):
    """The 15 lowest roots per state against the oracle's Davidson roots."""
    bar, _, tol = FORMS[precision]
    ref = np.array(gold["omega"])
    assert len(ref) == 15
    with _ctx(mol, nstates=15, block=30, tol=tol, precision=precision, **RSH) as c:
        c.build()
        om, _, rs, info = c.solve(want_x=False)
    err = np.abs(om - ref)
    print("precision %d: per-state |dOmega| against the oracle (Ha):" % precision,
          " ".join("%.1e" % e for e in err), "| %d iterations, %d matvecs" % (info.niter, info.nmatvec))
    assert info.converged
    assert np.all(err < bar), err
    if precision in (0, 2):
        # the same Davidson (guess, preconditioner, Gram-Schmidt, restart) in FP64-level
        # arithmetic takes the oracle's path: same iterations and products
        assert (info.niter, info.nmatvec) == (gold["niter"], gold["nmatvec"])
