"""Bounded device waits of the tensor-core pipelines (TR_ETIMEOUT).

With tr_options.wait_test = 1 the tensor-core kernels load no operands, so
their first pipeline wait can only end by running out after wait_cycles (set
here to about a millisecond); nothing is faulted and nothing is left in
flight.  The call must return TR_ETIMEOUT, and the same context must work
normally once the switch is off again."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED, FP64_TC = 1, 2
SHORT = 2_000_000  # SM cycles, about 1 ms


def _ctx(mol, **opts):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(**opts)
    c.set_molecule_from(mol)
    return c


@pytest.fixture(scope="module")
def mol():
    return synth.make_molecule(seed=7, n_heavy=3, n_h=3)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", [MIXED, FP64_TC])
def test_matvec_wait_runs_out_then_context_recovers(mol, precision):
    from paper_2603_29257_gb300 import tdarisp
    c = _ctx(mol, precision=precision, cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)
    c.build()
    X = synth.random_trial_block(11, 4, mol.nocc, mol.nvir)
    ref = c.matvec(X)
    c.set_options(wait_cycles=SHORT, wait_test=1)
    with pytest.raises(tdarisp.TDARispError) as e:
        c.matvec(X)
    assert e.value.code == tdarisp.TR_ETIMEOUT
    c.set_options(wait_cycles=0, wait_test=0)
    assert _rel(c.matvec(X), ref) < 1e-14
    # a short limit alone does not trip a healthy pipeline
    c.set_options(wait_cycles=SHORT)
    assert _rel(c.matvec(X), ref) < 1e-14


def test_build_and_solve_waits_run_out_then_context_recovers(mol):
    from paper_2603_29257_gb300 import tdarisp
    opts = dict(precision=FP64_TC, cx=0.25, nstates=3, tol=1e-8)
    good = _ctx(mol, **opts)
    good.build()
    om_ref = good.solve(want_x=False)[0]

    c = _ctx(mol, wait_cycles=SHORT, wait_test=1, **opts)
    with pytest.raises(tdarisp.TDARispError) as e:
        c.build()                                   # sliced MO transforms
    assert e.value.code == tdarisp.TR_ETIMEOUT
    c.set_options(wait_test=0)
    c.build()
    c.set_options(wait_test=1)
    with pytest.raises(tdarisp.TDARispError) as e:
        c.solve(want_x=False)                       # sliced block products of the Davidson step
    assert e.value.code == tdarisp.TR_ETIMEOUT
    c.set_options(wait_cycles=0, wait_test=0)
    om = c.solve(want_x=False)[0]
    assert np.abs(om - om_ref).max() < 1e-12


def test_wait_options_are_checked(mol):
    from paper_2603_29257_gb300 import tdarisp
    c = _ctx(mol)
    with pytest.raises(tdarisp.TDARispError):
        c.set_options(wait_cycles=-1)
    c.set_options(wait_cycles=0)
    with pytest.raises(tdarisp.TDARispError):
        c.set_options(wait_test=2)
