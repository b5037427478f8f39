"""Batched form: several molecules' Davidson solves in lockstep with one CUDA-graph
launch of all products per step (tr_solve_batch).  Each result must equal the
molecule solved alone and the oracle's dense eigh."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(3, 3), (5, 4), (2, 5), (7, 6), (4, 0)]


@pytest.fixture(scope="module")
def mols():
    out = []
    for k, (nh, nH) in enumerate(SIZES):
        m = synth.make_molecule(seed=500 + k, n_heavy=nh, n_h=nH)
        f = tda.build(m.Z, m.xyz, m.shells, m.aux_exp, m.C, m.eps, m.nocc, 0.25)
        out.append((m, np.linalg.eigvalsh(tda.explicit_A(f))[:6]))
    return out


def _ctxs(mols, precision, nstates=6):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    cs = []
    for k, (m, _) in enumerate(mols):
        c = tdarisp.Context(nstates=nstates - (k % 2), tol=1e-7, cx=0.25, precision=precision)
        c.set_molecule_from(m)
        c.build()
        cs.append(c)
    return cs


@pytest.mark.parametrize("precision,tol_alone,tol_ref", [(0, 1e-12, 1e-8), (1, 1e-8, 1e-5)])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_equals_alone_and_oracle(mols, precision, tol_alone, tol_ref, autotune):
    from paper_2603_29257_gb300 import tdarisp
    cs = _ctxs(mols, precision)
    res = tdarisp.solve_batch(cs, autotune=autotune)
    for k, ((m, w), c, (om, X, rs, info)) in enumerate(zip(mols, cs, res)):
        assert info.converged, k
        n = len(om)
        assert np.abs(om - w[:n]).max() < tol_ref, (k, np.abs(om - w[:n]))
        alone = tdarisp.Context(nstates=c.options.nstates, tol=1e-7, cx=0.25, precision=precision)
        alone.set_molecule_from(m)
        alone.build()
        om1, X1, rs1, info1 = alone.solve()
        assert np.abs(om - om1).max() < tol_alone, (k, np.abs(om - om1).max())
        ov = np.abs(np.einsum("kia,kia->k", X, X1))
        assert np.all(ov > 1 - 1e-6), (k, ov)


@pytest.mark.parametrize("precision", [0, 1])
def test_concurrent_builds_equal_sequential(mols, precision):
    """tr_build_batch (host threads, a stream per context) gives the tensors and
    the solves of contexts built one by one."""
    from paper_2603_29257_gb300 import tdarisp
    seq = _ctxs(mols, precision)
    par = []
    for k, (m, _) in enumerate(mols):
        c = tdarisp.Context(nstates=6 - (k % 2), tol=1e-7, cx=0.25, precision=precision)
        c.set_molecule_from(m)
        par.append(c)
    tdarisp.build_batch(par, nthreads=3)
    for a, b in zip(seq, par):
        for w in range(4):
            ta, tb = a.tensor(w), b.tensor(w)
            assert ta.shape == tb.shape
            assert np.array_equal(ta, tb), w
        assert np.array_equal(a.solve()[0], b.solve()[0])
