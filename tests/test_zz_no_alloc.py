"""tr_matvec_noalloc -- the matrix-vector product for callers that cannot
allocate device memory (CUDA-graph capture, foreign allocators with a hard cap,
loops that cannot afford cudaMalloc's device synchronisation).  It takes all of
its scratch from a static device array; its output must match tr_matvec's on
two calls in a row (the second call reuses the array the first one left behind).

Collected last on purpose: it also has to pass after everything else has run in
the same process."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(mol, **opts):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(**opts)
    c.set_molecule_from(mol)
    c.build()
    return c


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("case", ["small", "no_aux", "chunked"])
def test_noalloc_matches_matvec_on_two_calls(case):
    if case == "small":
        mol = synth.make_molecule(seed=7, n_heavy=3, n_h=3)
        opts = dict(cx=0.25)
        ms = (5, 3)
    elif case == "no_aux":
        # no auxiliary functions at all: neither a Coulomb nor an exchange term,
        # the product is the diagonal alone (no scratch is needed per vector)
        mol = synth.make_molecule(seed=7, n_heavy=3, n_h=3)
        mol.aux_exp = np.zeros_like(mol.aux_exp)
        opts = dict(cx=0.25)
        ms = (5, 3)
    else:
        # window large enough that the static array holds one aux function of the
        # exchange intermediate at a time: exercises the chunked path
        mol = synth.make_molecule(seed=31, n_heavy=60, n_h=60)
        opts = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)
        ms = (40, 7)
    c = _ctx(mol, **opts)
    for call, m in enumerate(ms):
        X = torch.from_numpy(synth.random_trial_block(50 + call, m, mol.nocc, mol.nvir)).cuda()
        ref = c.matvec(X)
        out = torch.full_like(X, float("nan"))
        c.matvec_noalloc(X, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < 1e-12, (case, call)


def test_noalloc_rejects_bad_calls():
    from paper_2603_29257_gb300 import tdarisp
    mol = synth.make_molecule(seed=7, n_heavy=3, n_h=3)
    c = _ctx(mol)
    X = torch.zeros((2, mol.nocc, mol.nvir), dtype=torch.float64, device="cuda")
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_noalloc(X, X)  # output overlaps input
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_noalloc(X.float(), torch.empty_like(X).float())  # not float64
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_noalloc(X[:, :, :-1], torch.empty_like(X)[:, :, :-1])  # wrong shape
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_noalloc(X, torch.empty((2, mol.nocc * mol.nvir), dtype=torch.float64, device="cuda"))
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_noalloc(X, torch.empty_like(X).transpose(1, 2).contiguous().transpose(1, 2))  # strided out
    with pytest.raises(tdarisp.TDARispError):
        c.matvec_noalloc(X.cpu(), torch.empty_like(X))  # host input
