"""Three-centre integrals through every kernel path, against the oracle element
by element.

A chunk of at least 8 whole J atoms (or 8 auxiliary s functions) runs the
heavy pair classes one warp per four shell pairs with lanes over the atoms;
smaller chunks and chunks that do not start on an atom keep one thread per
shell pair.  One molecule with 12 heavy atoms covers both in one context: the
whole J range (12 atoms: a full lane tile and a ragged one), a 5-atom range,
a range that starts inside an atom, the whole K range (12 s functions) and a
K range of 5."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import ints, tda
from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HYB = dict(cx=0.25, k_alpha=1.0, k_beta=0.0, omega=0.0)
RSH = dict(cx=1.0, k_alpha=0.222, k_beta=0.778, omega=0.2)


@pytest.fixture(scope="module")
def mol():
    # 12 heavy + 10 H atoms: nao 218, 48 J and 12 K auxiliary functions; the
    # shell pairs of each class have 1 to 25 kept primitive pairs
    return synth.make_molecule(seed=13, n_heavy=12, n_h=10)


@pytest.mark.parametrize("which", ["hyb", "rsh"])
def test_int3c_every_path(mol, which):
    from paper_2603_29257_gb300 import tdarisp
    import __graft_entry__
    __graft_entry__.build()
    op = HYB if which == "hyb" else RSH
    torch.zeros(1, device="cuda")
    c = tdarisp.Context(**op)
    c.set_molecule_from(mol)
    d = c.dims()
    assert d.naux_j == 48 and d.naux_k == 12
    for w, kind, args, ranges in (
            (0, "J", (1.0, 0.0, 0.0), ((0, 48), (4, 20), (1, 30), (44, 4))),
            (1, "K", (op["k_alpha"], op["k_beta"], op["omega"]), ((0, 12), (3, 5)))):
        aux = tda.aux_shells(mol.Z, mol.xyz, mol.aux_exp, kind)
        ref = ints.int3c(mol.xyz, mol.shells, aux, *args)
        scale = np.abs(ref).max()
        for p0, n in ranges:
            out = torch.zeros((n, d.nao, d.nao), dtype=torch.float64, device="cuda")
            c.int3c(w, p0, n, out)
            err = np.abs(out.cpu().numpy() - ref[p0:p0 + n]).max() / scale
            print(kind, "functions", p0, "..", p0 + n, "max relative error %.2e" % err)
            assert err < 1e-12, (kind, p0, n, err)
    c.close()
