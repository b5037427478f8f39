"""The seeded input generator (no TDA-risp arithmetic): long chains, the device
path of its dense linear algebra, and the molecules the stored golden values
were written for."""
from __future__ import annotations

import hashlib

import numpy as np
import pytest

from paper_2603_29257_gb300 import synth

torch = pytest.importorskip("torch")


def test_long_chain_keeps_its_distance_rules():
    """750 heavy atoms: the chain end gets trapped and regrows; every bond and
    every non-bonded distance still follows the stated rules (Angstrom)."""
    rng = np.random.default_rng(5499)
    Z, xyz = synth.chain_geometry(rng, 750, 750)
    heavy = xyz[:750]
    bonds = np.linalg.norm(np.diff(heavy, axis=0), axis=1)
    assert bonds.min() >= 1.35 - 1e-12 and bonds.max() <= 1.45 + 1e-12
    d = np.linalg.norm(heavy[:, None, :] - heavy[None, :, :], axis=2)
    far = np.abs(np.arange(750)[:, None] - np.arange(750)[None, :]) >= 2
    assert d[far].min() >= 2.0 - 1e-12
    hyd = xyz[750:]
    dh = np.linalg.norm(hyd[:, None, :] - heavy[None, :, :], axis=2)
    parent = np.arange(750) % 750
    assert np.allclose(dh[np.arange(750), parent], np.clip(dh[np.arange(750), parent], 1.06, 1.12))
    dh[np.arange(750), parent] = np.inf
    assert dh.min() >= 1.5 - 1e-12
    hh = np.linalg.norm(hyd[:, None, :] - hyd[None, :, :], axis=2) + np.eye(750) * 9.0
    assert hh.min() >= 1.4 - 1e-12


def test_torch_path_gives_the_same_molecule():
    """The overlap, eigendecomposition, QR and products run with torch (here on
    the host) from the same random numbers: same geometry and basis, the same
    orbitals up to rounding, and orthonormal in the numpy overlap."""
    a = synth.make_molecule(3, 12, 12)
    b = synth.make_molecule(3, 12, 12, device="cpu")
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.eps, b.eps)
    assert all(np.array_equal(x.exps, y.exps) and np.array_equal(x.coefs, y.coefs) for x, y in zip(a.shells, b.shells))
    S = synth.overlap_matrix(a.xyz, a.shells)
    St = synth.overlap_matrix(a.xyz, a.shells, "cpu").numpy()
    assert np.abs(S - St).max() < 1e-14
    assert np.abs(a.C - b.C).max() < 1e-9
    assert np.abs(b.C.T @ S @ b.C - np.eye(a.nao)).max() < 1e-12


def test_golden_molecules_are_unchanged():
    """The 24-atom molecule of the stored oracle values is generated bit for bit
    as when the values were written (hash of geometry, orbitals and energies)."""
    m = synth.molecule_24()
    h = hashlib.md5(m.xyz.tobytes() + m.C.tobytes() + m.eps.tobytes()).hexdigest()
    assert h == "c42c7ce616c0a3d467b6de533cec33c3"
