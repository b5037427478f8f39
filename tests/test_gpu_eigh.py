"""The Davidson driver's subspace eigensolver (tr_subspace_eigh: Householder
tridiagonalisation, Sturm multisection, inverse iteration in one thread-block
cluster) against LAPACK (numpy.linalg.eigh): eigenvalues, residuals and
orthonormality, on random, clustered, degenerate and already-reduced matrices."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_29257_gb300 import tdarisp
    torch.zeros(1, device="cuda")
    return tdarisp.Context()


def _check(ctx, H, nev, wtol=1e-12, rtol=1e-10):
    w, Y = ctx.subspace_eigh(H, nev)
    ref = np.linalg.eigvalsh(H)[:nev]
    scale = max(np.abs(np.linalg.eigvalsh(H)).max(), 1e-300)
    assert np.abs(w - ref).max() <= wtol * scale, np.abs(w - ref).max() / scale
    R = H @ Y - Y * w[None, :]
    assert np.abs(R).max() <= rtol * scale, np.abs(R).max() / scale
    G = Y.T @ Y
    assert np.abs(G - np.eye(nev)).max() <= rtol, np.abs(G - np.eye(nev)).max()
    return w, Y


def _sym(rng, k):
    A = rng.standard_normal((k, k))
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("k,nev", [(1, 1), (2, 1), (2, 2), (3, 2), (17, 5), (64, 15), (300, 15), (301, 30),
                                   (640, 64)])
def test_random(ctx, k, nev):
    rng = np.random.default_rng(k * 1000 + nev)
    _check(ctx, _sym(rng, k), nev)


def test_davidson_shaped(ctx):
    """Diagonal Ritz block plus coupling to a new block, positive spectrum of
    excitation-energy size (0.1 - 4 Ha), as in a Davidson iteration."""
    rng = np.random.default_rng(5)
    k0, p = 150, 30
    H = np.zeros((k0 + p, k0 + p))
    H[:k0, :k0] = np.diag(np.sort(rng.uniform(0.1, 4.0, k0)))
    B = 1e-3 * rng.standard_normal((k0, p))
    C = _sym(rng, p) * 0.01 + np.diag(rng.uniform(0.1, 4.0, p))
    H[:k0, k0:] = B
    H[k0:, :k0] = B.T
    H[k0:, k0:] = C
    _check(ctx, H, 15)


@pytest.mark.parametrize("gap", [0.0, 1e-12, 1e-9, 1e-6])
def test_clustered(ctx, gap):
    """Repeated and nearly repeated eigenvalues: the vectors of a cluster must
    come out orthonormal and span the invariant subspace."""
    rng = np.random.default_rng(11)
    k = 120
    lam = np.sort(rng.uniform(1.0, 3.0, k))
    lam[:4] = 0.5 + gap * np.arange(4)      # a cluster of four at the bottom
    lam[7:10] = 0.9 + gap * np.arange(3)    # and one of three inside the wanted range
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    H = (Q * lam[None, :]) @ Q.T
    H = 0.5 * (H + H.T)
    w, Y = _check(ctx, H, 12)
    # the cluster's vectors span the exact eigenspace
    P = Q[:, :4]
    assert np.linalg.norm(Y[:, :4] - P @ (P.T @ Y[:, :4])) < 1e-9


def test_already_reduced(ctx):
    """Diagonal and tridiagonal inputs (reflectors with tau = 0), unsorted."""
    rng = np.random.default_rng(3)
    d = rng.uniform(-2, 2, 50)
    _check(ctx, np.diag(d), 10)
    T = np.diag(d) + np.diag(rng.uniform(-1, 1, 49), 1)
    T = T + np.triu(T, 1).T
    _check(ctx, T, 10)
    # a block-diagonal matrix with a zero block between (exact zero columns)
    H = np.zeros((40, 40))
    H[:20, :20] = _sym(rng, 20)
    H[30:, 30:] = _sym(rng, 10)
    _check(ctx, H, 25)


def test_rejects_bad_arguments(ctx):
    from paper_2603_29257_gb300 import tdarisp
    with pytest.raises(tdarisp.TDARispError):
        ctx.subspace_eigh(np.eye(3), 4)
