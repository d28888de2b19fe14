"""Pins of the oracle's dense eigensolve of the projected Hamiltonian
(Alg. 1 step 4, ``oracle.chefsi.subspace_eigh``) and of the planted-spectrum
inputs the GPU eigensolver is tested on, against facts fixed by the
mathematics rather than by the oracle itself:

* a 2 x 2 matrix against the closed form of its eigenvalues and eigenvectors;
* a diagonal matrix: its sorted diagonal and the unit vectors, permuted;
* a planted spectrum Q diag(lam) Q^T: lam recovered to rounding, and the
  eigenvectors are Q's columns (up to sign) where lam is well separated;
* only the lower triangle is read (the upper one holds garbage);
* repeated eigenvalues: the projector onto the group's eigenvectors equals
  Q_g Q_g^T of the planted group, whatever basis is returned.
"""
import numpy as np
import pytest

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

U = 2.0 ** -53


def test_two_by_two_closed_form():
    a, b, c = 0.7, -0.3, 2.1
    w, V = O.subspace_eigh(np.array([[a, 99.0], [b, c]]))
    mid, rad = 0.5 * (a + c), np.hypot(0.5 * (a - c), b)
    assert np.allclose(w, [mid - rad, mid + rad], rtol=0, atol=4 * U * 3)
    for lam, v in zip(w, V):
        # (A - lam I) v = 0 with v = (b, lam - a) / norm
        ref = np.array([b, lam - a]) / np.hypot(b, lam - a)
        assert abs(abs(ref @ v) - 1.0) < 1e-15


def test_diagonal_matrix():
    d = np.array([3.0, -1.0, 2.0, 0.5])
    w, V = O.subspace_eigh(np.diag(d))
    order = np.argsort(d)
    assert np.array_equal(w, d[order])
    assert np.array_equal(np.abs(V), np.eye(4)[order])


def test_planted_spectrum_and_lower_triangle_only():
    lam = G.clustered_spectrum(300, seed=3)
    A = G.make_planted_symmetric(lam, seed=3)
    assert np.array_equal(A, A.T)
    Ag = np.tril(A) + np.triu(np.full_like(A, 1e3), 1)  # garbage above the diagonal
    w, V = O.subspace_eigh(Ag)
    norm = np.abs(lam).max()
    assert np.abs(w - lam).max() <= 64 * U * norm * 300 ** 0.5
    assert np.abs(V @ V.T - np.eye(300)).max() <= 64 * U * 300 ** 0.5
    # eigenvectors = planted directions (up to sign) where the gaps are wide
    Q = G._orthonormal_columns(np.random.default_rng(3 + 4), 300, 300)
    gaps = np.minimum(np.diff(lam, prepend=-np.inf), np.diff(lam, append=np.inf))
    wide = gaps > 1e-3
    cos = np.abs(np.sum(V * Q.T, axis=1))
    assert wide.sum() > 100
    assert np.abs(1.0 - cos[wide]).max() < 1e-10


def test_repeated_eigenvalues_projector():
    lam = G.clustered_spectrum(200, groups=[(0.5, 6, 0.0), (1.2, 3, 0.0)], seed=5)
    A = G.make_planted_symmetric(lam, seed=5)
    w, V = O.subspace_eigh(A)
    Q = G._orthonormal_columns(np.random.default_rng(5 + 4), 200, 200)
    for centre, size in ((0.5, 6), (1.2, 3)):
        sel_w = np.abs(w - centre) < 1e-9
        sel_l = lam == centre
        assert sel_w.sum() == size and sel_l.sum() == size
        P = V[sel_w].T @ V[sel_w]
        P_ref = Q[:, sel_l] @ Q[:, sel_l].T
        assert np.abs(P - P_ref).max() < 1e-12


@pytest.mark.parametrize("groups", [[], [(0.0, 5, 1e-9)], [(1.0, 40, 0.0)]])
def test_clustered_spectrum_generator(groups):
    lam = G.clustered_spectrum(120, groups=groups, seed=1)
    assert lam.shape == (120,) and np.all(np.diff(lam) >= 0)
    for centre, size, spread in groups:
        assert np.sum(np.abs(lam - centre) <= 10 * spread) >= size


# ---- the Cholesky factor and its inverse (Alg. 1 step 3), oracle.cholesky_inverse

def test_cholesky_two_by_two_closed_form():
    a, b, c = 4.0, 2.0, 5.0          # S = [[4, 2], [2, 5]] = L L^T, L = [[2, 0], [1, 2]]
    L, Li = O.cholesky_inverse(np.array([[a, -7.0], [b, c]]))
    assert np.allclose(L, [[2.0, 0.0], [1.0, 2.0]], rtol=0, atol=1e-15)
    assert np.allclose(Li, [[0.5, 0.0], [-0.25, 0.5]], rtol=0, atol=1e-15)


def test_cholesky_recovers_the_planted_factor():
    S, Lp = G.planted_cholesky(300, cond=1e4, seed=2)
    L, Li = O.cholesky_inverse(S)
    # the factor with a positive diagonal is unique
    assert np.abs(L - Lp).max() <= 1e-10 * np.abs(Lp).max()
    assert np.abs(Li @ L - np.eye(300)).max() <= 1e-12
    assert np.array_equal(np.triu(Li, 1), np.zeros((300, 300)))


def test_cholesky_rejects_an_indefinite_matrix():
    S, _ = G.planted_cholesky(50, negative_at=17, seed=3)
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky_inverse(S)
    # the leading 17 x 17 block is still positive definite, the 18 x 18 one is not
    O.cholesky_inverse(S[:17, :17])
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky_inverse(S[:18, :18])
