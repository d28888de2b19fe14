"""Pins of the oracle's re-alignment (Eqs. basis_rotation_1-3), pattern density
blocks (Eq. densitymatrix) and CholeskyQR2 / shifted CholeskyQR3, against
results fixed independently of the oracle's code: the global block-diagonal
product, least-squares projection (numpy lstsq), Householder QR, the dense
density matrix, and invariances."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G


def basis_case(seed=0, delta=0.05):
    nb_old = [4, 7, 5, 6]
    nb_new = [5, 7, 3, 6]
    nr = [20, 30, 9, 12]
    Vo, Vn = G.make_basis_pair(nb_old, nb_new, nr, delta=delta, seed=seed)
    X = np.random.default_rng(seed + 10).standard_normal((sum(nb_old), 11))
    return nb_old, nb_new, nr, Vo, Vn, X


def test_realign_equals_global_projection():
    """Eq. basis_rotation_1 with V assembled block-diagonally (disjoint supports)
    equals the per-element form of Eq. basis_rotation_3."""
    _, _, _, Vo, Vn, X = basis_case()
    Vo_g, Vn_g = sla.block_diag(*Vo), sla.block_diag(*Vn)
    ref = Vn_g.T @ (Vo_g @ X)
    got = O.realign(Vo, Vn, X)
    assert got.shape == ref.shape == (sum(v.shape[1] for v in Vn), X.shape[1])
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_realign_is_least_squares_projection():
    """With orthonormal new basis columns the re-aligned coefficients are the
    least-squares (l2) fit of the old function in the new basis, and the
    residual is orthogonal to the new basis."""
    nb_old, _, _, Vo, Vn, X = basis_case(seed=3)
    got = O.realign(Vo, Vn, X)
    off_o = np.concatenate([[0], np.cumsum(nb_old)])
    off_n = np.concatenate([[0], np.cumsum([v.shape[1] for v in Vn])])
    for K in range(len(Vo)):
        f = Vo[K] @ X[off_o[K]:off_o[K + 1]]
        ls = np.linalg.lstsq(Vn[K], f, rcond=None)[0]
        xk = got[off_n[K]:off_n[K + 1]]
        assert np.max(np.abs(xk - ls)) <= 1e-12 * max(1.0, np.max(np.abs(ls)))
        assert np.max(np.abs(Vn[K].T @ (f - Vn[K] @ xk))) <= 1e-12 * np.max(np.abs(f))


def test_realign_identity_and_rotated_basis():
    """Unchanged basis: coefficients unchanged. Same span, rotated: X' = Q^T X
    and the represented functions are preserved exactly."""
    nb_old, _, _, Vo, _, X = basis_case(seed=5)
    assert np.max(np.abs(O.realign(Vo, Vo, X) - X)) <= 1e-14 * np.max(np.abs(X))
    rng = np.random.default_rng(7)
    Qs = [np.linalg.qr(rng.standard_normal((n, n)))[0] for n in nb_old]
    Vr = [v @ q for v, q in zip(Vo, Qs)]
    got = O.realign(Vo, Vr, X)
    ref = np.vstack([q.T @ X[a:b] for q, a, b in zip(Qs, np.cumsum([0] + nb_old[:-1]), np.cumsum(nb_old))])
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(sla.block_diag(*Vr) @ got - sla.block_diag(*Vo) @ X)) <= 1e-13 * np.max(np.abs(X))


def test_realign_pins_catch_planted_mistakes():
    """A transposed overlap (V_old^T V_new) or the new basis on both sides fails
    the least-squares pin."""
    nb = [6, 6, 6]
    Vo, Vn = G.make_basis_pair(nb, nb, [15, 15, 15], delta=0.3, seed=2)
    X = np.random.default_rng(1).standard_normal((18, 4))
    ls = np.vstack([np.linalg.lstsq(Vn[K], Vo[K] @ X[6 * K:6 * K + 6], rcond=None)[0] for K in range(3)])
    transposed = np.vstack([(Vo[K].T @ Vn[K]) @ X[6 * K:6 * K + 6] for K in range(3)])
    same = O.realign(Vn, Vn, X)
    assert np.max(np.abs(O.realign(Vo, Vn, X) - ls)) <= 1e-12 * np.max(np.abs(ls))
    assert np.max(np.abs(transposed - ls)) > 1e-3
    assert np.max(np.abs(same - ls)) > 1e-3


def test_realign_rejects_mismatched_rows():
    _, _, _, Vo, Vn, X = basis_case()
    with pytest.raises(ValueError):
        O.realign(Vo, Vn, X[:-1])


def test_density_pattern_blocks_match_dense_density_matrix():
    cfg = G.ProblemConfig(name="pd", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                          nb=(4, 7), Ns=9, m=3, Ne=8.0, seed=4)
    H, X0, _, Ns, _ = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    X = X0.T
    f = np.random.default_rng(2).uniform(0, 1, Ns)
    P = X @ np.diag(f) @ X.T
    blocks = O.density_pattern_blocks(Ho, X, f)
    i = 0
    diag = O.density_blocks(Ho, X, f)
    where = {}
    for K in range(Ho.M):
        for Kp, _ in Ho.neighbours(K):
            ref = P[Ho.rows(K)][:, Ho.rows(Kp)]
            assert np.max(np.abs(blocks[i] - ref)) <= 1e-13 * np.max(np.abs(P))
            if Kp == K:
                assert np.max(np.abs(blocks[i] - diag[K])) <= 1e-13 * np.max(np.abs(P))
            where[(K, Kp)] = i
            i += 1
    for (K, Kp), e in where.items():
        assert np.max(np.abs(blocks[e] - blocks[where[(Kp, K)]].T)) <= 1e-13 * np.max(np.abs(P))


def ill_conditioned(n, ns, kappa, seed=0):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((n, ns)))[0]
    V = np.linalg.qr(rng.standard_normal((ns, ns)))[0]
    return U @ np.diag(np.geomspace(1.0, 1.0 / kappa, ns)) @ V.T


def householder_q(Y):
    Q, R = np.linalg.qr(Y)
    return Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_cholesky_qr2_orthonormal_and_matches_householder(kappa):
    Y = ill_conditioned(300, 20, kappa)
    Q, U = O.cholesky_qr2(Y)
    assert np.max(np.abs(Q.T @ Q - np.eye(20))) <= 1e-14
    assert np.max(np.abs(Q @ U - Y)) <= 1e-14 * np.max(np.abs(Y))
    assert np.allclose(U, np.triu(U)) and np.all(np.diag(U) > 0)
    assert np.max(np.abs(Q - householder_q(Y))) <= 1e-15 * kappa * 100
    if kappa >= 1e6:  # one Cholesky-QR pass loses orthogonality as kappa^2 u
        Q1, _, _ = O.cholesky_qr(Y)
        assert np.max(np.abs(Q1.T @ Q1 - np.eye(20))) > 1e-6


def test_shifted_cholesky_qr3_where_cholesky_fails():
    Y = ill_conditioned(400, 24, 1e12, seed=3)
    try:
        Q1, _, _ = O.cholesky_qr(Y)
        plain_ok = np.max(np.abs(Q1.T @ Q1 - np.eye(24))) < 1e-2
    except np.linalg.LinAlgError:
        plain_ok = False
    assert not plain_ok
    Q, U = O.shifted_cholesky_qr3(Y)
    assert np.max(np.abs(Q.T @ Q - np.eye(24))) <= 1e-14
    assert np.max(np.abs(Q @ U - Y)) <= 1e-14 * np.max(np.abs(Y))
    Qh = householder_q(Y)
    assert np.max(np.abs(Q @ Q.T - Qh @ Qh.T)) <= 1e-2   # same span up to kappa u
    # moderate conditioning: the same Q as one Cholesky-QR pass, whose own error is ~kappa^2 u
    Yw = ill_conditioned(200, 12, 1e3, seed=4)
    assert np.max(np.abs(O.shifted_cholesky_qr3(Yw)[0] - O.cholesky_qr(Yw)[0])) <= 10 * 1e3 ** 2 * 2.0 ** -53


def test_basis_pair_generator_properties():
    """Synthetic bases: orthonormal columns of the stated sizes, the new basis a
    small perturbation of the old one where sizes agree, seeded, and packed
    row-major in element order."""
    nb_old, nb_new, nr = [4, 7, 5], [5, 7, 3], [20, 30, 9]
    Vo, Vn = G.make_basis_pair(nb_old, nb_new, nr, delta=0.05, seed=1)
    for K, (a, b) in enumerate(zip(Vo, Vn)):
        assert a.shape == (nr[K], nb_old[K]) and b.shape == (nr[K], nb_new[K])
        assert np.max(np.abs(a.T @ a - np.eye(nb_old[K]))) <= 1e-13
        assert np.max(np.abs(b.T @ b - np.eye(nb_new[K]))) <= 1e-13
    # same size: the new basis spans nearly the old span (principal angles ~ delta)
    s = np.linalg.svd(Vo[1].T @ Vn[1], compute_uv=False)
    assert s.min() > 0.9
    Vo2, Vn2 = G.make_basis_pair(nb_old, nb_new, nr, delta=0.05, seed=1)
    assert all(np.array_equal(x, y) for x, y in zip(Vo + Vn, Vo2 + Vn2))
    packed = G.pack_blocks(Vo)
    assert packed.shape == (sum(r * n for r, n in zip(nr, nb_old)),)
    assert np.array_equal(packed[:nr[0] * nb_old[0]].reshape(nr[0], nb_old[0]), Vo[0])
    with pytest.raises(ValueError):
        G.make_basis_pair([40], [4], [20])   # more basis functions than grid points
