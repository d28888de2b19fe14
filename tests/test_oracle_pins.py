"""Pins for the FP64 oracle: each oracle function is checked against a result
the mathematics fixes without the oracle's own code path (brute-force dense
products, closed forms, exact spectra, factorisation uniqueness, invariants).
A few tests plant a plausible mistake in a copy of an oracle routine and check
that the pin catches it."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G


def small_problem(grid=(3, 2, 2), nb=(5, 9), stencil="27", periodic=(True, False, True), Ns=12, seed=3):
    cfg = G.ProblemConfig(name="t", grid=grid, periodic=periodic, stencil=stencil, nb=nb, Ns=Ns,
                          m=6, Ne=G.default_ne(Ns) if Ns > 20 else 2.0 * (Ns // 2), seed=seed)
    bs = G.make_blocks(cfg)
    return cfg, bs, O.DGHamiltonian.from_blocksparse(bs)


# ---------------------------------------------------------------- generator


def test_generator_structure_and_symmetry():
    cfg = G.CONFIGS["tiny_2x2x2"]
    bs = G.make_blocks(cfg)
    assert bs.M == 8 and bs.N == 256
    assert np.all(np.diff(bs.row_ptr) == 8)  # every element couples to all 8
    H = O.DGHamiltonian.from_blocksparse(bs)
    A = H.dense()
    assert np.array_equal(A, A.T)
    bs2 = G.make_blocks(cfg)
    assert np.array_equal(bs.values, bs2.values)


def test_generator_stencils_and_uneven_sizes():
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(4, 4, 4), nb=8, Ns=16)
    bs = G.make_blocks(cfg)
    assert np.all(np.diff(bs.row_ptr) == 27)
    cfg2 = G.scaled_copy(G.CONFIGS["sheet2d_24x20"], grid=(5, 4, 1), Ns=30)
    bs2 = G.make_blocks(cfg2)
    assert np.all(np.diff(bs2.row_ptr) == 9)
    assert bs2.nb.min() >= 40 and bs2.nb.max() <= 120
    A = O.DGHamiltonian.from_blocksparse(bs2).dense()
    assert np.array_equal(A, A.T)
    # diagonal blocks have the stated spectrum U[-1, 40]
    K0 = O.DGHamiltonian.from_blocksparse(bs2)
    d = np.linalg.eigvalsh(next(b for Kp, b in K0.neighbours(0) if Kp == 0))
    assert d.min() >= -1 - 1e-12 and d.max() <= 40 + 1e-12


# ---------------------------------------------------------------- mat-vec (Eq. matvec_3)


def test_matvec_equals_dense_product():
    _, bs, H = small_problem()
    X = np.random.default_rng(0).standard_normal((H.N, 7))
    ref = H.dense() @ X
    got = O.matvec(H, X)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_matvec_single_vector_and_empty_block():
    _, _, H = small_problem()
    x = np.random.default_rng(1).standard_normal((H.N, 1))
    assert np.allclose(O.matvec(H, x), H.dense() @ x, rtol=0, atol=1e-12)
    assert O.matvec(H, np.zeros((H.N, 0))).shape == (H.N, 0)


# ---------------------------------------------------------------- Chebyshev filter (Alg. 1 step 2)


def closed_form_filter(A, X, m, a, b, a0):
    """V diag(C_m((lambda - c)/e) / C_m((a0 - c)/e)) V^T X from a dense eigh."""
    lam, V = np.linalg.eigh(A)
    e, c = 0.5 * (b - a), 0.5 * (b + a)
    g = O.chebyshev_value(m, (lam - c) / e) / O.chebyshev_value(m, np.array([(a0 - c) / e]))[0]
    return V @ (g[:, None] * (V.T @ X))


def test_chebyshev_value_closed_forms():
    t = np.array([-3.0, -1.0, -0.3, 0.0, 0.7, 1.0, 2.5])
    assert np.allclose(O.chebyshev_value(2, t), 2 * t**2 - 1, rtol=1e-14, atol=1e-14)
    assert np.allclose(O.chebyshev_value(3, t), 4 * t**3 - 3 * t, rtol=1e-14, atol=1e-13)
    assert np.allclose(O.chebyshev_value(4, t), 8 * t**4 - 8 * t**2 + 1, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m", [1, 2, 5, 10, 20])
def test_filter_matches_closed_form(m):
    _, _, H = small_problem()
    A = H.dense()
    lam = np.linalg.eigvalsh(A)
    X = np.random.default_rng(m).standard_normal((H.N, 9))
    a0, b = lam[0] - 0.1, lam[-1] + 0.2
    a = lam[len(lam) // 3]
    ref = closed_form_filter(A, X, m, a, b, a0)
    got = O.chebyshev_filter(H, X, m, a, b, a0)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_filter_fixes_eigenvector_at_a0_and_damps_interval():
    _, _, H = small_problem()
    A = H.dense()
    lam, V = np.linalg.eigh(A)
    a0, b, a = lam[0], lam[-1], lam[len(lam) // 2]
    m = 9
    y = O.chebyshev_filter(H, V[:, :1], m, a, b, a0)
    assert np.allclose(y, V[:, :1], atol=1e-12)
    # eigenvectors with eigenvalue in [a, b] are damped by at most 1/|C_m(tau0)|
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    bound = 1.0 / abs(O.chebyshev_value(m, np.array([(a0 - c) / e]))[0])
    inside = np.where((lam >= a) & (lam <= b))[0]
    Y = O.chebyshev_filter(H, V[:, inside], m, a, b, a0)
    assert np.all(np.linalg.norm(Y, axis=0) <= bound * (1 + 1e-10))


def test_filter_degree_one_and_diagonal_matrix():
    d = np.array([-1.0, 0.5, 3.0, 10.0, 39.0])
    H = O.DGHamiltonian([5], [0, 1], [0], [0], np.diag(d).ravel())
    X = np.eye(5)
    a0, a, b = -1.5, 4.0, 40.0
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    y1 = O.chebyshev_filter(H, X, 1, a, b, a0)
    assert np.allclose(y1, np.diag((d - c) / (a0 - c)), atol=1e-15)
    y7 = O.chebyshev_filter(H, X, 7, a, b, a0)
    expect = O.chebyshev_value(7, (d - c) / e) / O.chebyshev_value(7, np.array([(a0 - c) / e]))[0]
    assert np.allclose(np.diag(y7), expect, rtol=1e-13, atol=1e-15)


def test_filter_rejects_bad_bounds():
    _, _, H = small_problem()
    X = np.ones((H.N, 1))
    for a, b, a0 in [(1.0, 1.0, 0.0), (2.0, 1.0, 0.0), (1.0, 2.0, 1.0)]:
        with pytest.raises(ValueError):
            O.chebyshev_filter(H, X, 3, a, b, a0)


def test_pin_catches_planted_filter_mistakes():
    """Mutants of the recurrence (wrong sign on the Y_{k-1} term, a missing
    shift, a shifted sigma index) must fail the closed-form pin."""
    _, _, H = small_problem()
    A = H.dense()
    lam = np.linalg.eigvalsh(A)
    X = np.random.default_rng(5).standard_normal((H.N, 4))
    m, a0, b, a = 8, lam[0] - 0.1, lam[-1] + 0.2, lam[len(lam) // 3]
    ref = closed_form_filter(A, X, m, a, b, a0)

    def mutant(kind):
        c, e, sig = O.filter_coefficients(m, a, b, a0)
        Yp = X.copy()
        shift = 0.0 if kind == "noshift" else c
        Y = (sig[1] / e) * (O.matvec(H, Yp) - shift * Yp)
        for k in range(1, m):
            s_new = sig[k] if kind == "index" else sig[k + 1]
            beta = sig[k] * s_new
            if kind == "sign":
                beta = -beta
            Yn = (2 * s_new / e) * (O.matvec(H, Y) - shift * Y) - beta * Yp
            Yp, Y = Y, Yn
        return Y

    for kind in ("sign", "noshift", "index"):
        err = np.linalg.norm(mutant(kind) - ref) / np.linalg.norm(ref)
        assert err > 1e-3, kind


# ---------------------------------------------------------------- Lanczos bound (Alg. 1 step 1)


def test_lanczos_bound_brackets_spectrum():
    _, _, H = small_problem()
    A = H.dense()
    lam = np.linalg.eigvalsh(A)
    v0 = np.random.default_rng(2).standard_normal(H.N)
    b, tmin, al, be = O.lanczos_bounds(H, v0, 10)
    gersh = np.max(np.sum(np.abs(A), axis=1))
    assert lam[-1] <= b <= gersh
    assert tmin >= lam[0] - 1e-12          # Ritz values lie inside the spectrum
    # T_k matches V^T A V built from scratch (three-term structure)
    assert len(al) == 10 and len(be) == 9


def test_lanczos_exact_on_small_diagonal():
    d = np.array([3.0, -2.0, 7.5, 1.0])
    H = O.DGHamiltonian([4], [0, 1], [0], [0], np.diag(d).ravel())
    b, tmin, _, _ = O.lanczos_bounds(H, np.ones(4), 10)   # k clipped to N = 4
    assert abs(b - 7.5) <= 1e-12 and abs(tmin + 2.0) <= 1e-12


def test_lanczos_invariant_start_vector_stops_early():
    d = np.array([3.0, -2.0, 7.5, 1.0])
    H = O.DGHamiltonian([4], [0, 1], [0], [0], np.diag(d).ravel())
    b, tmin, al, _ = O.lanczos_bounds(H, np.array([0.0, 0.0, 2.0, 0.0]), 10)
    assert len(al) == 1 and b == 7.5 and tmin == 7.5


# ---------------------------------------------------------------- Cholesky-QR (Alg. 1 step 3)


def test_cholesky_qr_matches_householder_qr():
    Y = np.random.default_rng(4).standard_normal((60, 12)) @ np.diag(np.logspace(0, 3, 12))
    Yh, U, S = O.cholesky_qr(Y)
    Qh, Rh = np.linalg.qr(Y)
    sgn = np.sign(np.diag(Rh))
    assert np.allclose(Yh, Qh * sgn[None, :], atol=1e-10)
    assert np.allclose(U, sgn[:, None] * Rh, rtol=1e-10, atol=1e-9)
    assert np.allclose(np.triu(U), U) and np.all(np.diag(U) > 0)
    assert np.max(np.abs(Yh.T @ Yh - np.eye(12))) <= 1e-10
    assert np.allclose(Yh @ U, Y, rtol=1e-12, atol=1e-10)


def test_cholesky_qr_rejects_rank_deficient():
    Y = np.random.default_rng(4).standard_normal((30, 5))
    Y[:, 3] = Y[:, 1]
    with pytest.raises(np.linalg.LinAlgError):
        O.cholesky_qr(Y)


# ---------------------------------------------------------------- Rayleigh-Ritz (steps 4-5)


def test_rayleigh_ritz_on_invariant_subspace_is_exact():
    _, _, H = small_problem()
    A = H.dense()
    lam, V = np.linalg.eigh(A)
    R = sla.qr(np.random.default_rng(6).standard_normal((8, 8)))[0]
    Yh = V[:, :8] @ R           # another orthonormal basis of the lowest 8
    X_new, D, HX = O.rayleigh_ritz(H, Yh)
    assert np.allclose(D, lam[:8], rtol=0, atol=1e-12)
    assert np.allclose(HX, A @ X_new, atol=1e-11)
    assert np.max(np.abs(HX - X_new * D[None, :])) <= 1e-11


def test_cycles_converge_to_dense_eigenvalues():
    cfg, bs, H = small_problem(Ns=14)
    A = H.dense()
    lam = np.linalg.eigvalsh(A)
    X = G.make_X(H.N, cfg.Ns, seed=1).T
    v0 = G.make_start_vector(H.N, 1)
    ritz = None
    for _ in range(30):
        out = O.chefsi_cycle(H, X, 8, cfg.Ne, 0.01, v0, prev_ritz=ritz)
        X, ritz = out["X"], out["ritz"]
    g = 3
    scale = max(abs(lam[0]), abs(lam[-1]))
    assert np.max(np.abs(ritz[:-g] - lam[:cfg.Ns - g])) <= 1e-10 * scale
    res = np.linalg.norm(A @ X[:, :-g] - X[:, :-g] * ritz[None, :-g], axis=0)
    assert np.max(res) <= 1e-9 * scale


# ---------------------------------------------------------------- occupations


def test_occupations_electron_count_and_symmetric_case():
    lam = np.linspace(-1.0, 3.0, 17)
    f, mu = O.fermi_occupations(lam, 13.0, 0.05)
    assert abs(2 * f.sum() - 13.0) <= 1e-13 * 13.0 + 1e-15   # the bisection stopping rule
    assert np.all((f >= 0) & (f <= 1)) and np.all(np.diff(f) <= 0)
    f2, mu2 = O.fermi_occupations(np.array([0.0, 1.0]), 2.0, 0.1)
    assert abs(mu2 - 0.5) <= 1e-12
    assert abs(f2[0] - 1 / (1 + np.exp(-5.0))) <= 1e-12


def test_occupations_extremes_and_errors():
    lam = np.array([-2.0, 0.0, 1.0, 5.0])
    f, _ = O.fermi_occupations(lam, 8.0, 0.01)
    assert np.allclose(f, 1.0, atol=1e-12)
    f, _ = O.fermi_occupations(lam, 0.0, 0.01)
    assert np.allclose(f, 0.0, atol=1e-12)
    f, _ = O.fermi_occupations(lam, 4.0, 1e-4)   # small kT: a step at the gap
    assert np.allclose(f, [1, 1, 0, 0], atol=1e-12)
    for Ne, kT in [(9.0, 0.01), (-1.0, 0.01), (2.0, 0.0)]:
        with pytest.raises(ValueError):
            O.fermi_occupations(lam, Ne, kT)


# ---------------------------------------------------------------- density blocks


def test_density_blocks_match_dense_density_matrix():
    _, _, H = small_problem()
    rng = np.random.default_rng(7)
    X = rng.standard_normal((H.N, 6))
    f = rng.uniform(0, 1, 6)
    P_dense = X @ np.diag(f) @ X.T
    blocks = O.density_blocks(H, X, f)
    for K in range(H.M):
        r = H.rows(K)
        assert np.allclose(blocks[K], P_dense[r, r], atol=1e-13)
        assert np.array_equal(blocks[K], blocks[K].T) or np.allclose(blocks[K], blocks[K].T, atol=1e-15)


def test_cycle_invariants_trace_and_orthonormality():
    cfg = G.CONFIGS["tiny_2x2x2"]
    bs = G.make_blocks(cfg)
    H = O.DGHamiltonian.from_blocksparse(bs)
    X = G.make_X(H.N, cfg.Ns, cfg.seed).T
    out = O.chefsi_cycle(H, X, cfg.m, cfg.Ne, cfg.kT, G.make_start_vector(H.N, cfg.seed))
    Xn = out["X"]
    assert np.max(np.abs(Xn.T @ Xn - np.eye(cfg.Ns))) <= 1e-11
    tr = sum(np.trace(P) for P in out["P"])
    assert abs(2 * tr - cfg.Ne) <= 1e-9
    assert out["a0"] < out["a"] < out["b"]
