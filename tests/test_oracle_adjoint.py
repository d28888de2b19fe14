"""Pins for the oracle's adjoint of the band energy E = sum_i f_i lambda_i of
one cycle: central finite differences of the oracle's own energy (tied,
symmetric perturbations of H and a random direction in X), the converged case
where the gradient reduces to sum_i g_i v_i v_i^T over exact eigenpairs of the
dense H with a vanishing X gradient, and planted mistakes that the pins catch."""
import numpy as np
import pytest

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G


def setup(Ns=10, m=6, seed=11):
    cfg = G.ProblemConfig(name="adj", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                          nb=(4, 7), Ns=Ns, m=m, Ne=float(Ns), seed=seed, kT=0.3)
    bs = G.make_blocks(cfg)
    H = O.DGHamiltonian.from_blocksparse(bs)
    lam = np.linalg.eigvalsh(H.dense())
    X = G.make_X(H.N, Ns, seed).T.copy()
    a0, b, a = lam[0] - 0.3, lam[-1] + 0.3, lam[Ns + 3]
    return cfg, bs, H, X, (a, b, a0)


def perturbed(bs, entries, h):
    vals = bs.values.copy()
    for off in entries:
        vals[off] += h
    return O.DGHamiltonian(bs.nb, bs.row_ptr, bs.col, bs.blk_off, vals)


def tied_entries(bs, H, e, j, jp):
    """Value offsets of H_KK'[j, j'] and its mirror H_K'K[j', j]."""
    K = int(np.searchsorted(bs.row_ptr, e, side="right") - 1)
    Kp = int(bs.col[e])
    nK, nKp = int(bs.nb[K]), int(bs.nb[Kp])
    a = int(bs.blk_off[e]) + j * nKp + jp
    f = [i for i in range(bs.row_ptr[Kp], bs.row_ptr[Kp + 1]) if bs.col[i] == K][0]
    b = int(bs.blk_off[f]) + jp * nK + j
    return sorted({a, b})


def test_h_gradient_matches_central_differences():
    cfg, bs, H, X, (a, b, a0) = setup()
    E, Gr, _ = O.band_energy_grad(H, X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
    assert abs(E - O.band_energy(H, X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)) <= 1e-12 * abs(E)
    T = O.tied_gradient(H, Gr)
    rng = np.random.default_rng(0)
    h = 1e-5
    scale = max(np.max(np.abs(t)) for t in T)
    for _ in range(16):
        e = int(rng.integers(0, bs.nnzb))
        K = int(np.searchsorted(bs.row_ptr, e, side="right") - 1)
        j, jp = int(rng.integers(0, bs.nb[K])), int(rng.integers(0, bs.nb[bs.col[e]]))
        ent = tied_entries(bs, H, e, j, jp)
        Ep = O.band_energy(perturbed(bs, ent, h), X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
        Em = O.band_energy(perturbed(bs, ent, -h), X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - T[e][j, jp]) <= 1e-6 * scale, (e, j, jp, fd, T[e][j, jp])


def test_x_gradient_matches_directional_difference():
    cfg, bs, H, X, (a, b, a0) = setup()
    _, _, Xbar = O.band_energy_grad(H, X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
    rng = np.random.default_rng(1)
    for _ in range(3):
        dX = rng.standard_normal(X.shape)
        h = 1e-6
        Ep = O.band_energy(H, X + h * dX, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
        Em = O.band_energy(H, X - h * dX, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
        fd = (Ep - Em) / (2 * h)
        an = float(np.sum(Xbar * dX))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_converged_gradient_is_dense_eigen_formula():
    cfg, bs, H, X, (a, b, a0) = setup(Ns=8, m=8)
    A = H.dense()
    lam, V = np.linalg.eigh(A)
    # converge the block first (cycles without gradients)
    Xc = X
    for _ in range(200):
        Yt = O.chebyshev_filter(H, Xc, cfg.m, a, b, a0)
        Xc, D, _ = O.rayleigh_ritz(H, O.cholesky_qr(Yt)[0])
    _, Gr, Xbar = O.band_energy_grad(H, Xc, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
    Ns = cfg.Ns
    f, _ = O.fermi_occupations(lam[:Ns], cfg.Ne, cfg.kT)
    g = O.energy_weights(lam[:Ns], f, cfg.kT)
    ref = O.block_outer(H, V[:, :Ns], V[:, :Ns], g)
    scale = max(np.max(np.abs(r)) for r in ref)
    for got, want in zip(Gr, ref):
        assert np.max(np.abs(got - want)) <= 1e-8 * scale
    assert np.linalg.norm(Xbar) <= 1e-8 * np.linalg.norm(Xc)


def test_pins_catch_planted_adjoint_mistakes(monkeypatch):
    """Drop the Fermi-level term of g (the dmu/dlambda coupling): the
    finite-difference pin must fail."""
    cfg, bs, H, X, (a, b, a0) = setup()
    monkeypatch.setattr(O, "energy_weights", lambda lam, f, kT: f + lam * (-f * (1 - f) / kT))
    _, Gr, _ = O.band_energy_grad(H, X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
    monkeypatch.undo()
    _, Gok, _ = O.band_energy_grad(H, X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
    T, Tok = O.tied_gradient(H, Gr), O.tied_gradient(H, Gok)
    diff = max(np.max(np.abs(x - y)) for x, y in zip(T, Tok))
    scale = max(np.max(np.abs(t)) for t in Tok)
    assert diff > 1e-3 * scale


def test_tied_gradient_of_diagonal_blocks_is_symmetric():
    cfg, bs, H, X, (a, b, a0) = setup()
    _, Gr, _ = O.band_energy_grad(H, X, cfg.m, a, b, a0, cfg.Ne, cfg.kT)
    T = O.tied_gradient(H, Gr)
    e = 0
    for K in range(H.M):
        for Kp, _ in H.neighbours(K):
            if K == Kp:
                assert np.allclose(T[e], T[e].T, rtol=0, atol=1e-12 * np.max(np.abs(T[e])))
            e += 1
