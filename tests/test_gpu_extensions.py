"""GPU parity, through the C ABI, of the steps around the cycle: re-alignment
to a new basis (Eq. basis_rotation_3), density blocks on H's pattern
(Eq. densitymatrix) and the CholeskyQR2 / shifted CholeskyQR3
orthonormalisations, against the FP64 oracle. All FP64 on both sides; the
re-alignment forms T_K = V_new^T V_old first on both, so results agree to a
few ulps of the largest entry."""
import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None
dev = torch.device("cuda:0")


def rel(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def realign_case(Ns=131, seed=0):
    cfg = G.ProblemConfig(name="new", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                          nb=(20, 90), Ns=Ns, m=3, Ne=8.0, seed=seed)
    H = G.make_blocks(cfg)
    nb_new = np.asarray(H.nb)
    rng = np.random.default_rng(seed + 5)
    nb_old = np.clip(nb_new + rng.integers(-6, 7, size=nb_new.shape), 1, 256)
    nr = np.maximum(nb_old, nb_new) + rng.integers(3, 40, size=nb_new.shape)
    Vo, Vn = G.make_basis_pair(nb_old, nb_new, nr, delta=0.1, seed=seed)
    X_old = rng.standard_normal((Ns, int(nb_old.sum())))
    return H, nb_old, nr, Vo, Vn, X_old


@pytest.mark.parametrize("Ns", [1, 131, 300])
def test_realign_matches_oracle(Ns):
    H, nb_old, nr, Vo, Vn, X_old = realign_case(Ns)
    ref = O.realign(Vo, Vn, X_old.T).T
    with D.Context(H) as ctx:
        # strided input and output blocks; the output padding stays untouched
        big_in = torch.full((Ns, X_old.shape[1] + 3), 5.0, dtype=torch.float64, device=dev)
        big_in[:, :X_old.shape[1]] = torch.from_numpy(X_old)
        out = torch.full((Ns, H.N + 7), -3.0, dtype=torch.float64, device=dev)
        ctx.realign(big_in[:, :X_old.shape[1]], nb_old, nr, torch.from_numpy(G.pack_blocks(Vo)).to(dev),
                    torch.from_numpy(G.pack_blocks(Vn)).to(dev), X_new=out[:, :H.N])
        got = out[:, :H.N].cpu().numpy()
        assert torch.all(out[:, H.N:] == -3.0)
    assert rel(got, ref) <= 1e-13


def test_realign_same_basis_is_identity_and_errors():
    H, nb_old, nr, Vo, Vn, X_old = realign_case(40)
    nb = np.asarray(H.nb)
    Vs, _ = G.make_basis_pair(nb, nb, nr, seed=9)
    X = np.random.default_rng(1).standard_normal((40, H.N))
    with D.Context(H) as ctx:
        Vd = torch.from_numpy(G.pack_blocks(Vs)).to(dev)
        Xd = torch.from_numpy(X).to(dev)
        got = ctx.realign(Xd, nb, nr, Vd, Vd).cpu().numpy()
        assert rel(got, X) <= 1e-14
        with pytest.raises(D.DGChefsiError) as e:  # output overlapping the input
            ctx.realign(Xd, nb, nr, Vd, Vd, X_new=Xd)
        assert e.value.status == "ERR_ARG"
        bad = nb.copy()
        bad[0] = 0
        with pytest.raises((D.DGChefsiError, ValueError)):
            ctx.realign(Xd, bad, nr, Vd, Vd)
        with pytest.raises(ValueError):
            ctx.realign(Xd, nb, nr, Vd[:-1], Vd)


def test_density_pattern_matches_oracle():
    cfg = G.ProblemConfig(name="pd", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                          nb=(30, 70), Ns=150, m=3, Ne=100.0, seed=4)
    H, X0, _, Ns, _ = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    f = np.random.default_rng(3).uniform(0, 1, Ns)
    ref = np.concatenate([b.ravel() for b in O.density_pattern_blocks(Ho, X0.T, f)])
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        fd = torch.from_numpy(f).to(dev)
        P = ctx.density_pattern(X, fd).cpu().numpy()
        Pd = ctx.unpack_density(ctx.density_blocks(X, fd))
    assert rel(P, ref) <= 1e-13
    for K in range(H.nb.shape[0]):  # diagonal blocks agree with the diagonal-block call
        e = [e for e in range(H.row_ptr[K], H.row_ptr[K + 1]) if H.col[e] == K][0]
        n = int(H.nb[K])
        blk = P[H.blk_off[e]:H.blk_off[e] + n * n].reshape(n, n)
        assert np.max(np.abs(blk - Pd[K].cpu().numpy())) <= 1e-12 * np.max(np.abs(blk))


def conditioned_block(N, Ns, kappa, seed):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((N, Ns)))[0]
    W = np.linalg.qr(rng.standard_normal((Ns, Ns)))[0]
    return U, (U @ np.diag(np.geomspace(1.0, 1.0 / kappa, Ns)) @ W.T)


def test_orthonormalisations_on_ill_conditioned_blocks():
    """cond(Y) = 1e6: one Cholesky-QR pass leaves X_new visibly non-orthonormal
    (kappa^2 u ~ 1e-4), CholeskyQR2 and shifted CholeskyQR3 orthonormalise to
    rounding and reproduce the Rayleigh-Ritz values of span(Y). cond(Y) = 1e9:
    the unshifted forms fail or degrade, the shifted form still orthonormalises."""
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, _, _, Ns, _ = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    hn = float(np.max(np.abs(np.linalg.eigvalsh(Ho.dense()))))
    U, Y = conditioned_block(Ho.N, Ns, 1e6, seed=2)
    _, ref, _ = O.rayleigh_ritz(Ho, U)
    results = {}
    with D.Context(H) as ctx:
        for mode in ("cholqr", "cholqr2", "shifted_cholqr3"):
            ctx.set_orthonormalisation(mode)
            Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).to(dev)
            ritz = ctx.rayleigh_ritz(Yd).cpu().numpy()
            Xn = Yd.cpu().numpy()
            results[mode] = (np.max(np.abs(Xn @ Xn.T - np.eye(Ns))), np.max(np.abs(ritz - ref)) / hn)
            print(f"ORTH kappa=1e6 {mode} orth={results[mode][0]:.2e} ritz={results[mode][1]:.2e}")
        assert results["cholqr"][0] > 1e-8
        for mode in ("cholqr2", "shifted_cholqr3"):
            assert results[mode][0] <= 1e-13 and results[mode][1] <= 1e-9
        _, Y9 = conditioned_block(Ho.N, Ns, 1e9, seed=3)
        ctx.set_orthonormalisation("shifted_cholqr3")
        Yd = torch.from_numpy(np.ascontiguousarray(Y9.T)).to(dev)
        ctx.rayleigh_ritz(Yd)
        Xn = Yd.cpu().numpy()
        assert np.max(np.abs(Xn @ Xn.T - np.eye(Ns))) <= 1e-13
        with pytest.raises(D.DGChefsiError) as e:  # unknown mode
            D._check(D._lib.dgchefsi_set_orthonormalisation(ctx._h, 7))
        assert e.value.status == "ERR_ARG"


@pytest.mark.parametrize("mode", ["cholqr2", "shifted_cholqr3"])
def test_cycle_with_other_orthonormalisation_matches_oracle(mode):
    """On a well-conditioned cycle every orthonormalisation gives the oracle's
    Ritz values and density blocks."""
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    lam = np.linalg.eigvalsh(Ho.dense())
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[Ns]
    Yt = O.chebyshev_filter(Ho, X0.T, cfg.m, a, b, a0)
    Q, _ = O.cholesky_qr2(Yt) if mode == "cholqr2" else O.shifted_cholesky_qr3(Yt)
    _, ref, _ = O.rayleigh_ritz(Ho, Q)
    with D.Context(H) as ctx:
        ctx.set_orthonormalisation(mode)
        Yd = torch.from_numpy(np.ascontiguousarray(Yt.T)).to(dev)
        ritz = ctx.rayleigh_ritz(Yd).cpu().numpy()
    assert np.max(np.abs(ritz - ref)) <= 1e-10 * max(abs(a0), abs(b))
