"""The eigensolve of the projected Hamiltonian (Alg. 1 step 4) in its refined
form, DGCHEFSI_EIG_REFINED: FP32 eigenvectors refined to FP64 accuracy by
Ogita-Aishima steps whose products run from exact BF16 slices on the tensor
cores, against the oracle's dense FP64 eigensolve (``O.subspace_eigh``) on
seeded planted spectra, through the C ABI.

For every case (n = 1000 and 1536, ragged against the 32-row tiles of the
small kernels and the 256-row tiles of the slice-pair kernel):
* eigenvalues within 64 u ||A|| sqrt(n) of the oracle's;
* V V^T = I and V A = diag(w) V to 64 u sqrt(n) (times ||A||): backward
  stable like the FP64 solver;
* eigenvectors of well-separated eigenvalues equal the oracle's up to sign,
  within 64 u sqrt(n) ||A|| / gap; for groups of repeated or nearly repeated
  eigenvalues the projector onto the group equals the oracle's.
Clusters of repeated values are resolved (statistics show them), a cluster
above 32 members hands over to the FP64 solver with the same results, and the
context's choice of solver follows DGCHEFSI_EIG_AUTO.
"""
import math

import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None
dev = torch.device("cuda:0")
U = 2.0 ** -53


def tiny_ctx():
    H, _, _, _, _ = G.make_problem(G.CONFIGS["tiny_2x2x2"])
    return D.Context(H)


def solve(ctx, A, pad=0):
    """GPU eigensolve of A (host array) with rows `pad` entries longer than n;
    the upper triangle is filled with garbage (it must not be read)."""
    n = A.shape[0]
    buf = torch.full((n, n + pad), 5.0, dtype=torch.float64, device=dev)
    At = torch.from_numpy(np.tril(A) + np.triu(np.full_like(A, 1e3), 1))
    buf[:, :n] = At.to(dev)
    w, V = ctx.subspace_eigh(buf[:, :n])
    return w.cpu().numpy(), V.cpu().numpy(), ctx.eigensolver_stats()


def check_against_oracle(A, w, V, groups=()):
    n = A.shape[0]
    wo, Vo = O.subspace_eigh(A)
    norm = np.abs(wo).max()
    tol = 64 * U * np.sqrt(n)
    ew = np.abs(w - wo).max() / norm
    eo = np.abs(V @ V.T - np.eye(n)).max()
    er = np.abs(V @ A - w[:, None] * V).max() / norm
    assert ew <= tol and eo <= tol and er <= tol, (ew, eo, er)
    in_group = np.zeros(n, bool)
    for centre, size, spread in groups:
        sel = np.abs(wo - centre) <= 10 * spread + 1e-12
        in_group |= sel
        P, Po = V[sel].T @ V[sel], Vo[sel].T @ Vo[sel]
        assert np.abs(P - Po).max() <= 1e-10, (centre, np.abs(P - Po).max())
    gaps = np.minimum(np.diff(wo, prepend=-np.inf), np.diff(wo, append=np.inf))
    sep = ~in_group & (gaps > 1e-6 * norm)
    dev_ = np.abs(1.0 - np.abs(np.sum(V * Vo, axis=1)))
    bound = (tol * norm / gaps) ** 2 + tol
    assert np.all(dev_[sep] <= bound[sep] + 1e-14), np.max(dev_[sep] - bound[sep])
    return ew, eo, er


@pytest.mark.parametrize("n", [1000, 1536])
def test_refined_matches_oracle(n):
    lam = G.clustered_spectrum(n, seed=n)
    A = G.make_planted_symmetric(lam, seed=n)
    with tiny_ctx() as ctx:
        ctx.set_eigensolver("refined")
        w, V, st = solve(ctx, A, pad=3)
    ew, eo, er = check_against_oracle(A, w, V)
    print(f"EIGH refined n={n}: eig {ew:.1e} orth {eo:.1e} resid {er:.1e} {st}")
    assert st["used"] == "refined" and st["fallback"] == 0 and 1 <= st["steps"] <= 5
    # from a whole-matrix start every step's update is a full product; it takes
    # the fewest slices whose splitting error 2 L max|E| 2^(-6s) (s + 4) stays
    # below 2^-53 L (the parity above holds with them)
    expect = [next((k for k in range(2, 10) if 2 * math.ldexp(k + 4, -6 * k) * e <= 2.0**-53), 10)
              for e in st["history"]]
    assert st["update_slices"] == expect and expect[-1] < 10


def test_refined_resolves_repeated_and_close_eigenvalues():
    groups = [(0.5, 8, 0.0), (1.25, 3, 0.0), (1.7, 13, 1e-9), (-0.4, 20, 1e-7)]
    lam = G.clustered_spectrum(1000, groups=groups, seed=7)
    A = G.make_planted_symmetric(lam, seed=7)
    with tiny_ctx() as ctx:
        ctx.set_eigensolver("refined")
        w, V, st = solve(ctx, A)
    ew, eo, er = check_against_oracle(A, w, V, groups)
    print(f"EIGH clusters: eig {ew:.1e} orth {eo:.1e} resid {er:.1e} {st}")
    assert st["used"] == "refined" and st["fallback"] == 0 and st["max_cluster"] >= 8


def test_cluster_above_32_hands_over_to_fp64_solver():
    groups = [(0.9, 44, 0.0)]
    lam = G.clustered_spectrum(600, groups=groups, seed=9)
    A = G.make_planted_symmetric(lam, seed=9)
    with tiny_ctx() as ctx:
        ctx.set_eigensolver("refined")
        w, V, st = solve(ctx, A)
    check_against_oracle(A, w, V, groups)
    assert st["used"] == "syevd" and st["fallback"] == 3 and st["max_cluster"] > 32


@pytest.mark.parametrize("n", [1, 2, 33])
def test_small_orders(n):
    lam = G.clustered_spectrum(n, seed=20 + n)
    A = G.make_planted_symmetric(lam, seed=20 + n)
    with tiny_ctx() as ctx:
        ctx.set_eigensolver("refined")
        w, V, st = solve(ctx, A)
    check_against_oracle(A, w, V)
    assert st["used"] == ("syevd" if n == 1 else "refined")


def test_auto_follows_subspace_products():
    lam = G.clustered_spectrum(300, seed=4)
    A = G.make_planted_symmetric(lam, seed=4)
    with tiny_ctx() as ctx:
        used = {}
        for prod in ("f64", "sliced_bf16"):
            ctx.set_subspace_products(prod)
            w, V, st = solve(ctx, A)
            check_against_oracle(A, w, V)
            used[prod] = st["used"]
        ctx.set_eigensolver("syevd")
        used["forced"] = solve(ctx, A)[2]["used"]
        with pytest.raises(D.DGChefsiError) as e:
            D._check(D._lib.dgchefsi_set_eigensolver(ctx._h, 7))
        assert e.value.status == "ERR_ARG"
    assert used == {"f64": "syevd", "sliced_bf16": "refined", "forced": "syevd"}


def test_identity_start_for_a_nearly_diagonal_matrix():
    """Every first-order coupling below 1/1000: no FP32 solve, the first step
    needs no products, and the result is the oracle's."""
    d = G.clustered_spectrum(1200, seed=31)
    A = G.near_diagonal_symmetric(d, 1e-10, seed=31)
    with tiny_ctx() as ctx:
        ctx.set_eigensolver("refined")
        w, V, st = solve(ctx, A)
    ew, eo, er = check_against_oracle(A, w, V)
    print(f"EIGH identity start: eig {ew:.1e} orth {eo:.1e} resid {er:.1e} {st}")
    assert st["used"] == "refined" and st["fallback"] == 0 and st["start_order"] == 0


@pytest.mark.parametrize(
    "n,top,repeats",
    [(600, 7, 0), (700, 37, 0), (900, 61, 0), (1100, 150, 0), (1300, 213, 0), (1600, 150, 0), (1600, 150, 3),
     (1600, 300, 0), (1600, 311, 0), (1600, 312, 0), (1600, 400, 0)],
)
def test_partial_start_for_a_coupled_top_block(n, top, repeats):
    # with 2e-8 background coupling 13, 41, 63 (odd orders: the Jacobi
    # tournament has an idle index), 156, 224, 160, 308, 319 and 320 (the
    # Jacobi kernel's largest order) and 406 rows reach the default start
    # threshold: the full and the block-structured first step
    """Only the last `top` rows are coupled: the FP32 start solves that block
    alone (its order is reported), the rest starts from unit vectors. With a
    block of at most n/8 rows the first step's products and update come from
    the block's rows and columns; `repeats` pairs of exactly equal, mutually
    uncoupled diagonal entries outside the block form clusters in that step,
    whose rows join the block of the update. Blocks up to 320 rows get their
    FP32 start from the library's cyclic Jacobi kernel (a 406-row coupled
    block still takes cuSOLVER's)."""
    d = G.clustered_spectrum(n, seed=33)
    A = G.near_diagonal_symmetric(d, 2e-8, top=top, top_coupling=0.05, seed=33)
    for r in range(repeats):
        i, j = 100 + 40 * r, 101 + 40 * r
        A[j, j] = A[i, i]
        A[i, j] = A[j, i] = 0.0
    with tiny_ctx() as ctx:
        ctx.set_eigensolver("refined")
        w, V, st = solve(ctx, A, pad=1)
    ew, eo, er = check_against_oracle(A, w, V)
    print(f"EIGH partial start n={n} repeats={repeats}: eig {ew:.1e} orth {eo:.1e} resid {er:.1e} {st}")
    assert st["used"] == "refined" and st["fallback"] == 0 and top <= st["start_order"] <= n // 2
    # blocks up to 320 rows start from this library's Jacobi kernel, larger ones from cuSOLVER
    assert st["start_solver"] == ("jacobi" if st["start_order"] <= 320 else "cusolver_fp32")
    if repeats:
        assert st["max_cluster"] >= 2


def test_cycles_refined_vs_fp64_solver_on_projected_hamiltonians():
    """The CheFSI cycles' own projected H (bulk 5x4x4, N = 5120, N_s = 400)
    with sliced products, five cycles from the random start: Ritz values and
    rotated blocks from the refined solver equal those from the FP64 solver
    cycle by cycle, the first cycle matches the oracle's, and the later
    cycles (a converging subspace) start from fewer FP32-solved rows."""
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(5, 4, 4), nb=64, Ns=400, m=10, name="bulk5x4x4")
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    out = {}
    with D.Context(H) as ctx:
        ctx.set_subspace_products("sliced_bf16")
        v = torch.from_numpy(v0).to(dev)
        for mode in ("syevd", "refined"):
            ctx.set_eigensolver(mode)
            X = torch.from_numpy(X0).to(dev)
            prev, out[mode] = None, []
            for cyc in range(5):
                res = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v, prev_ritz=prev)
                prev = res["ritz"].cpu().numpy()
                out[mode].append((prev, X.cpu().numpy(), res["bounds"], ctx.eigensolver_stats()))
    a, b, a0 = out["refined"][0][2]
    ref = O.chefsi_cycle(Ho, X0.T.copy(), cfg.m, Ne, cfg.kT, v0, bounds=(a, b, a0))
    scale = max(abs(a0), abs(b))
    eo = np.abs(out["refined"][0][0] - ref["ritz"]).max() / scale
    assert eo <= 1e-10
    orders = []
    for cyc in range(5):
        r_s, X_s = out["syevd"][cyc][:2]
        r_r, X_r, _, st = out["refined"][cyc]
        er = np.abs(r_r - r_s).max() / scale
        # rotated states: same up to sign where the Ritz values are separated
        gaps = np.minimum(np.diff(r_s, prepend=-np.inf), np.diff(r_s, append=np.inf)) / scale
        sep = gaps > 1e-6
        cos = np.abs(np.sum(X_r * X_s, axis=1)) / (np.linalg.norm(X_r, axis=1) * np.linalg.norm(X_s, axis=1))
        print(f"EIGH cycle {cyc}: ritz vs syevd {er:.1e}, min cos {cos[sep].min():.16f} {st}")
        assert st["used"] == "refined" and st["fallback"] == 0
        assert er <= 1e-12
        assert np.all(1.0 - cos[sep] <= 1e-18 / gaps[sep] ** 2 + 1e-13)
        orders.append(st["start_order"])
    print(f"EIGH cycle vs oracle {eo:.1e}, start orders {orders}")
    assert orders[0] == Ns and orders[-1] < Ns // 2
