"""The Cholesky factor's inverse of Alg. 1 step 3 from the recursive blocked
form on dense products (DGCHEFSI_CHOL_PRODUCTS), through the C ABI, against
the oracle's factorisation (``O.cholesky_inverse``) and cuSOLVER's potrf +
trtri on the same seeded matrices.

* Orders 64 (one leaf), 65 (a leaf of one row), 700 and 1100 (products on
  the FP64 cores over ragged splits) and 2500 (the top levels' products from
  BF16 slices): L^{-1} within 20 times the error of cuSOLVER's own result
  (both measured against the oracle), and L^{-1} S L^{-T} = I to the same.
* A badly conditioned matrix (cond 1e10, the Cholesky-QR regime; its
  diagonal spans five orders): the same comparison, which holds because S is
  equilibrated by powers of two before the sliced products.
* An indefinite matrix fails with ERR_NOT_SPD at the planted column, in the
  first leaf, in a later leaf and below a sliced level.
* Rayleigh-Ritz with either form on the CheFSI block gives the same Ritz
  values and density blocks.
"""
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


def inverse_factor(ctx, S, form, pad=0):
    n = S.shape[0]
    buf = torch.full((n, n + pad), 3.0, dtype=torch.float64, device=dev)
    buf[:, :n] = torch.from_numpy(np.tril(S) + np.triu(np.full_like(S, -9.0), 1)).to(dev)
    ctx.set_cholesky(form)
    ctx.cholesky_inverse(buf[:, :n])
    return np.tril(buf[:, :n].cpu().numpy())


@pytest.mark.parametrize("n,cond", [(64, 1e3), (65, 1e3), (700, 1e4), (1100, 1e4), (2500, 1e4), (1300, 1e10)])
def test_recursive_form_matches_oracle_like_cusolver(n, cond):
    S, _ = G.planted_cholesky(n, cond=cond, seed=n)
    _, Li_o = O.cholesky_inverse(S)
    with tiny_ctx() as ctx:
        Li_p = inverse_factor(ctx, S, "products", pad=2)
        Li_c = inverse_factor(ctx, S, "cusolver")
    scale = np.abs(Li_o).max()
    e_p = np.abs(Li_p - Li_o).max() / scale
    e_c = np.abs(Li_c - Li_o).max() / scale
    r_p = np.abs(Li_p @ S @ Li_p.T - np.eye(n)).max()
    r_c = np.abs(Li_c @ S @ Li_c.T - np.eye(n)).max()
    print(f"CHOL n={n} cond={cond:.0e}: vs oracle products {e_p:.1e} cusolver {e_c:.1e}; "
          f"L^-1 S L^-T - I products {r_p:.1e} cusolver {r_c:.1e}")
    assert e_p <= 20 * max(e_c, U)
    assert r_p <= 20 * max(r_c, U)


@pytest.mark.parametrize("n,col", [(200, 17), (1000, 700), (2300, 1900)])
def test_indefinite_matrix_fails_at_the_planted_column(n, col):
    S, _ = G.planted_cholesky(n, cond=1e2, negative_at=col, seed=n + col)
    with tiny_ctx() as ctx:
        buf = torch.from_numpy(S).to(dev)
        ctx.set_cholesky("products")
        with pytest.raises(D.DGChefsiError) as e:
            ctx.cholesky_inverse(buf)
    assert e.value.status == "ERR_NOT_SPD"
    assert f"column {col + 1}" in str(e.value)


def test_settings_and_arguments():
    with tiny_ctx() as ctx:
        with pytest.raises(D.DGChefsiError) as e:
            D._check(D._lib.dgchefsi_set_cholesky(ctx._h, 9))
        assert e.value.status == "ERR_ARG"
        S = torch.eye(3, dtype=torch.float64, device=dev)
        with pytest.raises(D.DGChefsiError) as e:
            D._check(D._lib.dgchefsi_cholesky_inverse(ctx._h, D._ptr(S), 3, 2))
        assert e.value.status == "ERR_ARG"
        D._check(D._lib.dgchefsi_cholesky_inverse(ctx._h, D._ptr(S), 0, 0))


def test_rayleigh_ritz_with_either_cholesky_form():
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(5, 4, 4), nb=64, Ns=700, m=10, name="bulk5x4x4")
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    out = {}
    with D.Context(H) as ctx:
        ctx.set_subspace_products("sliced_bf16")
        b, tmin = ctx.bounds(torch.from_numpy(v0).to(dev), 10)
        X = torch.from_numpy(X0).to(dev)
        Y = ctx.filter(X, cfg.m, tmin + (b - tmin) * Ns / H.N, b, tmin, prec="bf16x3")
        for form in ("cusolver", "products"):
            ctx.set_cholesky(form)
            Yb = Y.clone()
            ritz = ctx.rayleigh_ritz(Yb)
            f, _ = ctx.occupations(ritz, Ne, cfg.kT)
            out[form] = (ritz.cpu().numpy(), ctx.density_blocks(Yb, f).cpu().numpy())
    scale = max(abs(b), abs(tmin))
    er = np.abs(out["products"][0] - out["cusolver"][0]).max() / scale
    ep = np.linalg.norm(out["products"][1] - out["cusolver"][1]) / np.linalg.norm(out["cusolver"][1])
    print(f"CHOL Rayleigh-Ritz products vs cusolver: ritz {er:.1e}, density {ep:.1e}")
    assert er <= 1e-11 and ep <= 1e-10
