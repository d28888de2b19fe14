"""The block-sparse product H X (Eq. matvec_3) in FP64 from exact BF16 slices
on the tensor cores (dgchefsi_sliced_matvec, the H Y_hat of the sliced
Rayleigh-Ritz step), through the C ABI, against the FP64 oracle.

* Integer H and X of at most 12 bits: every row and state splits exactly into
  three slices, every slice-pair sum is an exact FP32 integer, so the product
  equals the exact integer product bit for bit, on uniform 64-wide elements,
  on uneven elements (40..120, padded columns) and on the 2D sheet, with
  ragged state counts, with 3 and 10 slices, and across several state panels.
* Gaussian H (the workload generator) and X: within the stated bound
  L m_r n_s (2^{-6s}(s + 4) + 6 u) plus FP64's own bound on the reference.
* Error paths: an element wider than 128 (ERR_UNSUPPORTED), a NaN in X
  (ERR_NONFINITE).
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None
dev = torch.device("cuda:0")
U = 2.0 ** -53


def integer_h(H, seed=0, lim=2047):
    """H's pattern with symmetric integer blocks in [-lim, lim]."""
    rng = np.random.default_rng(seed)
    vals = np.zeros_like(H.values)
    nb, rp, col, bo = H.nb, H.row_ptr, H.col, H.blk_off
    for K in range(len(nb)):
        for e in range(rp[K], rp[K + 1]):
            Kp = int(col[e])
            if Kp < K:
                continue
            n, k = int(nb[K]), int(nb[Kp])
            B = rng.integers(-lim, lim + 1, size=(n, k)).astype(np.float64)
            if Kp == K:
                B = np.triu(B) + np.triu(B, 1).T
            vals[bo[e]:bo[e] + n * k] = B.ravel()
            if Kp != K:
                f = [f for f in range(rp[Kp], rp[Kp + 1]) if int(col[f]) == K][0]
                vals[bo[f]:bo[f] + n * k] = B.T.ravel()
    return dataclasses.replace(H, values=vals)


def problems():
    bulk = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(4, 4, 4), nb=64, Ns=300, name="bulk4")
    uneven = G.ProblemConfig(name="uneven", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                             nb=(40, 120), Ns=200, m=7, Ne=150.0, seed=5)
    sheet = G.scaled_copy(G.CONFIGS["sheet2d_24x20"], grid=(4, 3, 1), Ns=130, name="sheet")
    return [bulk, uneven, sheet]


@pytest.mark.parametrize("slices", [3, 10])
@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_integer_operands_bit_exact(cfg, slices):
    H = integer_h(G.make_blocks(cfg), seed=1)
    Ns = 300 if cfg.name == "bulk4" else 131
    rng = np.random.default_rng(2)
    X = rng.integers(-2047, 2048, size=(Ns, int(np.sum(H.nb)))).astype(np.float64)
    X[3] = rng.integers(-3, 4, size=X.shape[1])        # a state of small integers
    ref = O.matvec(O.DGHamiltonian.from_blocksparse(H), X.T).T    # exact: |entries| < 2^36
    with D.Context(H) as ctx:
        Y = ctx.sliced_matvec(torch.from_numpy(X).to(dev), slices=slices).cpu().numpy()
    assert np.array_equal(Y, ref)


def test_integer_operands_bit_exact_over_several_state_panels():
    """9600 states of the 4x4x4 copy: the FP32 slabs of 55 pairs exceed the
    8 GB workspace cap, so the states run in two panels."""
    cfg = problems()[0]
    H = integer_h(G.make_blocks(cfg), seed=3)
    N = int(np.sum(H.nb))
    Ns = 9600
    assert 55 * 4 * N * Ns > 8 * 2 ** 30
    rng = np.random.default_rng(4)
    X = rng.integers(-2047, 2048, size=(Ns, N)).astype(np.float64)
    ref = O.matvec(O.DGHamiltonian.from_blocksparse(H), X.T).T
    with D.Context(H) as ctx:
        Y = ctx.sliced_matvec(torch.from_numpy(X).to(dev), slices=10).cpu().numpy()
    assert np.array_equal(Y, ref)


@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_gaussian_operands_within_bound(cfg):
    H = G.make_blocks(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    Ns = 257
    X = G.make_X(Ho.N, Ns, 7)
    X *= np.exp(np.random.default_rng(8).uniform(-3, 3, size=(Ns, 1)))     # states of different norms
    ref = O.matvec(Ho, X.T).T
    # per row r of H: L (its column count), m_r; per state: n_s
    L = np.zeros(Ho.N)
    m_r = np.zeros(Ho.N)
    for K in range(Ho.M):
        rows = Ho.rows(K)
        for _, blk in Ho.neighbours(K):
            L[rows] += blk.shape[1]
            m_r[rows] = np.maximum(m_r[rows], np.abs(blk).max(axis=1))
    n_s = np.abs(X).max(axis=1)
    absref = np.abs(X) @ np.abs(Ho.dense()).T                   # |X| |H|^T for FP64's own bound
    with D.Context(H) as ctx:
        for s in (10, 4):
            Y = ctx.sliced_matvec(torch.from_numpy(X).to(dev), slices=s).cpu().numpy()
            bound = np.outer(n_s, L * m_r) * (2.0 ** (-6 * s) * (s + 4) + 6 * U) + L[None, :] * U * absref
            err = np.abs(Y - ref)
            print(f"SLICED_HX {cfg.name} s={s} max err/bound {np.max(err / bound):.3e}")
            assert np.all(err <= bound)
            if s == 4:
                assert np.max(err / np.abs(ref).max()) > 1e-14     # fewer slices are less accurate


def test_sliced_matvec_error_paths():
    wide = G.ProblemConfig(name="wide", grid=(2, 1, 1), periodic=(False, False, False), stencil="27",
                           nb=160, Ns=4, m=2, Ne=2.0, seed=1)
    Hw = G.make_blocks(wide)
    with D.Context(Hw) as ctx:
        X = torch.zeros((4, ctx.N), dtype=torch.float64, device=dev)
        with pytest.raises(D.DGChefsiError) as e:
            ctx.sliced_matvec(X)
        assert e.value.status == "ERR_UNSUPPORTED"
    H = G.make_blocks(problems()[0])
    with D.Context(H) as ctx:
        X = torch.ones((5, ctx.N), dtype=torch.float64, device=dev)
        X[2, 17] = float("nan")
        with pytest.raises(D.DGChefsiError) as e:
            ctx.sliced_matvec(X)
        assert e.value.status == "ERR_NONFINITE"
        with pytest.raises(D.DGChefsiError) as e:
            ctx.sliced_matvec(X[:1], slices=17)
        assert e.value.status == "ERR_ARG"
