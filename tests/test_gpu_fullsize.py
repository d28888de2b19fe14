"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (autotuned unit shape; the sheet through the CUDA-graph form), on
outputs the oracle can compute one by one, plus properties that hold at any
size.

* Filter: every state is filtered independently (Eq. matvec_3 acts column by
  column), so the oracle filters a few sampled states of the full block and
  each must match the GPU's row to the filter tolerance (2 m u_op relative for
  the tensor-core forms, see test_gpu_tc; 1e-12 for FP64).
* Rayleigh-Ritz after a full-size mixed filter: each Ritz value equals the
  Rayleigh quotient of its vector (lambda_i = x_i^T H x_i, H applied by the
  library's FP64 mat-vec), the occupations give 2 sum f = N_e, and the
  density blocks give 2 tr P = N_e.
"""
import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None
U_OP = {"bf16x3": 2.0 ** -16, "f64": 0.5e-12 / 20}

_full = {}


def full(name):
    if name not in _full:
        cfg = G.CONFIGS[name]
        H = G.make_blocks(cfg)
        Ns, Ne = G.resolve_sizes(cfg, H)
        X0 = G.make_X(H.N, Ns, cfg.seed)
        _full[name] = (cfg, H, O.DGHamiltonian.from_blocksparse(H), X0, G.make_start_vector(H.N, cfg.seed), Ns, Ne)
    return _full[name]


def first_cycle_bounds(ctx, v0, Ns, N):
    b, tmin = ctx.bounds(torch.from_numpy(v0).cuda(), 10)
    return tmin + (b - tmin) * Ns / N, b, tmin


def check_rows(Y, Ho, X0, rows, m, a, b, a0, tol):
    ref = O.chebyshev_filter(Ho, X0[rows].T, m, a, b, a0).T
    for k, i in enumerate(rows):
        err = np.linalg.norm(Y[k] - ref[k]) / np.linalg.norm(ref[k])
        print(f"FULL state {i} rel {err:.3e} tol {tol:.3e}")
        assert err <= tol, (i, err)


@pytest.mark.parametrize("prec", ["bf16x3", "f64"])
def test_full_bulk_filter_sampled_states(prec):
    cfg, H, Ho, X0, v0, Ns, Ne = full("bulk3d_8x8x8")
    rows = [0, 1, 255, 256, 2047, 2048, Ns - 2, Ns - 1]   # first, tile edges, last tile
    with D.Context(H) as ctx:
        a, b, a0 = first_cycle_bounds(ctx, v0, Ns, H.N)
        X = torch.from_numpy(X0).cuda()
        Y = ctx.filter(X, cfg.m, a, b, a0, prec=prec)
        Ys = Y[rows].cpu().numpy()
    check_rows(Ys, Ho, X0, rows, cfg.m, a, b, a0, 2 * cfg.m * U_OP[prec])


def test_full_bulk_mixed_cycle_properties():
    cfg, H, Ho, X0, v0, Ns, Ne = full("bulk3d_8x8x8")
    with D.Context(H) as ctx:
        a, b, a0 = first_cycle_bounds(ctx, v0, Ns, H.N)
        X = torch.from_numpy(X0).cuda()
        Y = ctx.filter(X, cfg.m, a, b, a0, prec="bf16x3")
        ritz = ctx.rayleigh_ritz(Y)                      # Y is X_new now
        HX = ctx.matvec(Y)
        q = (Y * HX).sum(dim=1)
        scale = max(abs(a0), abs(b))
        err_q = float((q - ritz).abs().max()) / scale
        f, mu = ctx.occupations(ritz, Ne, cfg.kT)
        P = ctx.density_blocks(Y, f)
        tr = sum(float(torch.trace(p)) for p in ctx.unpack_density(P))
        r = ritz.cpu().numpy()
    print(f"FULL cycle rayleigh-quotient err {err_q:.3e}, 2 tr P - Ne = {2 * tr - Ne:.3e}")
    assert np.all(np.diff(r) >= 0)
    assert err_q <= 1e-9
    assert abs(2 * float(f.sum()) - Ne) <= 1e-10 * Ne
    assert abs(2 * tr - Ne) <= 1e-8 * Ne


def test_full_sheet_graph_filter_sampled_states():
    cfg, H, Ho, X0, v0, Ns, Ne = full("sheet2d_24x20")
    rows = [0, 255, 256, Ns // 2, Ns - 1]
    with D.Context(H) as ctx:
        a, b, a0 = first_cycle_bounds(ctx, v0, Ns, H.N)
        X = torch.from_numpy(X0).cuda()
        Y = torch.empty_like(X)
        ctx.filter_graph(X, cfg.m, a, b, a0, prec="bf16x3", Y=Y)
        Ys = Y[rows].cpu().numpy()
        del X, Y
    check_rows(Ys, Ho, X0, rows, cfg.m, a, b, a0, 2 * cfg.m * U_OP["bf16x3"])
    _full.pop("sheet2d_24x20", None)


def test_full_12cubed_filter_sampled_states():
    """The differentiation workload (12^3 elements, n_b = 48: every slice only
    partly filled) through the BF16x3 filter at full size."""
    cfg, H, Ho, X0, v0, Ns, Ne = full("bulk3d_12x12x12")
    rows = [0, 256, Ns // 2, Ns - 1]
    with D.Context(H) as ctx:
        a, b, a0 = first_cycle_bounds(ctx, v0, Ns, H.N)
        X = torch.from_numpy(X0).cuda()
        Y = ctx.filter(X, cfg.m, a, b, a0, prec="bf16x3")
        Ys = Y[rows].cpu().numpy()
        del X, Y
    check_rows(Ys, Ho, X0, rows, cfg.m, a, b, a0, 2 * cfg.m * U_OP["bf16x3"])
    _full.pop("bulk3d_12x12x12", None)
