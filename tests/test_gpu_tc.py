"""GPU parity of the tensor-core filter (TF32, BF16, split BF16x3) against the FP64
oracle, through the C ABI.

Comparisons are blockwise: for every state (row of Y) and for every element
block (the columns of one element K over all states) the relative error
||Y - Y_ref|| / ||Y_ref|| must stay within the tolerance, so a dropped
neighbour block of one element or a wrong 128-state tile cannot hide in the
norm of the whole block.

Tolerance against the FP64 filter: each recurrence step rounds its operands
to the tensor format (relative error u_op of a product: 2^-9 for TF32, whose
tensor core drops the low 13 mantissa bits of both factors, errors of the
same sign that add; 2^-8 for BF16; about 2^-16 for the hi/lo split, whose
missing lo*lo term and rounded lo are of order 2^-18 and whose FP32
accumulation over the neighbour sum adds ~2^-20) and the error of each step
is carried forward by the bounded scaled recurrence, so the filtered block
carries at most about m * u_op. The test allows 2 m u_op.

BF16 and TF32 are also compared with the oracle's filter that applies the
same operand roundings (oracle.chebyshev_filter_rounded). What is left
between the two is the order of the FP32 accumulation (~2^-24 sqrt(27 * 64)
~ 2.5e-6 of a product per step) and the operand roundings it flips (a
fraction ~1e-3 of the BF16 entries by 2^-8 each, ~1e-4 normwise per step),
so m 2^-10 is a bound with a wide margin; it is 8 (TF32) to 16 (BF16) times
tighter than 2 m u_op, tight enough to reject a dropped neighbour block.
"""
import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None

U_OP = {"tf32": 2.0 ** -9, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16}


def blockwise_errors(Y, ref, Ho):
    """Largest relative error over states (rows) and over element blocks (columns
    of one element, all states). A block is measured against its own norm or,
    when that is smaller, its share of the whole block's norm
    (||ref|| sqrt(rows/N_s) for a state, ||ref|| sqrt(n_K/N) for an element):
    the rounding error of a block scales with the sizes of the terms summed
    into it, not with what is left after they cancel, so a block whose filtered
    values happen to be small is not held to a tighter bound than its share."""
    d = Y - ref
    tot = max(np.linalg.norm(ref), 1e-300)
    Ns = ref.shape[0]
    st = np.linalg.norm(d, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), tot / np.sqrt(Ns))
    el = [np.linalg.norm(d[:, Ho.rows(K)]) / max(np.linalg.norm(ref[:, Ho.rows(K)]), tot * np.sqrt(Ho.nb[K] / Ho.N))
          for K in range(Ho.M)]
    return float(np.max(st)), float(np.max(el))


def blockwise_ok(Y, ref, Ho, tol):
    st, el = blockwise_errors(Y, ref, Ho)
    return np.isfinite(Y).all() and st <= tol and el <= tol


def assert_blockwise(Y, ref, Ho, tol, what=""):
    st, el = blockwise_errors(Y, ref, Ho)
    assert np.isfinite(Y).all(), what
    assert st <= tol and el <= tol, f"{what}: per-state {st:.3e}, per-element {el:.3e}, tolerance {tol:.3e}"


def emulated_tol(m):
    return m * 2.0 ** -10


def problems():
    tiny = G.CONFIGS["tiny_2x2x2"]
    bulk = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(4, 4, 4), nb=64, Ns=300, m=12, name="bulk4")
    uneven = G.ProblemConfig(name="uneven", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                             nb=(40, 120), Ns=200, m=7, Ne=150.0, seed=5)
    sheet = G.scaled_copy(G.CONFIGS["sheet2d_24x20"], grid=(4, 3, 1), Ns=130, m=9, name="sheet")
    return [tiny, bulk, uneven, sheet]


_cache = {}


def problem(cfg):
    if cfg.name not in _cache:
        H, X0, v0, Ns, Ne = G.make_problem(cfg)
        Ho = O.DGHamiltonian.from_blocksparse(H)
        _cache[cfg.name] = (H, Ho, X0, v0, Ns, Ne, np.linalg.eigvalsh(Ho.dense()))
    return _cache[cfg.name]


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_filter_tc_matches_oracle(cfg, prec):
    H, Ho, X0, _, Ns, _, lam = problem(cfg)
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[min(Ns, Ho.N - 1)]
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        for m in sorted({1, 2, cfg.m}):
            Y = ctx.filter(torch.from_numpy(X0).to(dev), m, a, b, a0, prec=prec).cpu().numpy()
            ref = O.chebyshev_filter(Ho, X0.T, m, a, b, a0).T
            st, el = blockwise_errors(Y, ref, Ho)
            print(f"FILTER_ERR {cfg.name} {prec} m={m} state={st:.3e} element={el:.3e} "
                  f"bound={2 * m * U_OP[prec]:.3e}")
            assert_blockwise(Y, ref, Ho, 2 * m * U_OP[prec], f"{cfg.name} {prec} m={m}")
            if prec in ("bf16", "tf32"):
                em = O.chebyshev_filter_rounded(Ho, X0.T, m, a, b, a0, prec).T
                st, el = blockwise_errors(Y, em, Ho)
                print(f"FILTER_EMU_ERR {cfg.name} {prec} m={m} state={st:.3e} element={el:.3e} "
                      f"bound={emulated_tol(m):.3e}")
                assert_blockwise(Y, em, Ho, emulated_tol(m), f"{cfg.name} {prec} m={m} vs rounded oracle")


def _drop_block(Ho, K, Kp):
    """H with the block (K, K') zeroed, as a kernel that skipped element K's
    neighbour slice K' would see it (the mirror block (K', K) is kept)."""
    vals = Ho.values.copy()
    for e in range(Ho.row_ptr[K], Ho.row_ptr[K + 1]):
        if int(Ho.col[e]) == Kp:
            vals[Ho.blk_off[e]:Ho.blk_off[e] + int(Ho.nb[K]) * int(Ho.nb[Kp])] = 0.0
    return O.DGHamiltonian(Ho.nb, Ho.row_ptr, Ho.col, Ho.blk_off, vals)


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
def test_blockwise_comparison_rejects_a_dropped_neighbour_block(prec):
    """Planted fault, built on the host: the filter of the 4x4x4 copy with one
    face block of element 5 left out, rounded the way the form rounds. The
    comparison the parity tests use must reject it, while the GPU result
    passes the same comparison."""
    cfg = problems()[1]
    H, Ho, X0, _, Ns, _, lam = problem(cfg)
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[min(Ns, Ho.N - 1)]
    m = cfg.m
    bad_H = _drop_block(Ho, 5, 4)
    if prec == "bf16x3":
        ref, bad, tol = (O.chebyshev_filter(Ho, X0.T, m, a, b, a0).T, O.chebyshev_filter(bad_H, X0.T, m, a, b, a0).T,
                         2 * m * U_OP[prec])
    else:
        ref = O.chebyshev_filter_rounded(Ho, X0.T, m, a, b, a0, prec).T
        bad = O.chebyshev_filter_rounded(bad_H, X0.T, m, a, b, a0, prec).T
        tol = emulated_tol(m)
    st, el = blockwise_errors(bad, ref, Ho)
    print(f"PLANTED {prec} state={st:.3e} element={el:.3e} tol={tol:.3e}")
    assert not blockwise_ok(bad, ref, Ho, tol)
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        Y = ctx.filter(torch.from_numpy(X0).to(dev), m, a, b, a0, prec=prec).cpu().numpy()
    assert blockwise_ok(Y, ref, Ho, tol)


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
def test_filter_tc_ragged_states_and_strides(prec):
    """N_s not a multiple of the 128-state tile, a row stride wider than N, and
    the padding of the caller's block left untouched."""
    H, Ho, X0, _, _, _, lam = problem(problems()[2])
    Ns = 131
    dev = torch.device("cuda:0")
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[Ns]
    with D.Context(H) as ctx:
        big = torch.full((Ns, Ho.N + 5), 3.0, dtype=torch.float64, device=dev)
        big[:, :Ho.N] = torch.from_numpy(X0[:Ns])
        out = torch.full_like(big, -7.0)
        ctx.filter(big[:, :Ho.N], 5, a, b, a0, prec=prec, Y=out[:, :Ho.N])
        ref = O.chebyshev_filter(Ho, X0[:Ns].T, 5, a, b, a0).T
        Y = out[:, :Ho.N].cpu().numpy()
        assert_blockwise(Y, ref, Ho, 10 * U_OP[prec], f"ragged {prec}")
        assert torch.all(out[:, Ho.N:] == -7.0)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "tf32"])
def test_mixed_cycles_converge(prec):
    """Mixed-precision filter + FP64 Rayleigh-Ritz on the tiny 2x2x2 problem:
    after 20 cycles the lowest N_s - 8 Ritz values agree with a dense eigensolve.
    The split BF16 filter must reach the 1e-8 target; one rounding of BF16 or
    TF32 operands per step leaves a floor of order u_op^2 * spread."""
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, Ho, X0, v0, Ns, Ne, lam = problem(cfg)
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        prev = None
        for _ in range(cfg.cycles):
            out = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v, prev_ritz=prev, prec=prec)
            prev = out["ritz"].cpu().numpy()
    g = 8
    scale = max(abs(lam[0]), abs(lam[-1]))
    err = np.max(np.abs(prev[:Ns - g] - lam[:Ns - g])) / scale
    print(f"RITZ_ERR tiny {prec} {err:.3e}")
    limit = {"bf16x3": 1e-8, "tf32": 1e-4, "bf16": 1e-3}[prec]
    assert err <= limit


SHAPES = {32: [(4, 2, 0), (2, 2, 0), (4, 2, 1), (4, 2, 2)], 64: [(2, 2, 0), (1, 2, 0), (2, 1, 0), (2, 2, 1), (2, 2, 2)],
          128: [(2, 1, 0), (1, 2, 0), (1, 2, 1), (1, 2, 2)]}


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "tf32"])
@pytest.mark.parametrize("cfg", problems()[:3], ids=lambda c: c.name)
def test_every_unit_shape_matches_oracle(cfg, prec):
    """Each work-unit shape the autotuner may pick gives the same filter."""
    H, Ho, X0, _, Ns, _, lam = problem(cfg)
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[min(Ns, Ho.N - 1)]
    ref = O.chebyshev_filter(Ho, X0.T, cfg.m, a, b, a0).T
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        acc = 32 if Ho.nb.max() <= 32 else (64 if Ho.nb.max() <= 64 else 128)
        for G, T, lay in SHAPES[acc]:
            ctx.set_tile_shape(prec, G, T, lay)
            assert ctx.tile_shape(prec) == (G, T, acc, lay)
            Y = ctx.filter(torch.from_numpy(X0).to(dev), cfg.m, a, b, a0, prec=prec).cpu().numpy()
            st, el = blockwise_errors(Y, ref, Ho)
            print(f"SHAPE_ERR {cfg.name} {prec} G={G} T={T} layout={lay} state={st:.3e} element={el:.3e}")
            assert_blockwise(Y, ref, Ho, 2 * cfg.m * U_OP[prec], f"{cfg.name} {prec} G={G} T={T} layout={lay}")
        ctx.set_tile_shape(prec, 0, 0)  # back to the autotuner
        ctx.filter(torch.from_numpy(X0).to(dev), 2, a, b, a0, prec=prec)
        G, T, _, lay = ctx.tile_shape(prec)
        assert (G, T, lay) in SHAPES[acc]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_graph_filter_equals_direct_filter(prec):
    """The CUDA-graph replay gives bit-identical results to ordinary launches,
    also after the bounds (hence the recurrence coefficients) change."""
    H, Ho, X0, _, Ns, _, lam = problem(problems()[2])   # uneven element sizes
    dev = torch.device("cuda:0")
    X = torch.from_numpy(X0).to(dev)
    with D.Context(H) as ctx:
        Yg = torch.empty_like(X)
        for shift in (0.5, 1.5, 0.5):
            a0, b, a = lam[0] - shift, lam[-1] + shift, lam[Ns]
            Yd = ctx.filter(X, 7, a, b, a0, prec=prec)
            ctx.filter_graph(X, 7, a, b, a0, prec=prec, Y=Yg)
            assert torch.equal(Yd, Yg), shift
        ref = O.chebyshev_filter(Ho, X0.T, 7, lam[Ns], lam[-1] + 0.5, lam[0] - 0.5).T
        assert_blockwise(Yg.cpu().numpy(), ref, Ho, 14 * U_OP[prec], f"graph {prec}")
    with D.Context(H) as ctx:  # the FP64 graph replays the FP64 steps bit for bit
        Yg = torch.empty_like(X)
        for shift in (0.5, 1.5):
            a0, b, a = lam[0] - shift, lam[-1] + shift, lam[Ns]
            Yd = ctx.filter(X, 6, a, b, a0, prec="f64")
            ctx.filter_graph(X, 6, a, b, a0, prec="f64", Y=Yg)
            torch.cuda.synchronize()
            assert torch.equal(Yd, Yg), shift


@pytest.mark.parametrize("prec", ["bf16x3", "f64"])
def test_graph_recaptured_after_buffers_move(prec):
    """A direct call with more states regrows the library's iterate buffers
    between two graph calls of the same shape; the second graph call must
    capture again (not replay a graph that refers to freed memory) and still
    give the direct result."""
    H, Ho, X0, _, Ns, _, lam = problem(problems()[1])
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[Ns]
    X = torch.from_numpy(X0[:100]).to(torch.device("cuda:0"))
    Xbig = torch.from_numpy(X0).to(torch.device("cuda:0"))
    with D.Context(H) as ctx:
        Yg = torch.empty_like(X)
        ctx.filter_graph(X, 5, a, b, a0, prec=prec, Y=Yg)
        ctx.filter(Xbig, 5, a, b, a0, prec=prec)          # regrows the workspace / iterates
        ctx.filter_graph(X, 5, a, b, a0, prec=prec, Y=Yg)
        torch.cuda.synchronize()
        assert torch.equal(Yg, ctx.filter(X, 5, a, b, a0, prec=prec))


def edge_problems():
    one = G.ProblemConfig(name="one_element", grid=(1, 1, 1), periodic=(False, False, False), stencil="27",
                          nb=5, Ns=3, m=4, Ne=2.0, seed=1)
    ones = G.ProblemConfig(name="unit_elements", grid=(4, 1, 1), periodic=(True, False, False), stencil="27",
                           nb=1, Ns=2, m=3, Ne=2.0, seed=2)
    odd = G.ProblemConfig(name="odd_sizes", grid=(3, 1, 1), periodic=(False, False, False), stencil="27",
                          nb=(7, 21), Ns=1, m=5, Ne=1.0, seed=3)
    return [one, ones, odd]


@pytest.mark.parametrize("cfg", edge_problems(), ids=lambda c: c.name)
def test_edge_shapes_filter_and_rayleigh_ritz(cfg):
    """One element, 1-wide elements, odd element sizes, a single state: every
    precision of the filter and the FP64 Rayleigh-Ritz still match the oracle."""
    H, X0, _, Ns, Ne = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    lam = np.linalg.eigvalsh(Ho.dense())
    a0, b = lam[0] - 0.5, lam[-1] + 0.5
    a = 0.5 * (lam[0] + lam[-1]) if Ho.N <= Ns else lam[Ns]
    dev = torch.device("cuda:0")
    ref = O.chebyshev_filter(Ho, X0.T, cfg.m, a, b, a0).T
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        for prec in ("f64", "tf32", "bf16", "bf16x3"):
            Y = ctx.filter(X, cfg.m, a, b, a0, prec=prec).cpu().numpy()
            tol = 1e-11 if prec == "f64" else 2 * cfg.m * U_OP[prec]
            assert_blockwise(Y, ref, Ho, tol, f"{cfg.name} {prec}")
        Yg = torch.from_numpy(np.ascontiguousarray(ref)).to(dev)
        ritz = ctx.rayleigh_ritz(Yg).cpu().numpy()
    Yh, _, _ = O.cholesky_qr(ref.T)
    _, Do, _ = O.rayleigh_ritz(Ho, Yh)
    assert np.max(np.abs(ritz - Do)) <= 1e-10 * max(abs(a0), abs(b))


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "f64"])
def test_filter_host_equals_device_filter(prec):
    """dgchefsi_filter_host pipelines chunks of states between host and device;
    each state is filtered independently, so every chunking gives the device
    filter's result bit for bit, for pinned, strided and pageable host blocks."""
    H, Ho, X0, _, Ns, _, lam = problem(problems()[1])   # N_s = 300: ragged last chunk
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[Ns]
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        ref = ctx.filter(torch.from_numpy(X0).to(dev), 6, a, b, a0, prec=prec).cpu()
        Xh = torch.from_numpy(X0).pin_memory()
        for chunk in (0, 100, 1000):
            Yh = ctx.filter_host(Xh, 6, a, b, a0, prec=prec, chunk=chunk)
            assert torch.equal(Yh, ref), chunk
        big = torch.full((Ns, Ho.N + 9), 2.0, dtype=torch.float64).pin_memory()
        big[:, :Ho.N] = torch.from_numpy(X0)
        out = torch.full((Ns, Ho.N + 9), -1.0, dtype=torch.float64).pin_memory()
        ctx.filter_host(big[:, :Ho.N], 6, a, b, a0, prec=prec, Y=out[:, :Ho.N], chunk=128)
        assert torch.equal(out[:, :Ho.N], ref)
        assert torch.all(out[:, Ho.N:] == -1.0)
        Yp = ctx.filter_host(torch.from_numpy(X0.copy()), 6, a, b, a0, prec=prec)   # pageable
        assert torch.equal(Yp, ref)
