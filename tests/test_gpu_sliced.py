"""FP64 products rebuilt from exact BF16 slices on the tensor cores (the Ozaki
scheme) and the Rayleigh-Ritz step / cycle that uses them, through the C ABI.

* Integer operands of at most 12 bits: every slice is exact after two slices,
  every slice-pair product is an exactly accumulated integer, and the FP64
  sums are exact, so the result equals the exact integer product bit for bit
  (ragged K chunks, strided operands, both operand layouts, triangular A,
  several column panels, pair sums at the 2^24 edge of exact FP32
  accumulation). The slice pairs run on the library's tcgen05 step kernel.
* Gaussian operands with rows scaled over e^{+-3}: |C - A B| within the
  splitting bound sum over chunks of L m_r n_c (2^{-6s}(s + 4) + (5 + chunks) u)
  plus FP64's own bound on the reference product; fewer slices are less
  accurate.
* Cycles with the sliced products match the FP64 oracle at the FP64 path's
  tolerances (Ritz values 1e-10 of max(|a0|, |b|), density blocks 1e-9), on
  blocks with one and with several K chunks, and the tiny problem converges
  to the dense spectrum.
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
L_CHUNK = 4096


def tiny_ctx():
    H, _, _, _, _ = G.make_problem(G.CONFIGS["tiny_2x2x2"])
    return D.Context(H)


def strided(a, pad=3, fill=7.0):
    """a as a CUDA tensor whose rows are `pad` entries longer than its width."""
    big = torch.full((a.shape[0], a.shape[1] + pad), fill, dtype=torch.float64, device=dev)
    big[:, :a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a))
    return big[:, :a.shape[1]]


@pytest.mark.parametrize("b_rows,a_lower", [(True, False), (False, False), (False, True), (True, True)])
@pytest.mark.parametrize("slices", [3, 10])
def test_integer_operands_bit_exact(b_rows, a_lower, slices):
    rng = np.random.default_rng(11)
    M, Nc, K = 190, 333, 2 * L_CHUNK + 1000
    A = rng.integers(-2047, 2048, size=(M, K)).astype(np.int64)
    A[5] = rng.integers(-5, 6, size=K)           # a row of small integers (one slice)
    Bm = rng.integers(-2047, 2048, size=(Nc, K) if b_rows else (K, Nc)).astype(np.int64)
    Aeff = np.tril(A) if a_lower else A
    ref = (Aeff @ (Bm.T if b_rows else Bm)).astype(np.float64)   # exact: |entries| < 2^36
    with tiny_ctx() as ctx:
        out = torch.full((M, Nc + 5), -1.0, dtype=torch.float64, device=dev)
        ctx.sliced_gemm(strided(A.astype(np.float64)), strided(Bm.astype(np.float64), pad=8), b_rows=b_rows,
                        a_lower=a_lower, slices=slices, out=out[:, :Nc])
        got = out.cpu().numpy()
    assert np.array_equal(got[:, :Nc], ref)
    assert np.all(got[:, Nc:] == -1.0)


@pytest.mark.parametrize("case", ["gram_same", "gram_two", "stacked", "panels"])
def test_lower_triangle_only_bit_exact(case):
    """tri > 0: only the entries C[r, c] with c <= r mod tri are formed, bit
    for bit the exact integer product, and every other entry keeps its value.
    A symmetric Gram with A == B (one slice set) and with two operands, two
    stacked symmetric products (tri = M / 2, the refinement's [G; S] form),
    both over ragged tiles and K chunks, and a product wide enough (16 slices)
    to run in column panels, where the line is followed across panels."""
    rng = np.random.default_rng(21)
    slices = 10
    if case == "panels":
        M = Nc = 4500
        K, slices, tri = 300, 16, 4500
        assert 136 * 4 * M * Nc > 8 * 2 ** 30
    elif case == "stacked":
        M, Nc, K, tri = 1200, 600, 5000, 600
    else:
        M = Nc = 700
        K, tri = 2 * L_CHUNK + 900, 700
    A = rng.integers(-2047, 2048, size=(M, K)).astype(np.int64)
    if case == "stacked":
        A[:Nc] = rng.integers(-2047, 2048, size=(Nc, K))
        Bt = A[:Nc].copy()
    elif case in ("gram_same", "panels"):
        Bt = A
    else:
        Bt = rng.integers(-2047, 2048, size=(Nc, K)).astype(np.int64)
    ref = (A @ Bt.T).astype(np.float64)
    r = np.arange(M)[:, None]
    c = np.arange(Nc)[None, :]
    want = c <= r % tri
    with tiny_ctx() as ctx:
        At = torch.from_numpy(A.astype(np.float64)).to(dev)
        Bd = At if case in ("gram_same", "panels") else torch.from_numpy(Bt.astype(np.float64)).to(dev)
        out = torch.full((M, Nc), -1.0, dtype=torch.float64, device=dev)
        ctx.sliced_gemm(At, Bd, b_rows=True, slices=slices, out=out, tri=tri)
        got = out.cpu().numpy()
    assert np.array_equal(got[want], ref[want])
    assert np.all(got[~want] == -1.0)


@pytest.mark.parametrize("b_rows", [True, False])
def test_pair_sums_at_the_fp32_limit_bit_exact(b_rows):
    """One full K chunk (4096) of same-sign operands whose digits reach their
    bounds: 4064 = 2^12 - 32 splits (row exponent 12) into q_0 = 64, q_1 = -32,
    so the slice pairs sum to 64 * 64 * 4096 = 2^24, -2^23 and 2^22 exactly at
    the edge of exact FP32 accumulation. The other rows and columns are
    positive integers below 4064. The result must equal the exact integer
    product bit for bit."""
    rng = np.random.default_rng(5)
    M, Nc, K = 70, 90, L_CHUNK
    A = rng.integers(2000, 4065, size=(M, K)).astype(np.int64)
    A[:3] = 4064
    Bt = rng.integers(2000, 4065, size=(Nc, K)).astype(np.int64)
    Bt[:4] = 4064
    ref = (A @ Bt.T).astype(np.float64)                     # exact: entries < 2^37
    assert ref[0, 0] == 4096 * 4064 ** 2
    B = Bt if b_rows else np.ascontiguousarray(Bt.T)
    with tiny_ctx() as ctx:
        out = torch.empty((M, Nc), dtype=torch.float64, device=dev)
        ctx.sliced_gemm(torch.from_numpy(A.astype(np.float64)).to(dev), torch.from_numpy(B.astype(np.float64)).to(dev),
                        b_rows=b_rows, slices=10, out=out)
        got = out.cpu().numpy()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("b_rows", [True, False])
def test_integer_operands_bit_exact_over_column_panels(b_rows):
    """16 slices (136 pairs, digits by the FP64 path) on a 2048 x 8000 output:
    the FP32 pair slabs exceed the 8 GB workspace cap, so the columns run in
    two panels of 128-column tiles, the second one ragged."""
    rng = np.random.default_rng(9)
    M, Nc, K = 2048, 8000, 300
    assert 136 * 4 * M * Nc > 8 * 2 ** 30
    A = rng.integers(-2047, 2048, size=(M, K)).astype(np.int64)
    Bt = rng.integers(-2047, 2048, size=(Nc, K)).astype(np.int64)
    ref = (A @ Bt.T).astype(np.float64)
    B = Bt if b_rows else np.ascontiguousarray(Bt.T)
    with tiny_ctx() as ctx:
        out = torch.empty((M, Nc), dtype=torch.float64, device=dev)
        ctx.sliced_gemm(torch.from_numpy(A.astype(np.float64)).to(dev), torch.from_numpy(B.astype(np.float64)).to(dev),
                        b_rows=b_rows, slices=16, out=out)
        got = out.cpu().numpy()
    assert np.array_equal(got, ref)


def splitting_bound(A, B, s, balance=False):
    """Sum over K chunks of L m_r n_c (2^{-6s}(s + 4) + (5 + chunks) u), B given
    as the rows of the right operand's transpose. balance: the operands as the
    A B form splits them, column k of A times 2^{s_k} and row k of the right
    operand times 2^{-s_k}, s_k the exponent of that row's maximum."""
    if balance:
        sk = np.frexp(np.abs(B).max(axis=0))[1]
        A, B = np.ldexp(A, sk[None, :]), np.ldexp(B, -sk[None, :])
    K = A.shape[1]
    nch = -(-K // L_CHUNK)
    bound = np.zeros((A.shape[0], B.shape[0]))
    for c in range(nch):
        a = A[:, c * L_CHUNK:(c + 1) * L_CHUNK]
        b = B[:, c * L_CHUNK:(c + 1) * L_CHUNK]
        L = a.shape[1]
        bound += L * np.outer(np.abs(a).max(1), np.abs(b).max(1)) * (2.0 ** (-6 * s) * (s + 4) + (5 + nch) * U)
    return bound


@pytest.mark.parametrize("b_rows", [True, False])
def test_gaussian_operands_within_bound(b_rows):
    rng = np.random.default_rng(3)
    M, Nc, K = 256, 320, 2 * L_CHUNK + 808
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((Nc, K)) * np.exp(rng.uniform(-3, 3, (Nc, 1)))   # B as rows of B^T
    ref = A @ B.T
    absab = np.abs(A) @ np.abs(B).T
    gamma = K * U / (1 - K * U)
    errs = {}
    with tiny_ctx() as ctx:
        Bd = torch.from_numpy(B if b_rows else np.ascontiguousarray(B.T)).to(dev)
        for s in (7, 10):
            got = ctx.sliced_gemm(torch.from_numpy(A).to(dev), Bd, b_rows=b_rows, slices=s).cpu().numpy()
            err = np.abs(got - ref)
            assert np.all(err <= splitting_bound(A, B, s, balance=not b_rows) + gamma * absab), s
            errs[s] = float(np.max(err / absab))
    print(f"SLICED b_rows={b_rows} max |C - A B| / (|A||B|): s=7 {errs[7]:.2e}, s=10 {errs[10]:.2e}")
    assert errs[10] <= 1e-15 < errs[7]


def test_edge_sizes_and_errors():
    rng = np.random.default_rng(5)
    with tiny_ctx() as ctx:
        A = torch.empty((7, 0), dtype=torch.float64, device=dev)
        B = torch.empty((9, 0), dtype=torch.float64, device=dev)
        out = torch.full((7, 9), 3.0, dtype=torch.float64, device=dev)
        ctx.sliced_gemm(A, B, out=out)                      # K = 0: C = 0
        assert torch.all(out == 0.0)
        A1 = rng.standard_normal((1, 5))
        B1 = rng.standard_normal((1, 5))
        got = ctx.sliced_gemm(torch.from_numpy(A1).to(dev), torch.from_numpy(B1).to(dev)).item()
        assert abs(got - (A1 @ B1.T).item()) <= 1e-15 * (np.abs(A1) @ np.abs(B1).T).item()
        Abad = torch.from_numpy(rng.standard_normal((20, 50))).to(dev)
        Abad[3, 7] = float("nan")
        with pytest.raises(D.DGChefsiError) as e:
            ctx.sliced_gemm(Abad, torch.from_numpy(rng.standard_normal((4, 50))).to(dev))
        assert e.value.status == "ERR_NONFINITE"
        for s in (1, 17):
            with pytest.raises(D.DGChefsiError) as e:
                ctx.sliced_gemm(Abad, Abad, slices=s)
            assert e.value.status == "ERR_ARG"
            with pytest.raises(D.DGChefsiError) as e:
                ctx.set_subspace_products("sliced_bf16", s)
            assert e.value.status == "ERR_ARG"
        with pytest.raises(D.DGChefsiError) as e:
            D._check(D._lib.dgchefsi_set_subspace_products(ctx._h, 5, 10))
        assert e.value.status == "ERR_ARG"


def cycle_configs():
    tiny = G.CONFIGS["tiny_2x2x2"]
    uneven = G.ProblemConfig(name="uneven", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                             nb=(40, 120), Ns=100, m=7, Ne=150.0, seed=5)
    bulk = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(5, 4, 4), nb=64, Ns=200, m=10, name="bulk5x4x4")
    return [tiny, uneven, bulk]   # N = 256, ~1000, 5120 (two K chunks, the second ragged)


@pytest.mark.parametrize("cfg", cycle_configs(), ids=lambda c: c.name)
def test_cycles_with_sliced_products_match_oracle(cfg):
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    with D.Context(H) as ctx:
        ctx.set_subspace_products("sliced_bf16", 10)
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        prev = None
        for cyc in range(3):
            Xin = X.cpu().numpy().T.copy()
            out = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v, prev_ritz=prev)
            a, b, a0 = out["bounds"]
            ref = O.chefsi_cycle(Ho, Xin, cfg.m, Ne, cfg.kT, v0, bounds=(a, b, a0))
            scale = max(abs(a0), abs(b))
            ritz = out["ritz"].cpu().numpy()
            er = np.max(np.abs(ritz - ref["ritz"])) / scale
            Pr = O.packed_density(Ho, ref["P"])
            ep = np.linalg.norm(out["P"].cpu().numpy() - Pr) / np.linalg.norm(Pr)
            print(f"SLICED cycle {cfg.name} {cyc}: ritz {er:.2e}, density {ep:.2e}")
            assert er <= 1e-10 and ep <= 1e-9, cyc
            prev = ritz


def test_tiny_converges_with_sliced_products():
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    lam = np.linalg.eigvalsh(O.DGHamiltonian.from_blocksparse(H).dense())
    with D.Context(H) as ctx:
        ctx.set_subspace_products("sliced_bf16")
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        prev = None
        for _ in range(cfg.cycles):
            prev = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v, prev_ritz=prev)["ritz"].cpu().numpy()
    g = 8
    assert np.max(np.abs(prev[:Ns - g] - lam[:Ns - g])) <= 1e-10 * max(abs(lam[0]), abs(lam[-1]))


def test_full_bulk_rayleigh_ritz_sliced_vs_f64_products():
    """8x8x8 workload (N = 32768, N_s = 4096: eight K chunks for the Gram and
    projected-H products, 4096 for the triangular and rotation products), in
    the bench's configuration: a BF16x3-filtered block after one mixed cycle
    (warm), Rayleigh-Ritz with FP64 products and with sliced products from the
    same block. Ritz values agree to the FP64 tolerance, the rotated blocks are
    orthonormal, and the density blocks of the occupied states agree."""
    cfg = G.CONFIGS["bulk3d_8x8x8"]
    H = G.make_blocks(cfg)
    Ns, Ne = G.resolve_sizes(cfg, H)
    X0 = G.make_X(H.N, Ns, cfg.seed)
    v0 = G.make_start_vector(H.N, cfg.seed)
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).cuda()
        out = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=torch.from_numpy(v0).cuda(), prec="bf16x3")
        r = out["ritz"].cpu().numpy()
        b = out["bounds"][1]
        Y = ctx.filter(X, cfg.m, float(r[-1]), b, float(r[0]), prec="bf16x3")
        Y2 = Y.clone()
        ritz = {}
        P = {}
        for mode, Yb in (("f64", Y), ("sliced_bf16", Y2)):
            ctx.set_subspace_products(mode)
            ritz[mode] = ctx.rayleigh_ritz(Yb)
            f, _ = ctx.occupations(ritz[mode], Ne, cfg.kT)
            P[mode] = ctx.density_blocks(Yb, f)
            G_ = Yb @ Yb.T
            G_.diagonal().sub_(1.0)
            assert float(G_.abs().max()) <= 1e-12, mode
        scale = max(abs(float(r[0])), abs(b))
        er = float((ritz["f64"] - ritz["sliced_bf16"]).abs().max()) / scale
        ep = float(torch.linalg.norm(P["f64"] - P["sliced_bf16"]) / torch.linalg.norm(P["f64"]))
    print(f"SLICED full 8x8x8 warm: ritz {er:.2e}, density {ep:.2e}")
    assert er <= 1e-10 and ep <= 1e-9


def adjoint_case(kind):
    if kind == "small":
        cfg = G.ProblemConfig(name="adj", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                              nb=(4, 7), Ns=10, m=6, Ne=10.0, seed=11, kT=0.3)
    elif kind == "tiny":
        cfg = G.scaled_copy(G.CONFIGS["tiny_2x2x2"], Ns=48, m=7, Ne=64.0)
        cfg = G.ProblemConfig(**{**cfg.__dict__, "kT": 0.05})
    else:
        cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(3, 3, 3), nb=16, Ns=64, m=9, Ne=96.0)
    H, X0, _, Ns, Ne = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    lam = np.linalg.eigvalsh(Ho.dense())
    return cfg, H, Ho, X0, Ns, Ne, (lam[min(Ns + 3, len(lam) - 1)], lam[-1] + 0.3, lam[0] - 0.3)


@pytest.mark.parametrize("kind", ["small", "tiny", "bulk3"])
def test_band_energy_gradient_with_sliced_products_matches_oracle(kind):
    """The band-energy adjoint with the sliced products against the oracle's
    adjoint, at the FP64 path's tolerances (E 1e-11, dE/dH and dE/dX 1e-8 of
    their largest entry)."""
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = adjoint_case(kind)
    E_o, G_o, Xb_o = O.band_energy_grad(Ho, X0.T, cfg.m, a, b, a0, Ne, cfg.kT)
    with D.Context(H) as ctx:
        ctx.set_subspace_products("sliced_bf16")
        E, _, Hb, Xb = ctx.energy_grad(torch.from_numpy(X0).to(dev), cfg.m, a, b, a0, Ne, cfg.kT)
    Gflat = np.concatenate([g.ravel() for g in G_o])
    eH = float(np.max(np.abs(Hb.cpu().numpy() - Gflat)) / np.max(np.abs(Gflat)))
    eX = float(np.max(np.abs(Xb.cpu().numpy() - Xb_o.T)) / np.max(np.abs(Xb_o)))
    print(f"SLICED adjoint {kind}: E {abs(E - E_o) / abs(E_o):.2e}, dE/dH {eH:.2e}, dE/dX {eX:.2e}")
    assert abs(E - E_o) <= 1e-11 * abs(E_o) and eH <= 1e-8 and eX <= 1e-8


@pytest.mark.parametrize("prec", ["f64", "bf16x3"])
def test_band_energy_gradient_sliced_vs_f64_products_two_chunks(prec):
    """N = 5120 (two K chunks): with either filter form, the gradient with
    sliced products equals the one with FP64-core products to the FP64
    tolerances."""
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(5, 4, 4), nb=64, Ns=200, m=10, Ne=300.0, name="adj5x4x4")
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        b, tmin = ctx.bounds(torch.from_numpy(v0).to(dev), 10)
        a0, a = tmin, tmin + (b - tmin) * Ns / H.N
        E0, _, H0, X0b = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, prec=prec)
        ctx.set_subspace_products("sliced_bf16")
        E1, _, H1, X1b = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, prec=prec)
    eH = float((H1 - H0).abs().max() / H0.abs().max())
    eX = float((X1b - X0b).abs().max() / X0b.abs().max())
    print(f"SLICED adjoint 5x4x4 {prec}: E {abs(E1 - E0) / abs(E0):.2e}, dE/dH {eH:.2e}, dE/dX {eX:.2e}")
    assert abs(E1 - E0) <= 1e-11 * abs(E0) and eH <= 1e-8 and eX <= 1e-8
