"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerances (FP64 on both sides, only the summation order differs):
  * mat-vec, filter, density blocks: max |GPU - oracle| <= 1e-11 * max |oracle|
  * Lanczos bound: 1e-10 relative (same start vector, same step order)
  * Ritz values: |d lambda_i| <= 1e-10 * max(|a0|, |b|) (normwise; lambda may be ~0)
  * occupations: 1e-10 absolute on f (f in [0, 1]), 1e-10 * scale on mu
X_new itself is not unique (signs, degenerate Ritz pairs), so the rotated
block is compared through the density blocks, which are.
"""
import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None


def problems():
    tiny = G.CONFIGS["tiny_2x2x2"]
    uneven = G.ProblemConfig(name="uneven", grid=(3, 2, 2), periodic=(True, False, True), stencil="27",
                             nb=(40, 120), Ns=100, m=7, Ne=150.0, seed=5)
    bulk = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(4, 4, 4), nb=64, Ns=300, m=12, name="bulk4")
    sheet = G.scaled_copy(G.CONFIGS["sheet2d_24x20"], grid=(4, 3, 1), Ns=130, m=9, name="sheet")
    return [tiny, uneven, bulk, sheet]


_cache = {}


def problem(cfg):
    if cfg.name not in _cache:
        H, X0, v0, Ns, Ne = G.make_problem(cfg)
        _cache[cfg.name] = (H, O.DGHamiltonian.from_blocksparse(H), X0, v0, Ns, Ne)
    return _cache[cfg.name]


def spectrum(cfg):
    key = cfg.name + ":eig"
    if key not in _cache:
        _cache[key] = np.linalg.eigvalsh(problem(cfg)[1].dense())
    return _cache[key]


def rel_max(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_matvec(cfg, dev):
    H, Ho, X0, _, _, _ = problem(cfg)
    with D.Context(H) as ctx:
        Y = ctx.matvec(torch.from_numpy(X0).to(dev))
        ref = O.matvec(Ho, X0.T).T
        assert rel_max(Y.cpu().numpy(), ref) <= 1e-11


def test_matvec_strided_and_ragged(dev):
    H, Ho, X0, _, _, _ = problem(problems()[1])
    Ns = 37
    with D.Context(H) as ctx:
        big = torch.full((Ns, Ho.N + 13), 7.0, dtype=torch.float64, device=dev)
        Xv = big[:, :Ho.N]
        Xv.copy_(torch.from_numpy(X0[:Ns]))
        out = torch.full_like(big, -3.0)
        Yv = out[:, :Ho.N]
        ctx.matvec(Xv, Yv)
        ref = O.matvec(Ho, X0[:Ns].T).T
        assert rel_max(Yv.cpu().numpy(), ref) <= 1e-11
        assert torch.all(out[:, Ho.N:] == -3.0)      # padding never written


@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_filter_f64(cfg, dev):
    H, Ho, X0, _, Ns, _ = problem(cfg)
    lam = spectrum(cfg)
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[min(Ns, Ho.N - 1)]
    with D.Context(H) as ctx:
        for m in sorted({1, 2, cfg.m}):
            Y = ctx.filter(torch.from_numpy(X0).to(dev), m, a, b, a0, prec="f64")
            ref = O.chebyshev_filter(Ho, X0.T, m, a, b, a0).T
            assert rel_max(Y.cpu().numpy(), ref) <= 1e-11, m


@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_bounds(cfg, dev):
    H, Ho, _, v0, _, _ = problem(cfg)
    with D.Context(H) as ctx:
        for k in (1, 4, 10):
            b, t = ctx.bounds(torch.from_numpy(v0).to(dev), k)
            bo, to, _, _ = O.lanczos_bounds(Ho, v0, k)
            assert abs(b - bo) <= 1e-10 * abs(bo)
            assert abs(t - to) <= 1e-10 * max(abs(to), abs(bo))


@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_rayleigh_ritz_occupations_density(cfg, dev):
    H, Ho, X0, _, Ns, Ne = problem(cfg)
    lam = spectrum(cfg)
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[min(Ns, Ho.N - 1)]
    Yt = O.chebyshev_filter(Ho, X0.T, cfg.m, a, b, a0)
    Yh, U, _ = O.cholesky_qr(Yt)
    kappa_S = np.linalg.cond(U) ** 2
    Xo, Do, _ = O.rayleigh_ritz(Ho, Yh)
    fo, muo = O.fermi_occupations(Do, Ne, cfg.kT)
    Po = O.packed_density(Ho, O.density_blocks(Ho, Xo, fo))
    scale = max(abs(a0), abs(b))
    with D.Context(H) as ctx:
        Y = torch.from_numpy(np.ascontiguousarray(Yt.T)).to(dev)
        ritz = ctx.rayleigh_ritz(Y)
        assert np.max(np.abs(ritz.cpu().numpy() - Do)) <= 1e-10 * scale
        Xg = Y.cpu().numpy()
        # Cholesky-QR loses orthogonality in proportion to cond(S) = cond(Y)^2
        assert np.max(np.abs(Xg @ Xg.T - np.eye(Ns))) <= 1e-12 * kappa_S + 1e-12
        f, mu = ctx.occupations(ritz, Ne, cfg.kT)
        assert np.max(np.abs(f.cpu().numpy() - fo)) <= 1e-9
        assert abs(mu.item() - muo) <= 1e-10 * scale
        P = ctx.density_blocks(Y, f)
        assert np.linalg.norm(P.cpu().numpy() - Po) <= 1e-9 * np.linalg.norm(Po)


@pytest.mark.parametrize("cfg", problems(), ids=lambda c: c.name)
def test_gram(cfg, dev):
    H, Ho, X0, _, Ns, _ = problem(cfg)
    with D.Context(H) as ctx:
        S = ctx.gram(torch.from_numpy(X0).to(dev)).cpu().numpy()
    Yt, _, So = None, None, O.cholesky_qr(X0.T)[2]
    assert np.array_equal(S, S.T)
    assert rel_max(S, So) <= 1e-12


def test_occupations_and_density_on_oracle_inputs(dev):
    H, Ho, X0, _, Ns, Ne = problem(problems()[2])
    rng = np.random.default_rng(3)
    lam = np.sort(rng.uniform(-1, 40, Ns))
    with D.Context(H) as ctx:
        for Ne_, kT in [(Ne, 0.01), (0.0, 0.01), (2.0 * Ns, 0.01), (Ne, 1e-4), (Ne, 2.0)]:
            f, mu = ctx.occupations(torch.from_numpy(lam).to(dev), Ne_, kT)
            fo, muo = O.fermi_occupations(lam, Ne_, kT)
            assert np.max(np.abs(f.cpu().numpy() - fo)) <= 1e-9, (Ne_, kT)
        f = rng.uniform(0, 1, Ns)
        P = ctx.density_blocks(torch.from_numpy(X0).to(dev), torch.from_numpy(f).to(dev))
        Po = O.packed_density(Ho, O.density_blocks(Ho, X0.T, f))
        assert rel_max(P.cpu().numpy(), Po) <= 1e-11


@pytest.mark.parametrize("cfg", problems()[:3], ids=lambda c: c.name)
def test_cycle_matches_oracle_cycle_by_cycle(cfg, dev):
    """Several cycles; each cycle's oracle run gets the GPU's bounds (a, b, a0)
    and the GPU's starting block, and the Ritz values and density blocks must
    agree. The Lanczos bound itself is compared in test_bounds."""
    H, Ho, X0, v0, Ns, Ne = problem(cfg)
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        prev = None
        for cyc in range(3):
            Xin = X.cpu().numpy().T.copy()
            out = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v, prev_ritz=prev)
            a, b, a0 = out["bounds"]
            ref = O.chefsi_cycle(Ho, Xin, cfg.m, Ne, cfg.kT, v0, bounds=(a, b, a0))
            bo, to, _, _ = O.lanczos_bounds(Ho, v0, 10)
            assert abs(b - bo) <= 1e-10 * abs(bo)
            scale = max(abs(a0), abs(b))
            ritz = out["ritz"].cpu().numpy()
            assert np.max(np.abs(ritz - ref["ritz"])) <= 1e-10 * scale, cyc
            Pr = O.packed_density(Ho, ref["P"])
            assert np.linalg.norm(out["P"].cpu().numpy() - Pr) <= 1e-9 * np.linalg.norm(Pr), cyc
            prev = ritz


def test_tiny_converges_to_dense_spectrum(dev):
    """20 cycles of the tiny 2x2x2 problem: the lowest N_s - 8 Ritz values match
    a dense eigensolve of H and 2 tr P equals the electron count."""
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, Ho, X0, v0, Ns, Ne = problem(cfg)
    lam = spectrum(cfg)
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        prev = None
        for _ in range(cfg.cycles):
            out = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v, prev_ritz=prev)
            prev = out["ritz"].cpu().numpy()
        g = 8
        scale = max(abs(lam[0]), abs(lam[-1]))
        assert np.max(np.abs(prev[:Ns - g] - lam[:Ns - g])) <= 1e-10 * scale
        tr = sum(float(torch.trace(p)) for p in ctx.unpack_density(out["P"]))
        assert abs(2 * tr - Ne) <= 1e-8 * Ne
        A = Ho.dense()
        Xn = X.cpu().numpy().T
        res = np.linalg.norm(A @ Xn[:, :Ns - g] - Xn[:, :Ns - g] * prev[None, :Ns - g], axis=0)
        assert np.max(res) <= 1e-9 * scale


def test_error_paths(dev):
    H, Ho, X0, v0, Ns, Ne = problem(problems()[0])
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        for a, b, a0 in [(1.0, 1.0, 0.0), (2.0, 1.0, 0.0), (1.0, 2.0, 1.5)]:
            with pytest.raises(D.DGChefsiError) as e:
                ctx.filter(X, 3, a, b, a0)
            assert e.value.status == "ERR_ARG"
        with pytest.raises(D.DGChefsiError):
            ctx.filter(X, 0, 1.0, 2.0, 0.0)
        with pytest.raises(D.DGChefsiError):
            ctx.filter(X, 3, 1.0, 2.0, 0.0, Y=X)            # aliasing
        with pytest.raises(D.DGChefsiError) as e:
            ctx.occupations(torch.zeros(4, dtype=torch.float64, device=dev), 9.0, 0.01)
        assert e.value.status == "ERR_ARG"
        Y = X.clone()
        Y[5] = 0.0                                          # rank-deficient block: S has a zero pivot
        with pytest.raises(D.DGChefsiError) as e:
            ctx.rayleigh_ritz(Y)
        assert e.value.status == "ERR_NOT_SPD"
        with pytest.raises(D.DGChefsiError):
            ctx.bounds(torch.zeros(Ho.N, dtype=torch.float64, device=dev))
        # the context still works after the errors
        out = ctx.matvec(X)
        assert rel_max(out.cpu().numpy(), O.matvec(Ho, X0.T).T) <= 1e-11


def test_bounded_wait_times_out_and_context_survives(dev):
    """Failure detection: a device wait that nothing satisfies gives up after
    its bound and reports a timeout; the context keeps working."""
    H, Ho, X0, _, _, _ = problem(problems()[0])
    with D.Context(H) as ctx:
        import time
        t0 = time.time()
        status, msg = ctx.selftest_wait(50_000_000)   # 50 ms
        assert status == "ERR_TIMEOUT" and "gave up" in msg
        assert time.time() - t0 < 5.0
        Y = ctx.matvec(torch.from_numpy(X0).to(dev))
        assert rel_max(Y.cpu().numpy(), O.matvec(Ho, X0.T).T) <= 1e-11
