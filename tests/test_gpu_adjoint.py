"""GPU adjoint of the band energy (dgchefsi_energy_grad, the autograd
Function) against the FP64 oracle's adjoint, through the C ABI.

Both sides are FP64 and run the same steps; the GPU recomputes the filter
from checkpoints. Tolerances: E to 1e-11 relative; dE/dH (per stored entry)
and dE/dX to 1e-8 of their largest entry (the Gram and projected matrices
carry cond(Y~)^2 rounding into Z = U^{-1} Q, as in the forward tests)."""
import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None
A = pytest.importorskip("paper_1606_03416_gb300.autograd") if torch.cuda.is_available() else None


def case(kind):
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
    a0, b, a = lam[0] - 0.3, lam[-1] + 0.3, lam[min(Ns + 3, len(lam) - 1)]
    return cfg, H, Ho, X0, Ns, Ne, (a, b, a0)


def rel(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("kind", ["small", "tiny", "bulk3"])
def test_energy_grad_matches_oracle(kind):
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case(kind)
    E_o, G_o, Xb_o = O.band_energy_grad(Ho, X0.T, cfg.m, a, b, a0, Ne, cfg.kT)
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        E, ritz, Hb, Xb = ctx.energy_grad(torch.from_numpy(X0).to(dev), cfg.m, a, b, a0, Ne, cfg.kT)
    assert abs(E - E_o) <= 1e-11 * abs(E_o)
    Gflat = np.concatenate([g.ravel() for g in G_o])
    assert rel(Hb.cpu().numpy(), Gflat) <= 1e-8
    assert rel(Xb.cpu().numpy(), Xb_o.T) <= 1e-8


def test_checkpoint_stride_does_not_change_result():
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("small")
    dev = torch.device("cuda:0")
    X = torch.from_numpy(X0).to(dev)
    with D.Context(H) as ctx:
        ref = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, stride=1)
        for s in (2, 0, cfg.m):
            out = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, stride=s)
            assert out[0] == pytest.approx(ref[0], rel=1e-14)
            assert torch.allclose(out[2], ref[2], rtol=0, atol=1e-12 * float(ref[2].abs().max()))
            assert torch.allclose(out[3], ref[3], rtol=0, atol=1e-12 * float(ref[3].abs().max()))


def test_autograd_function_and_central_differences():
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("small")
    dev = torch.device("cuda:0")
    vals = torch.from_numpy(H.values.copy()).to(dev).requires_grad_(True)
    X = torch.from_numpy(X0).to(dev).requires_grad_(True)
    mirror = A.mirror_index(H)
    with D.Context(H) as ctx:
        E = A.band_energy(vals, X, ctx, cfg.m, a, b, a0, Ne, cfg.kT)
        E.backward()
        tied = A.tie_symmetric(vals.grad, mirror).cpu().numpy()
        rng = np.random.default_rng(3)
        h = 1e-5
        base = H.values.copy()
        scale = np.max(np.abs(tied))
        for _ in range(8):
            i = int(rng.integers(0, base.size))
            ent = sorted({i, int(mirror[i])})
            fd = []
            for sgn in (1.0, -1.0):
                v = base.copy()
                v[ent] += sgn * h
                with torch.no_grad():
                    fd.append(float(A.band_energy(torch.from_numpy(v).to(dev), X.detach(), ctx, cfg.m, a, b, a0,
                                                  Ne, cfg.kT)))
            assert abs((fd[0] - fd[1]) / (2 * h) - tied[i]) <= 1e-6 * scale
        dX = torch.from_numpy(np.random.default_rng(4).standard_normal(X0.shape)).to(dev)
        with torch.no_grad():
            vv = torch.from_numpy(base).to(dev)
            Ep = float(A.band_energy(vv, X.detach() + 1e-6 * dX, ctx, cfg.m, a, b, a0, Ne, cfg.kT))
            Em = float(A.band_energy(vv, X.detach() - 1e-6 * dX, ctx, cfg.m, a, b, a0, Ne, cfg.kT))
        an = float((X.grad * dX).sum())
        assert abs((Ep - Em) / 2e-6 - an) <= 1e-6 * max(1.0, abs(an))


def test_converged_gradient_is_dense_eigen_formula():
    """3x3x3 elements, n_b = 16: converge with FP64 cycles, then the H gradient
    equals sum_i g_i v_i v_i^T over exact eigenpairs and dE/dX vanishes."""
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("bulk3")
    lam, V = np.linalg.eigh(Ho.dense())
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        Y = torch.empty_like(X)
        for _ in range(200):
            ctx.filter(X, cfg.m, a, b, a0, Y=Y)
            ctx.rayleigh_ritz(Y)
            X, Y = Y, X
        E, ritz, Hb, Xb = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT)
    f, _ = O.fermi_occupations(lam[:Ns], Ne, cfg.kT)
    g = O.energy_weights(lam[:Ns], f, cfg.kT)
    ref = np.concatenate([r.ravel() for r in O.block_outer(Ho, V[:, :Ns], V[:, :Ns], g)])
    assert rel(Hb.cpu().numpy(), ref) <= 1e-8
    assert float(Xb.norm()) <= 1e-8 * float(X.norm())


# ---- tensor-core forms: filter, checkpoints and backward recurrence on the
# tcgen05 step kernel with FP32 iterates; Rayleigh-Ritz and its adjoint FP64.
# Each filter step rounds its operands with relative error u_op (see
# test_gpu_tc), so the iterates carry about m * u_op, and Cholesky-QR turns a
# relative perturbation of Y_m into one of the orthonormal basis (hence of E,
# the weights and Z) at most cond(Y_m) times larger. Tolerance on E and on the
# largest gradient entries: 2 m u_op cond(Y_m).
U_OP = {"tf32": 2.0 ** -9, "bf16x3": 2.0 ** -16}


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
@pytest.mark.parametrize("kind", ["small", "tiny", "bulk3"])
def test_tensor_core_energy_grad_matches_oracle(kind, prec):
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case(kind)
    E_o, G_o, Xb_o = O.band_energy_grad(Ho, X0.T, cfg.m, a, b, a0, Ne, cfg.kT)
    kappa = np.linalg.cond(O.chebyshev_filter(Ho, X0.T, cfg.m, a, b, a0))
    tol = 2 * cfg.m * U_OP[prec] * kappa
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        E, ritz, Hb, Xb = ctx.energy_grad(torch.from_numpy(X0).to(dev), cfg.m, a, b, a0, Ne, cfg.kT, prec=prec)
    Gflat = np.concatenate([g.ravel() for g in G_o])
    eE, eH, eX = abs(E - E_o) / abs(E_o), rel(Hb.cpu().numpy(), Gflat), rel(Xb.cpu().numpy(), Xb_o.T)
    print(f"TC_GRAD {kind} {prec} cond={kappa:.2e} E={eE:.2e} H={eH:.2e} X={eX:.2e} tol={tol:.2e}")
    assert np.isfinite(Hb.cpu().numpy()).all() and np.isfinite(Xb.cpu().numpy()).all()
    assert eE <= tol and eH <= tol and eX <= tol


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_tensor_core_grad_independent_of_checkpoint_stride(prec):
    """Recomputed segments reproduce the forward iterates bit for bit (same
    kernel, same inputs, operand copies rebuilt by the same rounding), so the
    gradient does not depend on the checkpoint stride at all."""
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("tiny")
    dev = torch.device("cuda:0")
    X = torch.from_numpy(X0).to(dev)
    with D.Context(H) as ctx:
        ref = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, stride=1, prec=prec)
        # the energy-only call (no checkpoints) runs the same filter kernel
        assert ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, grad=False, prec=prec)[0] == ref[0]
        for s in (2, 3, 0, cfg.m):
            out = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, stride=s, prec=prec)
            assert out[0] == ref[0]
            assert torch.equal(out[2], ref[2]) and torch.equal(out[3], ref[3]), s


def test_tensor_core_autograd_matches_fp64_gradient():
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("bulk3")
    kappa = np.linalg.cond(O.chebyshev_filter(Ho, X0.T, cfg.m, a, b, a0))
    dev = torch.device("cuda:0")
    grads = {}
    with D.Context(H) as ctx:
        for prec in ("f64", "bf16x3"):
            vals = torch.from_numpy(H.values.copy()).to(dev).requires_grad_(True)
            X = torch.from_numpy(X0).to(dev).requires_grad_(True)
            E = A.band_energy(vals, X, ctx, cfg.m, a, b, a0, Ne, cfg.kT, prec=prec)
            E.backward()
            grads[prec] = (float(E), vals.grad.cpu().numpy(), X.grad.cpu().numpy())
    tol = 2 * cfg.m * U_OP["bf16x3"] * kappa
    assert abs(grads["bf16x3"][0] - grads["f64"][0]) <= tol * abs(grads["f64"][0])
    assert rel(grads["bf16x3"][1], grads["f64"][1]) <= tol
    assert rel(grads["bf16x3"][2], grads["f64"][2]) <= tol


def test_tensor_core_converged_gradient_is_dense_eigen_formula():
    """The FP32-iterate (BF16x3) gradient at the converged 3x3x3 n_b = 16 state
    against sum_i g_i v_i v_i^T over exact eigenpairs, within the tensor-core
    tolerance 2 m u_op cond(Y_m) of the other tests; dE/dX stays at that level."""
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("bulk3")
    lam, V = np.linalg.eigh(Ho.dense())
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        Y = torch.empty_like(X)
        for _ in range(200):
            ctx.filter(X, cfg.m, a, b, a0, Y=Y)
            ctx.rayleigh_ritz(Y)
            X, Y = Y, X
        E, ritz, Hb, Xb = ctx.energy_grad(X, cfg.m, a, b, a0, Ne, cfg.kT, prec="bf16x3")
        Xc = X.cpu().numpy()
    kappa = np.linalg.cond(O.chebyshev_filter(Ho, Xc.T, cfg.m, a, b, a0))
    tol = 2 * cfg.m * U_OP["bf16x3"] * kappa
    f, _ = O.fermi_occupations(lam[:Ns], Ne, cfg.kT)
    g = O.energy_weights(lam[:Ns], f, cfg.kT)
    ref = np.concatenate([r.ravel() for r in O.block_outer(Ho, V[:, :Ns], V[:, :Ns], g)])
    err = rel(Hb.cpu().numpy(), ref)
    xb = float(Xb.norm()) / float(X.norm())
    print(f"TC_CONVERGED cond={kappa:.2e} H={err:.2e} Xbar={xb:.2e} tol={tol:.2e}")
    assert err <= tol and xb <= tol


@pytest.mark.parametrize("prec", ["f64", "bf16x3"])
@pytest.mark.parametrize("m", [1, 2])
def test_energy_grad_lowest_degrees(m, prec):
    """Degrees 1 and 2: one segment, no recomputed iterates (m = 1: a single
    checkpoint; m = 2: the pair), for both the FP64 and the tensor-core
    gradient, against the oracle adjoint."""
    cfg, H, Ho, X0, Ns, Ne, (a, b, a0) = case("small")
    E_o, G_o, Xb_o = O.band_energy_grad(Ho, X0.T, m, a, b, a0, Ne, cfg.kT)
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        E, _, Hb, Xb = ctx.energy_grad(torch.from_numpy(X0).to(dev), m, a, b, a0, Ne, cfg.kT, prec=prec)
    Gflat = np.concatenate([g.ravel() for g in G_o])
    if prec == "f64":
        tol = 1e-8
    else:
        tol = 2 * m * U_OP[prec] * np.linalg.cond(O.chebyshev_filter(Ho, X0.T, m, a, b, a0))
    assert abs(E - E_o) <= max(tol, 1e-11) * abs(E_o)
    assert rel(Hb.cpu().numpy(), Gflat) <= tol
    assert rel(Xb.cpu().numpy(), Xb_o.T) <= tol
