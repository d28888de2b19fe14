"""Plain FP64 CPU oracle for one CheFSI cycle on a block-sparse DG Hamiltonian.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. It shares no code with
the CUDA library (no kernels, headers, helpers or tables); both sides are fed
the same arrays from the seeded input generator and nothing else.

Orientation follows the paper: a block of vectors X is N x N_s with one state
per column, and x_K (rows off_K .. off_K + J_K) is the part of X on element K.
Everything is float64, NumPy/SciPy, written for clarity, not speed.

Sections of arXiv:1606.03416 followed here:
  * Sec. II.B, Eqs. eigvalue_prob / HDG_sub_blocks  -> the block-sparse H
  * Sec. III.A, Algorithm 1 (CheFSI cycle), steps 1-5
  * Sec. III.B.1, Eqs. matvec_1 .. matvec_3          -> ``matvec``
  * Sec. III.B.2 (Cholesky-QR, projection, rotation) -> ``cholesky_qr``,
    ``rayleigh_ritz``; the dense eigensolve of the projected H alone ->
    ``subspace_eigh``; the Cholesky factor and its inverse alone ->
    ``cholesky_inverse``
  * Sec. II.C, Eqs. densitymatrix / electron_density_from_DM, and the Fermi-Dirac
    occupations of Eq. KS_DG_Energy -> ``fermi_occupations``, ``density_blocks``

Readings where the paper is silent (each is also listed in the design notes):
  * Filter (Alg. 1 step 2): the *scaled* three-term Chebyshev recurrence of the
    CheFSI literature the paper cites, with [a, b] mapped to [-1, 1] and the
    result normalised by C_m at a0 (the lower end of the wanted spectrum).
    Unscaled p_m(H) X differs by the scalar C_m((a0-c)/e) only.
  * Bounds (Alg. 1 step 1): k-step Lanczos with full re-orthogonalisation from
    a given start vector; upper bound = max eig(T_k) + |beta_k|. Lower filter
    bound a = largest previous Ritz value, a0 = smallest; first cycle:
    a0 = min eig(T_k), a = a0 + (b - a0) * N_s / N.
  * Cholesky-QR fails loudly (``np.linalg.LinAlgError``) if S is not SPD.
  * Occupations: spin factor 2, so sum_i 2 f_i = N_e; mu by bisection on
    [lambda_1 - 50 kT, lambda_Ns + 50 kT] until |2 sum f - N_e| <= 1e-13 N_e
    or 200 halvings.

Parity unpinned: ``first_cycle_bounds`` (a heuristic the paper does not state;
the bounds change only the convergence rate, not the fixed point, and parity
tests pass the same bounds to both sides) and the accuracy floor of the
mixed-precision filter (measured, not a property of this module).

Parity pins (tests/test_oracle_pins.py) check every function here against
results the mathematics fixes independently of this code: brute-force dense
products, the closed form V C_m(Lambda) V^T X of the filter, dense eigh of H,
QR uniqueness, exact spectra of diagonal matrices, and trace / symmetry
identities. The precision forms' rounded filter (``chebyshev_filter_rounded``)
is pinned in tests/test_oracle_rounded.py: its BF16 rounding against
PyTorch's conversion, its TF32 cut against the closed form, exactness on
operands that need no rounding, and its distance from the FP64 filter.
``lowest_eigenvalues`` is a library eigensolve of the assembled matrix (the
definition of the exact spectrum).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class DGHamiltonian:
    """Block-sparse symmetric H (Eq. HDG_sub_blocks): H_{K;K'} nonzero only for
    neighbouring elements K' in N(K), each block dense J_K x J_K'."""

    def __init__(self, nb, row_ptr, col, blk_off, values):
        self.nb = np.asarray(nb, dtype=np.int64)
        self.row_ptr = np.asarray(row_ptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.blk_off = np.asarray(blk_off, dtype=np.int64)
        self.values = np.asarray(values, dtype=np.float64)
        self.M = int(self.nb.shape[0])
        self.off = np.zeros(self.M + 1, dtype=np.int64)
        self.off[1:] = np.cumsum(self.nb)
        self.N = int(self.off[-1])

    @classmethod
    def from_blocksparse(cls, bs):
        return cls(bs.nb, bs.row_ptr, bs.col, bs.blk_off, bs.values)

    def rows(self, K):
        return slice(int(self.off[K]), int(self.off[K + 1]))

    def neighbours(self, K):
        """Pairs (K', H_{K;K'}) over K' in N(K) (including K itself)."""
        for e in range(self.row_ptr[K], self.row_ptr[K + 1]):
            Kp = int(self.col[e])
            nK, nKp = int(self.nb[K]), int(self.nb[Kp])
            start = int(self.blk_off[e])
            yield Kp, self.values[start:start + nK * nKp].reshape(nK, nKp)

    def dense(self):
        """Dense N x N matrix assembled entry by entry from the blocks."""
        A = np.zeros((self.N, self.N))
        for K in range(self.M):
            for Kp, blk in self.neighbours(K):
                A[self.rows(K), self.rows(Kp)] = blk
        return A


def matvec(H: DGHamiltonian, X: np.ndarray) -> np.ndarray:
    """Y = H X for an N x k block, element by element (Eq. matvec_3):
    y_K = sum over K' in N(K) of H_{K;K'} x_{K'}, a sum of dense GEMMs."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.zeros_like(X)
    for K in range(H.M):
        acc = np.zeros((int(H.nb[K]),) + X.shape[1:])
        for Kp, blk in H.neighbours(K):
            acc += blk @ X[H.rows(Kp)]
        Y[H.rows(K)] = acc
    return Y


def filter_coefficients(m: int, a: float, b: float, a0: float):
    """Scalars of the scaled recurrence for Alg. 1 step 2.

    e = (b - a)/2 and c = (b + a)/2 map [a, b] to [-1, 1]; sigma_1 = e/(a0 - c)
    is 1/C_1(tau0) with tau0 = (a0 - c)/e, and sigma_{k+1} = 1/(2/sigma_1 - sigma_k)
    is C_k(tau0)/C_{k+1}(tau0) by the Chebyshev three-term rule.
    Returns (c, e, sigmas) with sigmas[k] = sigma_k for k = 1..m (index 0 unused).
    """
    if not (a0 < a < b) or m < 1:
        raise ValueError("need a0 < a < b and m >= 1")
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    sig = [0.0] * (m + 1)
    sig[1] = e / (a0 - c)
    for k in range(1, m):
        sig[k + 1] = 1.0 / (2.0 / sig[1] - sig[k])
    return c, e, sig


def chebyshev_filter(H: DGHamiltonian, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Y~ = p_m(H) X with [a, b] mapped to [-1, 1] (Alg. 1 step 2).

    p_m(t) = C_m((t - c)/e) / C_m((a0 - c)/e), evaluated by the three-term
    recurrence Y_{k+1} = (2 sigma_{k+1}/e)(H - cI) Y_k - sigma_k sigma_{k+1} Y_{k-1},
    starting from Y_0 = X and Y_1 = (sigma_1/e)(H - cI) X.
    """
    c, e, sig = filter_coefficients(m, a, b, a0)
    Y_prev = np.array(X, dtype=np.float64, copy=True)
    Y = (sig[1] / e) * (matvec(H, Y_prev) - c * Y_prev)
    for k in range(1, m):
        Y_next = (2.0 * sig[k + 1] / e) * (matvec(H, Y) - c * Y) - (sig[k] * sig[k + 1]) * Y_prev
        Y_prev, Y = Y, Y_next
    return Y


# --------------------------------------------------------------------------
# Precision forms of the filter: the same recurrence with the operand
# roundings of the tensor-core forms (filter products in TF32 or BF16 with
# FP32 accumulation, FP32 iterates). Used to compare those forms with the
# rounding they are meant to have, which is far tighter than comparing them
# with the FP64 filter. Each product is evaluated exactly (FP64 here); only
# the order of the FP32 accumulation is not emulated.
# --------------------------------------------------------------------------


def round_fp32(x) -> np.ndarray:
    """Round to the nearest FP32 value (returned as float64)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_bf16(x) -> np.ndarray:
    """Round FP32 values to BF16 (8 significant bits), nearest, ties to even:
    add half of the dropped 16 bits (minus one unless the kept last bit is
    odd) and clear them. Finite inputs only."""
    b = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def truncate_tf32(x) -> np.ndarray:
    """FP32 values cut to TF32 (11 significant bits) by dropping the low 13
    mantissa bits, the way the TF32 tensor-core product reads FP32 operands."""
    b = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return b.view(np.float32).astype(np.float64)


def _with_values(H: DGHamiltonian, values) -> DGHamiltonian:
    return DGHamiltonian(H.nb, H.row_ptr, H.col, H.blk_off, values)


def shifted_values(H: DGHamiltonian, c: float) -> np.ndarray:
    """Values of H - cI, block by block (the shift on the diagonal blocks' diagonals)."""
    v = H.values.copy()
    for K in range(H.M):
        for e in range(H.row_ptr[K], H.row_ptr[K + 1]):
            if int(H.col[e]) == K:
                n = int(H.nb[K])
                idx = int(H.blk_off[e]) + np.arange(n) * (n + 1)
                v[idx] -= c
    return v


def chebyshev_filter_rounded(H: DGHamiltonian, X: np.ndarray, m: int, a: float, b: float, a0: float,
                             fmt: str) -> np.ndarray:
    """Alg. 1 step 2 with the operand roundings of a tensor-core form.

    The operator is H - cI rounded to FP32, the iterates are FP32, the
    recurrence scalars FP32, and each product (H - cI) Y_k uses operands
    rounded to the form's type:
      "bf16"    bf16(H - cI) bf16(Y_k)
      "bf16x3"  hi = bf16(v), lo = bf16(v - hi) for both operands;
                hi*hi + lo(H)*hi(Y) + hi(H)*lo(Y)
      "tf32"    tf32(H - cI) tf32(Y_k), TF32 cut from FP32 as above
    then Y_{k+1} = fp32(alpha_k fp32(P) - fp32(beta_k Y_{k-1})) with the
    scalars of the scaled recurrence (alpha_0 = s_1/e, beta_0 = 0)."""
    c, alpha, beta = _recurrence_coefficients(m, a, b, a0)
    Hs = round_fp32(shifted_values(H, c))
    if fmt == "tf32":
        ops = [(truncate_tf32(Hs), "t")]
    elif fmt in ("bf16", "bf16x3"):
        hi = round_bf16(Hs)
        ops = [(hi, "hi")]
        if fmt == "bf16x3":
            ops += [(round_bf16(Hs - hi), "hi"), (hi, "lo")]
    else:
        raise ValueError(f"unknown format {fmt!r}")
    ops = [(_with_values(H, v), which) for v, which in ops]

    def parts(Y):
        if fmt == "tf32":
            return {"t": truncate_tf32(Y)}
        hi = round_bf16(Y)
        return {"hi": hi, "lo": round_bf16(Y - hi)}

    Y_prev = None
    Y = round_fp32(X)
    for k in range(m):
        p = parts(Y)
        P = sum(matvec(Hop, p[which]) for Hop, which in ops)
        al, be = float(np.float32(alpha[k])), float(np.float32(beta[k]))
        prev = round_fp32(be * Y_prev) if Y_prev is not None else 0.0
        Y_prev, Y = Y, round_fp32(al * round_fp32(P) - prev)
    return Y


def lanczos_bounds(H: DGHamiltonian, v0: np.ndarray, k: int = 10):
    """Upper spectral bound by k Lanczos steps (Alg. 1 step 1).

    Full re-orthogonalisation (one classical Gram-Schmidt pass against all
    previous Lanczos vectors after the three-term step). Returns
    (b_upper, theta_min, alphas, betas): b_upper = max eig(T_k) + |beta_k| with
    beta_k the norm of the last residual, theta_min = min eig(T_k). Stops early
    (k reduced) if a residual vanishes (an invariant subspace was found).
    """
    k = int(min(k, H.N))
    v = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    V = [v]
    alphas, betas = [], []
    beta_prev = 0.0
    v_prev = np.zeros_like(v)
    beta_last = 0.0
    for j in range(k):
        w = matvec(H, V[j][:, None])[:, 0] - beta_prev * v_prev
        alpha = float(V[j] @ w)
        w = w - alpha * V[j]
        Vm = np.stack(V, axis=1)
        w = w - Vm @ (Vm.T @ w)
        alphas.append(alpha)
        beta = float(np.linalg.norm(w))
        beta_last = beta
        if j == k - 1 or beta == 0.0:
            break
        betas.append(beta)
        v_prev = V[j]
        V.append(w / beta)
        beta_prev = beta
    T_eigs = sla.eigh_tridiagonal(np.array(alphas), np.array(betas), eigvals_only=True)
    return float(T_eigs[-1] + abs(beta_last)), float(T_eigs[0]), alphas, betas


def first_cycle_bounds(b_upper: float, theta_min: float, Ns: int, N: int):
    """(a, a0) for the first cycle, before any Ritz values exist (parity
    unpinned: a reading of the paper's silence, see the module header)."""
    a0 = theta_min
    a = a0 + (b_upper - a0) * Ns / N
    return a, a0


def cholesky_qr(Y: np.ndarray):
    """Alg. 1 step 3: S = Y^T Y, S = U^T U (U upper, positive diagonal), and
    Y_hat with Y_hat U = Y. Returns (Y_hat, U, S). Raises LinAlgError if S is
    not positive definite."""
    S = Y.T @ Y
    U = np.linalg.cholesky(S).T  # numpy gives lower L with S = L L^T
    Y_hat = sla.solve_triangular(U, Y.T, trans="T", lower=False).T
    return Y_hat, U, S


def cholesky_inverse(S: np.ndarray):
    """The factor of Alg. 1 step 3 on its own: S = L L^T (L lower, positive
    diagonal; L = U^T for the paper's S = U^T U) from the lower triangle of S
    (the upper one is not read), and L^{-1}, the factor Y_hat^T = L^{-1} Y^T
    applies. Raises ``np.linalg.LinAlgError`` if S is not positive definite.
    The definition: a library Cholesky factorisation and a triangular solve
    against the identity."""
    Lo = np.tril(np.asarray(S, dtype=np.float64))
    L = np.linalg.cholesky(Lo + np.tril(Lo, -1).T)
    Li = sla.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    return L, Li


def rayleigh_ritz(H: DGHamiltonian, Y_hat: np.ndarray):
    """Alg. 1 steps 4-5: H_hat = Y_hat^T (H Y_hat), symmetrised; H_hat Q = Q D
    with D ascending; X_new = Y_hat Q. Returns (X_new, D, H X_new)."""
    W = matvec(H, Y_hat)
    Hh = Y_hat.T @ W
    Hh = 0.5 * (Hh + Hh.T)
    D, Q = np.linalg.eigh(Hh)
    return Y_hat @ Q, D, W @ Q


def subspace_eigh(A: np.ndarray):
    """Alg. 1 step 4 on its own: the eigen-decomposition of the symmetric
    matrix whose lower triangle is held in A (the upper one is not read).
    Returns (w, V): w ascending, row i of V the unit eigenvector of w[i] (the
    library's layout). The definition itself: a dense FP64 symmetric eigensolve."""
    L = np.tril(np.asarray(A, dtype=np.float64))
    D, Q = np.linalg.eigh(L + np.tril(L, -1).T, UPLO="L")
    return D, np.ascontiguousarray(Q.T)


def _fermi(x: np.ndarray) -> np.ndarray:
    """1/(1 + exp(x)) without overflow."""
    out = np.empty_like(x)
    pos = x > 0
    ex = np.exp(-x[pos])
    out[pos] = ex / (1.0 + ex)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def fermi_occupations(ritz: np.ndarray, Ne: float, kT: float):
    """Fermi-Dirac occupations f_i = 1/(1 + exp((lambda_i - mu)/kT)) with mu
    fixed by the electron count 2 sum_i f_i = N_e (spin factor 2, Eq.
    KS_DG_Energy). mu by bisection. Returns (f, mu)."""
    lam = np.asarray(ritz, dtype=np.float64)
    Ns = lam.shape[0]
    if kT <= 0 or Ne < 0 or Ne > 2 * Ns:
        raise ValueError("need kT > 0 and 0 <= Ne <= 2 Ns")
    lo = float(lam.min()) - 50.0 * kT
    hi = float(lam.max()) + 50.0 * kT
    tol = 1e-13 * Ne
    mu = 0.5 * (lo + hi)
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        count = 2.0 * _fermi((lam - mu) / kT).sum()
        if abs(count - Ne) <= tol:
            break
        if count < Ne:
            lo = mu
        else:
            hi = mu
    return _fermi((lam - mu) / kT), mu


def density_blocks(H: DGHamiltonian, X: np.ndarray, f: np.ndarray):
    """Diagonal blocks of the density matrix (Eq. densitymatrix with K' = K):
    P_KK = sum_i f_i x_{i;K} x_{i;K}^T, one J_K x J_K block per element."""
    return [X[H.rows(K)] @ np.diag(f) @ X[H.rows(K)].T for K in range(H.M)]


def chefsi_cycle(H: DGHamiltonian, X: np.ndarray, m: int, Ne: float, kT: float, v0: np.ndarray,
                 prev_ritz=None, k_lanczos: int = 10, bounds=None):
    """One CheFSI cycle (Alg. 1) followed by occupations and density blocks.

    ``bounds`` = (a, b, a0) overrides step 1 (used when both sides must see
    identical bounds). Returns a dict with the filter bounds, the new block,
    Ritz values, occupations, mu and the diagonal density blocks."""
    Ns = X.shape[1]
    if bounds is None:
        b, theta_min, _, _ = lanczos_bounds(H, v0, k_lanczos)
        if prev_ritz is None:
            a, a0 = first_cycle_bounds(b, theta_min, Ns, H.N)
        else:
            a, a0 = float(np.max(prev_ritz)), float(np.min(prev_ritz))
    else:
        a, b, a0 = bounds
    Yt = chebyshev_filter(H, X, m, a, b, a0)
    Yh, _, _ = cholesky_qr(Yt)
    X_new, D, HX = rayleigh_ritz(H, Yh)
    f, mu = fermi_occupations(D, Ne, kT)
    P = density_blocks(H, X_new, f)
    return dict(a=a, b=b, a0=a0, X=X_new, ritz=D, HX=HX, f=f, mu=mu, P=P)


def lowest_eigenvalues(H: DGHamiltonian, n: int) -> np.ndarray:
    """The n smallest eigenvalues of H, ascending, from a dense FP64 symmetric
    eigensolve (LAPACK through SciPy) of the assembled matrix: the exact values
    the Ritz values of Alg. 1 converge to (Sec. III.A). A reference for
    convergence, not a step of the cycle."""
    A = H.dense()
    return sla.eigh(A, eigvals_only=True, subset_by_index=[0, n - 1], overwrite_a=True, check_finite=False,
                    driver="evr")


def chebyshev_value(m: int, t):
    """C_m(t) from its trigonometric / hyperbolic closed form (used by the pins)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ta = np.abs(t[~inside])
    out[~inside] = np.sign(t[~inside]) ** m * np.cosh(m * np.arccosh(ta))
    return out


def packed_density(H: DGHamiltonian, blocks) -> np.ndarray:
    """Concatenate P_KK row-major in element order (the library's packed form)."""
    return np.concatenate([np.asarray(b).ravel() for b in blocks]) if blocks else np.zeros(0)



# --------------------------------------------------------------------------
# Band energy of one cycle and its adjoint (differentiation of the cycle).
#
# E(H, X) = sum_i f_i lambda_i for one cycle (filter -> Cholesky-QR ->
# Rayleigh-Ritz -> occupations) with the filter bounds (a, b, a0), N_e and kT
# held fixed. The paper does not differentiate the cycle; the adjoint below is
# derived from the steps above:
#   * occupations: f'_i = -f_i (1 - f_i)/kT and mu(lambda) from sum f = N_e/2
#     give g_i = dE/dlambda_i = f_i + lambda_i f'_i - f'_i (sum_j lambda_j f'_j)/(sum_j f'_j);
#   * Rayleigh-Ritz on span(Y~): with Z = U^{-1} Q (so X_new = Y~ Z) and
#     R = H X_new - X_new Lambda, dlambda_i = x_i^T dH x_i + 2 r_i^T dY~ z_i, hence
#     dE/dH (each stored entry independent) gets sum_i g_i x_i x_i^T and
#     Y~bar = 2 R G Z^T;
#   * filter: reverse the recurrence Y_{k+1} = alpha_k (H - cI) Y_k - beta_k Y_{k-1}
#     (alpha_0 = s_1/e, beta_0 = 0; alpha_k = 2 s_{k+1}/e, beta_k = s_k s_{k+1}):
#     W_m = Y~bar, dE/dH += alpha_k W_{k+1} Y_k^T, W_k = alpha_k (H - cI) W_{k+1} - beta_{k+1} W_{k+2},
#     and X bar = W_0.
# Gradients w.r.t. H are returned per stored block as if every stored entry
# were independent; a symmetric perturbation of H_{KK'}[j, j'] = H_{K'K}[j', j]
# changes E by G_{KK'}[j, j'] + G_{K'K}[j', j] (see ``tied_gradient``).
# --------------------------------------------------------------------------


def _recurrence_coefficients(m, a, b, a0):
    c, e, sig = filter_coefficients(m, a, b, a0)
    alpha = [sig[1] / e] + [2.0 * sig[k + 1] / e for k in range(1, m)]
    beta = [0.0] + [sig[k] * sig[k + 1] for k in range(1, m)]
    return c, alpha, beta


def band_energy(H: DGHamiltonian, X, m, a, b, a0, Ne, kT):
    """E = sum_i f_i lambda_i after one cycle with fixed bounds."""
    Yt = chebyshev_filter(H, X, m, a, b, a0)
    Yh, _, _ = cholesky_qr(Yt)
    _, D, _ = rayleigh_ritz(H, Yh)
    f, _ = fermi_occupations(D, Ne, kT)
    return float(np.sum(f * D))


def energy_weights(lam, f, kT):
    """g_i = dE/dlambda_i with the Fermi level following the eigenvalues."""
    fp = -f * (1.0 - f) / kT
    s = fp.sum()
    shift = (lam * fp).sum() / s if s != 0.0 else 0.0
    return f + lam * fp - fp * shift


def block_outer(H: DGHamiltonian, A, B, w=None):
    """Per stored block (K, K'): sum_i w_i A[K rows, i] B[K' rows, i]^T."""
    Aw = A if w is None else A * w[None, :]
    out = []
    for K in range(H.M):
        for Kp, _ in H.neighbours(K):
            out.append(Aw[H.rows(K)] @ B[H.rows(Kp)].T)
    return out


def band_energy_grad(H: DGHamiltonian, X, m, a, b, a0, Ne, kT):
    """(E, G, Xbar): the band energy, dE/dH per stored block (list in block-CSR
    order, each stored entry independent) and dE/dX (N x N_s)."""
    c, alpha, beta = _recurrence_coefficients(m, a, b, a0)
    Ys = [np.array(X, dtype=np.float64, copy=True)]
    for k in range(m):
        nxt = alpha[k] * (matvec(H, Ys[k]) - c * Ys[k])
        if k > 0:
            nxt -= beta[k] * Ys[k - 1]
        Ys.append(nxt)
    Yt = Ys[m]
    Yh, U, _ = cholesky_qr(Yt)
    Wh = matvec(H, Yh)
    Hh = Yh.T @ Wh
    lam, Q = np.linalg.eigh(0.5 * (Hh + Hh.T))
    X_new, HX = Yh @ Q, Wh @ Q
    f, _ = fermi_occupations(lam, Ne, kT)
    E = float(np.sum(f * lam))
    g = energy_weights(lam, f, kT)
    # Rayleigh-Ritz part
    G = block_outer(H, X_new, X_new, g)
    Z = sla.solve_triangular(U, Q, lower=False)   # X_new = Y~ Z
    R = HX - X_new * lam[None, :]
    W_next = 2.0 * (R * g[None, :]) @ Z.T         # Y~bar
    W_next2 = np.zeros_like(W_next)
    # filter part: reverse recurrence
    for k in range(m - 1, -1, -1):
        for idx, blk in enumerate(block_outer(H, W_next, Ys[k])):
            G[idx] = G[idx] + alpha[k] * blk
        Wk = alpha[k] * (matvec(H, W_next) - c * W_next)
        if k + 1 < m:
            Wk -= beta[k + 1] * W_next2
        W_next2, W_next = W_next, Wk
    return E, G, W_next


def tied_gradient(H: DGHamiltonian, G):
    """dE for symmetric perturbations: for each stored block (K, K') the matrix
    T with T[j, j'] = dE/d(H_KK'[j, j'] and H_K'K[j', j] together) =
    G_KK'[j, j'] + G_K'K[j', j] (for K = K' the diagonal counts once)."""
    index = {}
    e = 0
    for K in range(H.M):
        for Kp, _ in H.neighbours(K):
            index[(K, Kp)] = e
            e += 1
    out = []
    for K in range(H.M):
        for Kp, _ in H.neighbours(K):
            t = G[index[(K, Kp)]] + G[index[(Kp, K)]].T
            if K == Kp:
                t = t - np.diag(np.diag(G[index[(K, K)]]))
            out.append(t)
    return out


# --------------------------------------------------------------------------
# Beyond one cycle.
#  * Re-alignment of the coefficients to the next SCF step's basis
#    (Sec. III.B.3, Eqs. basis_rotation_1-3).
#  * Density-matrix blocks on all of H's pattern (Eq. densitymatrix for
#    neighbouring K, K'; the paper computes the diagonal ones, Sec. II.C).
#  * CholeskyQR2 and shifted CholeskyQR3, alternatives to the Cholesky-QR of
#    Alg. 1 step 3, whose loss of stability on ill-conditioned filtered blocks
#    the paper mentions (Sec. III.B.2). Readings: CholeskyQR2 is Cholesky-QR
#    applied twice (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014); the shifted
#    form first factors Y^T Y + s I with s = 11 (n N_s + N_s (N_s + 1)) u ||Y||_F^2
#    (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020, with the Frobenius
#    norm in place of the 2-norm, an upper bound they allow), u = 2^-53, then
#    applies CholeskyQR2. All three give the same Q (the thin-QR factor with
#    positive R diagonal) in exact arithmetic.
# --------------------------------------------------------------------------


def realign(V_old, V_new, X: np.ndarray) -> np.ndarray:
    """Eq. basis_rotation_3: X_K^{(i+1)} = (V_K^{i+1})^T V_K^{i} X_K^{(i)} on every
    element K. V_old[K] is R_K x J_K^{i} (element K's old basis functions
    sampled on its R_K grid points), V_new[K] is R_K x J_K^{i+1}; X is
    (sum_K J_K^{i}) x N_s with element K's rows consecutive. Elements have
    disjoint supports, so the global product of Eq. basis_rotation_1 splits
    into these per-element products (Eq. basis_rotation_2)."""
    rows, out, o = [], [], 0
    for K in range(len(V_old)):
        n = V_old[K].shape[1]
        rows.append((o, o + n))
        o += n
    if o != X.shape[0]:
        raise ValueError("X rows do not match the old basis sizes")
    for K, (r0, r1) in enumerate(rows):
        out.append((V_new[K].T @ V_old[K]) @ X[r0:r1])
    return np.vstack(out)


def density_pattern_blocks(H: DGHamiltonian, X: np.ndarray, f: np.ndarray):
    """Eq. densitymatrix on every stored block of H: P_KK' = sum_i f_i
    x_{i;K} x_{i;K'}^T for K' in N(K), in block-CSR order."""
    out = []
    for K in range(H.M):
        for Kp, _ in H.neighbours(K):
            out.append(X[H.rows(K)] @ np.diag(f) @ X[H.rows(Kp)].T)
    return out


def cholesky_qr2(Y: np.ndarray):
    """CholeskyQR2: Y = Q1 U1 by Cholesky-QR, then Q1 = Q U2. Returns (Q, U)
    with U = U2 U1 upper triangular, Y = Q U."""
    Q1, U1, _ = cholesky_qr(Y)
    Q, U2, _ = cholesky_qr(Q1)
    return Q, U2 @ U1


def shifted_cholesky_qr3(Y: np.ndarray):
    """Shifted CholeskyQR3: U1 = chol(Y^T Y + s I), Q1 = Y U1^{-1}, then
    CholeskyQR2 of Q1. Returns (Q, U) with Y = Q U."""
    n, ns = Y.shape
    S = Y.T @ Y
    s = 11.0 * (n * ns + ns * (ns + 1)) * 2.0 ** -53 * float(np.sum(Y * Y))
    U1 = np.linalg.cholesky(S + s * np.eye(ns)).T
    Q1 = sla.solve_triangular(U1, Y.T, trans="T", lower=False).T
    Q, U23 = cholesky_qr2(Q1)
    return Q, U23 @ U1
