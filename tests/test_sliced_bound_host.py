"""Host checks of the arithmetic behind the FP64 products from BF16 slices
(error-free splitting, Ozaki et al. 2012), on a NumPy restatement of the
digits: no GPU, no library call.

* digits: |q_0| <= 64, |q_i| <= 32, exact in BF16 (8 significant bits), and
  |v - sum_i q_i 2^{-6(i+1)}| <= 2^{-6s}/2 for every double incl. subnormals;
  so a slice-pair product summed over a 4096-long chunk is an integer of
  magnitude <= 2^24, exact in FP32 whatever the summation order;
* the product built from the kept pairs (i + j <= s - 1) meets the stated
  bound sum over chunks of L m_r n_c (2^{-6s}(s + 4) + (5 + chunks) u);
* balancing the K index of an A B product by B's row exponents keeps the
  accuracy of states whose norms differ by 1e5 (a filtered block), which
  per-column scaling alone loses.
"""
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -53
L_CHUNK = 4096


def digits(x, e, s):
    """Balanced base-64 digits (q_0 .. q_{s-1}) of round(x 2^{-e} 2^{6s}) for
    |x| < 2^e, in exact integer arithmetic (Python ints)."""
    F = Fraction(x) * Fraction(2) ** (6 * s - e)
    F = int(F + Fraction(1, 2)) if F >= 0 else -int(-F + Fraction(1, 2))
    q = [0] * s
    for i in range(s - 1, 0, -1):
        d = ((F + 32) & 63) - 32
        q[i] = d
        F = (F - d) >> 6
    q[0] = F
    return q


def frexp_exp(a):
    m = np.max(np.abs(a))
    return int(np.frexp(m)[1]) if m > 0 else 0


def test_digit_bounds_and_remainder():
    rng = np.random.default_rng(0)
    for trial in range(400):
        s = int(rng.integers(2, 11))
        row = rng.standard_normal(12) * 2.0 ** rng.integers(-1060, 1000) * 2.0 ** rng.integers(-60, 1, 12)
        if trial % 5 == 0:
            row[0] = 5e-324 * int(rng.integers(1, 10 ** 6))        # subnormal
        if trial % 7 == 0:
            row[1] = 0.0
        e = frexp_exp(row)
        for x in row:
            q = digits(float(x), e, s)
            assert abs(q[0]) <= 64 and all(-32 <= d <= 31 for d in q[1:])
            v = Fraction(float(x)) * Fraction(2) ** (-e)
            rem = abs(v - sum(Fraction(d) * Fraction(2) ** (-6 * (i + 1)) for i, d in enumerate(q)))
            assert rem <= Fraction(1, 2) * Fraction(2) ** (-6 * s)


def test_worst_case_chunk_sum_is_exact_in_fp32():
    # every entry at its row maximum gives q_0 = +-64 throughout: 4096 * 64 * 64 = 2^24
    q = digits(1.0 - 2.0 ** -53, 0, 10)
    assert q[0] == 64
    total = L_CHUNK * q[0] * q[0]
    assert total == 2 ** 24 and float(np.float32(total)) == total
    assert all(abs(a * b) * L_CHUNK <= 2 ** 24 for a in (64, 32) for b in (64, 32))


def split_rows(A, s):
    """Slices of the rows of A over K chunks as int64 arrays and exponents."""
    out = []
    for c0 in range(0, A.shape[1], L_CHUNK):
        a = A[:, c0:c0 + L_CHUNK]
        es = [frexp_exp(r) for r in a]
        Q = np.zeros((s,) + a.shape, dtype=np.int64)
        for r in range(a.shape[0]):
            for k in range(a.shape[1]):
                Q[:, r, k] = digits(float(a[r, k]), es[r], s)
        out.append((Q, np.array(es)))
    return out


def sliced_product(A, Bt, s):
    """A Bt^T from the slices, kept pairs i + j <= s - 1, exact integer pair
    products, FP64 combination as the reduction does it."""
    C = np.zeros((A.shape[0], Bt.shape[0]))
    for (Qa, ea), (Qb, eb) in zip(split_rows(A, s), split_rows(Bt, s)):
        g = [sum(Qa[i] @ Qb[t - i].T for i in range(t + 1)) for t in range(s)]
        h = 0.0
        for b in range((s + 4) // 5 - 1, -1, -1):
            B = np.zeros(C.shape, dtype=np.int64)
            for t in range(5 * b, 5 * b + 5):
                B = B * 64 + (g[t] if t < s else 0)
            h = h * 2.0 ** -30 + B.astype(np.float64)
        C += np.ldexp(h, ea[:, None] + eb[None, :] - 36)
    return C


def stated_bound(A, Bt, s):
    nch = -(-A.shape[1] // L_CHUNK)
    bound = np.zeros((A.shape[0], Bt.shape[0]))
    for c0 in range(0, A.shape[1], L_CHUNK):
        a, b = A[:, c0:c0 + L_CHUNK], Bt[:, c0:c0 + L_CHUNK]
        bound += a.shape[1] * np.outer(np.abs(a).max(1), np.abs(b).max(1)) * (2.0 ** (-6 * s) * (s + 4) + (5 + nch) * U)
    return bound


def exact_product(A, Bt):
    return np.array([[float(sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))) for b in Bt] for a in A])


@pytest.mark.parametrize("s", [4, 7, 10])
def test_sliced_product_within_stated_bound(s):
    rng = np.random.default_rng(s)
    M, N, K = 5, 4, L_CHUNK + 300                     # two chunks, the second ragged
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    Bt = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, 1)))
    A[1, 17] *= 1e4                                   # a spiky row
    C = sliced_product(A, Bt, s)
    ref = exact_product(A, Bt)
    assert np.all(np.abs(C - ref) <= stated_bound(A, Bt, s))


def test_balancing_keeps_small_norm_states():
    """Y_hat^T = U^{-T} Y^T with state norms 1e5 .. 1: with the K index
    (states) balanced by the exponents of Y^T's rows the sliced product is as
    accurate per output row as FP64; with per-column scaling alone the
    small-norm states lose digits."""
    rng = np.random.default_rng(1)
    N, Ns = 96, 24
    X = np.linalg.qr(rng.standard_normal((N, Ns)))[0]
    d = np.geomspace(1e5, 1.0, Ns)
    Y = X * d + 1e-3 * rng.standard_normal((N, Ns)) * d
    Lc = np.linalg.cholesky(Y.T @ Y)
    A = np.linalg.inv(Lc)                              # U^{-T}, lower triangular
    B = Y.T                                            # K (states) x N
    ref = exact_product(A, B.T)
    row_scale = np.abs(ref).max(axis=1, keepdims=True)
    s = 10
    plain = sliced_product(A, np.ascontiguousarray(B.T), s)
    sk = np.array([frexp_exp(r) for r in B])
    bal = sliced_product(np.ldexp(A, sk[None, :]), np.ascontiguousarray(np.ldexp(B, -sk[:, None]).T), s)
    err_plain = float(np.max(np.abs(plain - ref) / row_scale))
    err_bal = float(np.max(np.abs(bal - ref) / row_scale))
    err_f64 = float(np.max(np.abs(A @ B - ref) / row_scale))
    assert err_bal <= max(8 * err_f64, 1e-15) and err_plain > 100 * err_bal


def test_block_sparse_product_within_stated_bound():
    """H X from slices as the block-sparse product splits it: each row of H
    with one exponent over the columns of its neighbour blocks (at most 4096,
    one chunk), each state with one exponent over all N entries. The result is
    within L m_r n_s (2^{-6s}(s + 4) + 6 u) of the exact product, L the row's
    column count, m_r its largest |entry|, n_s the state's largest |entry| over
    all of it (so a state that is large away from the row's columns gets a
    looser but still valid bound)."""
    rng = np.random.default_rng(12)
    nb = [5, 7, 4, 6]                                   # a chain of 4 elements, neighbours K-1, K, K+1
    off = np.concatenate([[0], np.cumsum(nb)])
    N = int(off[-1])
    H = np.zeros((N, N))
    for K in range(4):
        for Kp in (K - 1, K, K + 1):
            if 0 <= Kp < 4:
                H[off[K]:off[K + 1], off[Kp]:off[Kp + 1]] = rng.standard_normal((nb[K], nb[Kp])) * 10.0 ** (K - 2)
    H = 0.5 * (H + H.T)
    Ns = 6
    X = rng.standard_normal((Ns, N)) * np.exp(rng.uniform(-3, 3, (Ns, 1)))
    X[2, off[3]:] *= 1e6                                # large only on the last element
    exact = np.array([[float(sum(Fraction(float(H[r, c])) * Fraction(float(X[t, c])) for c in range(N)))
                       for r in range(N)] for t in range(Ns)])
    for s in (4, 10):
        Y = np.zeros((Ns, N))
        bound = np.zeros((Ns, N))
        for r in range(N):
            cols = np.nonzero(H[r])[0]
            L = len(cols)
            er = frexp_exp(H[r, cols])
            qh = np.array([digits(float(H[r, c]), er, s) for c in cols], dtype=np.int64)      # L x s
            for t_ in range(Ns):
                es = frexp_exp(X[t_])
                qx = np.array([digits(float(X[t_, c]), es, s) for c in cols], dtype=np.int64)
                g = [int(sum(int(qh[:, i] @ qx[:, t - i]) for i in range(t + 1))) for t in range(s)]
                assert all(abs(int(qh[:, i] @ qx[:, j])) <= 2 ** 24 for i in range(s) for j in range(s - i))
                h = 0.0
                for b in range((s + 4) // 5 - 1, -1, -1):
                    Bv = 0
                    for t in range(5 * b, 5 * b + 5):
                        Bv = Bv * 64 + (g[t] if t < s else 0)
                    h = h * 2.0 ** -30 + float(Bv)
                Y[t_, r] = np.ldexp(h, er + es - 36)
                bound[t_, r] = L * np.abs(H[r, cols]).max() * np.abs(X[t_]).max() * (2.0 ** (-6 * s) * (s + 4) + 6 * U)
        assert np.all(np.abs(Y - exact) <= bound)
