"""Pins of the oracle's rounded filter (oracle.chebyshev_filter_rounded): the
Chebyshev recurrence of Alg. 1 step 2 with the operand roundings of the
tensor-core precision forms (BF16, split BF16x3, TF32 operands, FP32
accumulation and iterates).

* The BF16 rounding equals PyTorch's float32 -> bfloat16 conversion
  (round to nearest, ties to even), ties included.
* The TF32 cut equals floor(|x| 2^(11 - e)) 2^(e - 11) with sign, e the
  frexp exponent of x (11 significant bits kept, the rest dropped).
* When every operand is exactly representable (small integers, a degree-1
  filter whose scalar is a power of two) no rounding happens and the rounded
  filter equals the FP64 one exactly, in every form.
* On the tiny workload each form's distance from the FP64 filter lies between
  a twentieth of and twice m u_op (so the roundings are applied, and applied
  once per operand), and the split form is more than 100 times closer than
  plain BF16.
"""
import numpy as np
import pytest
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G


def test_bf16_rounding_matches_torch_including_ties():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-30, 30, 200000))
    x32 = x.astype(np.float32)
    # exact ties: a BF16 value plus half of its last place, both parities of the kept bit
    base = rng.standard_normal(1000).astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    ties = (base | np.uint32(0x8000)).view(np.float32)
    for v in (x32, ties, -ties):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(O.round_bf16(v), ref)


def test_tf32_cut_keeps_eleven_significant_bits():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-30, 30, 100000))).astype(np.float32).astype(np.float64)
    f, e = np.frexp(np.abs(x))                         # |x| = f 2^e, f in [0.5, 1)
    ref = np.sign(x) * np.floor(f * 2.0 ** 11) * 2.0 ** (e - 11)
    assert np.array_equal(O.truncate_tf32(x), ref)


def _integer_problem():
    cfg = G.CONFIGS["tiny_2x2x2"]
    H = O.DGHamiltonian.from_blocksparse(G.make_blocks(cfg))
    rng = np.random.default_rng(3)
    vals = np.zeros_like(H.values)
    for K in range(H.M):          # symmetric blocks of small integers
        for e in range(H.row_ptr[K], H.row_ptr[K + 1]):
            Kp = int(H.col[e])
            if Kp < K:
                continue
            n, k = int(H.nb[K]), int(H.nb[Kp])
            B = rng.integers(-4, 5, size=(n, k)).astype(np.float64)
            if Kp == K:
                B = np.triu(B) + np.triu(B, 1).T
            vals[H.blk_off[e]:H.blk_off[e] + n * k] = B.ravel()
            if Kp != K:
                f = [f for f in range(H.row_ptr[Kp], H.row_ptr[Kp + 1]) if int(H.col[f]) == K][0]
                vals[H.blk_off[f]:H.blk_off[f] + n * k] = B.T.ravel()
    X = rng.integers(-8, 9, size=(H.N, 5)).astype(np.float64)
    return O.DGHamiltonian(H.nb, H.row_ptr, H.col, H.blk_off, vals), X


@pytest.mark.parametrize("fmt", ["bf16", "bf16x3", "tf32"])
def test_exact_operands_are_not_rounded(fmt):
    H, X = _integer_problem()
    # a = 0, b = 4, a0 = -2: c = 2, e = 2, sigma_1 = -1/2, alpha_0 = -1/4 (exact)
    ref = O.chebyshev_filter(H, X, 1, 0.0, 4.0, -2.0)
    got = O.chebyshev_filter_rounded(H, X, 1, 0.0, 4.0, -2.0, fmt)
    assert np.array_equal(got, ref)


def test_rounding_error_sizes_on_the_tiny_workload():
    cfg = G.CONFIGS["tiny_2x2x2"]
    Hb, X0, _, Ns, _ = G.make_problem(cfg)
    H = O.DGHamiltonian.from_blocksparse(Hb)
    lam = np.linalg.eigvalsh(H.dense())
    a0, b, a = lam[0] - 0.5, lam[-1] + 0.5, lam[Ns]
    m = cfg.m
    ref = O.chebyshev_filter(H, X0.T, m, a, b, a0)
    err = {}
    for fmt, u in (("bf16", 2.0 ** -8), ("tf32", 2.0 ** -10), ("bf16x3", 2.0 ** -16)):
        Y = O.chebyshev_filter_rounded(H, X0.T, m, a, b, a0, fmt)
        err[fmt] = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
        assert 0.05 * m * u <= err[fmt] <= 2 * m * u, (fmt, err[fmt])
    assert err["bf16x3"] * 100 < err["bf16"]
