"""Host logic of the autograd wrapper (no GPU): the mirror index and the
symmetric tying of per-entry gradients agree with the oracle's definition."""
import numpy as np
import torch

from oracle import chefsi as O
from paper_1606_03416_gb300 import inputs as G


def test_tie_symmetric_matches_oracle_definition():
    from paper_1606_03416_gb300 import autograd as A
    cfg = G.ProblemConfig(name="t", grid=(3, 2, 2), periodic=(True, False, True), stencil="27", nb=(3, 6), Ns=4,
                          m=2, Ne=4.0, seed=2)
    bs = G.make_blocks(cfg)
    H = O.DGHamiltonian.from_blocksparse(bs)
    rng = np.random.default_rng(0)
    g = rng.standard_normal(bs.values.shape[0])
    mirror = A.mirror_index(bs)
    assert np.array_equal(bs.values[mirror], bs.values)          # H is symmetric
    assert np.array_equal(mirror[mirror], np.arange(mirror.size))  # an involution
    tied = A.tie_symmetric(torch.from_numpy(g), mirror).numpy()
    blocks, e = [], 0
    for K in range(H.M):
        for Kp, blk in H.neighbours(K):
            n = blk.size
            blocks.append(g[bs.blk_off[e]:bs.blk_off[e] + n].reshape(blk.shape))
            e += 1
    ref = np.concatenate([t.ravel() for t in O.tied_gradient(H, blocks)])
    assert np.allclose(tied, ref, rtol=0, atol=1e-14)
