"""Stored values of the tiny workload's first cycle (tests/golden, written by
tests/golden/make_golden.py from the FP64 oracle). CPU: the oracle still
reproduces them, so a change to its arithmetic shows up here and must come
with regenerated fixtures. GPU: the CUDA path matches them without calling
the oracle at test time."""
import os
import sys

import numpy as np
import pytest
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden as MG  # noqa: E402

from paper_1606_03416_gb300 import inputs as G  # noqa: E402

FIXTURE = os.path.join(HERE, "golden", "tiny_2x2x2_cycle1.txt")


def test_oracle_reproduces_stored_values():
    stored = MG.read(FIXTURE)
    now = MG.tiny_cycle_values()
    assert set(stored) == set(now)
    for k, v in now.items():
        v = np.asarray(v)
        assert np.max(np.abs(v - stored[k])) <= 1e-12 * max(1.0, np.max(np.abs(stored[k]))), k


@pytest.mark.gpu
def test_cuda_path_matches_stored_values():
    D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi")
    g = MG.read(FIXTURE)
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    dev = torch.device("cuda:0")
    scale = max(abs(g["a0"][0]), abs(g["b"][0]))
    with D.Context(H) as ctx:
        X = torch.from_numpy(X0).to(dev)
        v = torch.from_numpy(v0).to(dev)
        b, tmin = ctx.bounds(v, 10)
        assert abs(b - g["b"][0]) <= 1e-10 * scale and abs(tmin - g["a0"][0]) <= 1e-10 * scale
        Y = ctx.filter(X, cfg.m, g["a"][0], g["b"][0], g["a0"][0], prec="f64").cpu().numpy()
        assert abs(np.linalg.norm(Y) - g["filter_fro"][0]) <= 1e-12 * g["filter_fro"][0]
        assert np.max(np.abs(Y[0, :8] - g["filter_state0_first8"])) <= 1e-12 * np.max(np.abs(Y))
        out = ctx.cycle(X, cfg.m, Ne, cfg.kT, v0=v)
        ritz = out["ritz"].cpu().numpy()
        assert np.max(np.abs(ritz - g["ritz"])) <= 1e-10 * scale
        assert abs(float(out["mu"].item()) - g["mu"][0]) <= 1e-10 * scale
        f = out["f"].cpu().numpy()
        assert abs(f.sum() - g["sum_f"][0]) <= 1e-10 * Ns
        tr = sum(float(np.trace(p.cpu().numpy())) for p in ctx.unpack_density(out["P"]))
        assert abs(tr - g["trace_P"][0]) <= 1e-10 * Ns
        assert abs(float((f * ritz).sum()) - g["band_energy"][0]) <= 1e-10 * scale * Ns
