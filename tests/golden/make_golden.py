"""Writes the stored expected values under tests/golden from the FP64 oracle
only (no CUDA code is imported or run). Usage: python tests/golden/make_golden.py

tiny_2x2x2_cycle1.txt: the first CheFSI cycle (Alg. 1) of the tiny 2x2x2
workload (n_b = 32, N = 256, N_s = 48, m = 10, N_e = 64, kT = 0.01, seed 0):
  * Alg. 1 step 1: Lanczos upper bound b (10 steps, seeded start vector) and
    the first-cycle reading of the lower bounds a0 = theta_min, a = a0 +
    (b - a0) N_s / N;
  * Alg. 1 step 2 (scaled three-term recurrence): the Frobenius norm of the
    filtered block and its first 8 entries of state 0;
  * Alg. 1 steps 3-5: the N_s Ritz values;
  * occupations (spin factor 2, bisection for mu): mu and sum_i f_i;
  * density blocks (Eq. densitymatrix, K' = K): sum_K tr P_KK;
  * band energy E = sum_i f_i lambda_i of the cycle.

bulk3d_8x8x8_spectrum.txt (written only with --spectrum: a dense eigensolve
of the N = 32768 matrix, about an hour of host time): the ceil(N_e / 2) = 3973
smallest eigenvalues of the 8x8x8 bulk-3D workload's H (seed 0), the exact
values the occupied Ritz values converge to (Alg. 1), from
oracle.chefsi.lowest_eigenvalues. The benchmark measures cycles to a Ritz
error of 1e-8 against them.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import chefsi as O  # noqa: E402
from paper_1606_03416_gb300 import inputs as G  # noqa: E402


def tiny_cycle_values():
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    Ho = O.DGHamiltonian.from_blocksparse(H)
    out = O.chefsi_cycle(Ho, X0.T, cfg.m, Ne, cfg.kT, v0)
    Yt = O.chebyshev_filter(Ho, X0.T, cfg.m, out["a"], out["b"], out["a0"])
    return {
        "a": [out["a"]], "b": [out["b"]], "a0": [out["a0"]],
        "filter_fro": [float(np.linalg.norm(Yt))],
        "filter_state0_first8": [float(v) for v in Yt[:8, 0]],
        "ritz": [float(v) for v in out["ritz"]],
        "mu": [out["mu"]], "sum_f": [float(np.sum(out["f"]))],
        "trace_P": [float(sum(np.trace(p) for p in out["P"]))],
        "band_energy": [float(np.sum(out["f"] * out["ritz"]))],
    }


def bulk3d_spectrum():
    cfg = G.CONFIGS["bulk3d_8x8x8"]
    H = G.make_blocks(cfg)
    n = int(np.ceil(cfg.Ne / 2))
    lam = O.lowest_eigenvalues(O.DGHamiltonian.from_blocksparse(H), n)
    return {"n": [n], "eigenvalues": [float(v) for v in lam]}


def write(path, values, header):
    with open(path, "w") as fh:
        for line in header.strip().splitlines():
            fh.write(f"# {line}\n")
        for k, v in values.items():
            fh.write(f"{k}: " + " ".join(repr(float(x)) for x in v) + "\n")


def read(path):
    vals = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, rest = line.split(":", 1)
            vals[k.strip()] = np.array([float(x) for x in rest.split()])
    return vals


if __name__ == "__main__":
    if "--spectrum" in sys.argv:
        write(os.path.join(HERE, "bulk3d_8x8x8_spectrum.txt"), bulk3d_spectrum(),
              "The ceil(N_e/2) = 3973 smallest eigenvalues of the 8x8x8 bulk-3D H (seed 0),\n"
              "ascending, written by tests/golden/make_golden.py --spectrum from the FP64\n"
              "oracle (dense symmetric eigensolve of the assembled H).")
        print("written spectrum")
        sys.exit(0)
    write(os.path.join(HERE, "tiny_2x2x2_cycle1.txt"), tiny_cycle_values(),
          "First CheFSI cycle of the tiny 2x2x2 workload (seed 0), written by\n"
          "tests/golden/make_golden.py from the FP64 oracle (Alg. 1 steps 1-5,\n"
          "occupations, Eq. densitymatrix). See that script for each quantity.")
    print("written")
