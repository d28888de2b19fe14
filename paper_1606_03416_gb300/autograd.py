"""torch.autograd.Function for the band energy of one CheFSI cycle.

E(values, X) = sum_i f_i lambda_i after one cycle (filter -> Cholesky-QR ->
Rayleigh-Ritz -> Fermi occupations) with the filter bounds, N_e and kT held
fixed. Forward and backward both run in the library (dgchefsi_energy_grad):
the backward recomputes the forward, keeping iterate pairs every
ceil(sqrt(m)) filter steps and recomputing each segment in reverse.

``values`` are H's stored block entries in the layout given to the context;
its gradient treats every stored entry as independent. For a symmetric
parameterisation (H_KK'[j, j'] and H_K'K[j', j] one parameter) use
``tie_symmetric``.
"""
from __future__ import annotations

import numpy as np
import torch


class BandEnergy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, values, X, lib_ctx, m, a, b, a0, Ne, kT, stride=0, prec="f64"):
        lib_ctx.set_values(values)
        E, _, _, _ = lib_ctx.energy_grad(X, m, a, b, a0, Ne, kT, grad=False, prec=prec)
        fctx.save_for_backward(values, X)
        fctx.params = (lib_ctx, m, a, b, a0, Ne, kT, stride, prec)
        return torch.tensor(E, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(fctx, gE):
        values, X = fctx.saved_tensors
        lib_ctx, m, a, b, a0, Ne, kT, stride, prec = fctx.params
        lib_ctx.set_values(values)
        _, _, Hb, Xb = lib_ctx.energy_grad(X, m, a, b, a0, Ne, kT, grad=True, stride=stride, prec=prec)
        return gE * Hb, gE * Xb, None, None, None, None, None, None, None, None, None


def band_energy(values, X, lib_ctx, m, a, b, a0, Ne, kT, stride=0, prec="f64"):
    """E = sum_i f_i lambda_i of one cycle; prec selects the filter's arithmetic
    ("f64", or a tensor-core form "tf32", "bf16", "bf16x3" with FP32 iterates)."""
    return BandEnergy.apply(values, X, lib_ctx, m, a, b, a0, Ne, kT, stride, prec)


def mirror_index(H) -> np.ndarray:
    """For every stored entry H_KK'[j, j'] the position of H_K'K[j', j]."""
    nb, rp, col, off = (np.asarray(H.nb), np.asarray(H.row_ptr), np.asarray(H.col), np.asarray(H.blk_off))
    where = {}
    for K in range(len(nb)):
        for e in range(rp[K], rp[K + 1]):
            where[(K, int(col[e]))] = e
    mirror = np.empty(int(np.asarray(H.values).shape[0]), dtype=np.int64)
    for (K, Kp), e in where.items():
        f = where[(Kp, K)]
        nK, nKp = int(nb[K]), int(nb[Kp])
        j = np.arange(nK)[:, None]
        jp = np.arange(nKp)[None, :]
        mirror[off[e] + (j * nKp + jp).ravel()] = (off[f] + jp * nK + j).ravel()
    return mirror


def tie_symmetric(grad_values: torch.Tensor, mirror: np.ndarray) -> torch.Tensor:
    """dE for symmetric perturbations: g + g[mirror], counting self-mirrored
    (diagonal) entries once."""
    idx = torch.as_tensor(mirror, device=grad_values.device)
    self_mirrored = idx == torch.arange(idx.numel(), device=grad_values.device)
    return torch.where(self_mirrored, grad_values, grad_values + grad_values[idx])
