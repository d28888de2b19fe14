"""Thin ctypes binding of libdgchefsi.so (C ABI in include/dgchefsi.h).

Argument marshalling only: every step runs in the library's CUDA kernels (and
its cuSOLVER calls for the dense N_s x N_s factorisations). Torch tensors are
used for device memory and the current CUDA stream. There is no CPU fallback:
if the library is missing, importing this module raises.

Layout: a block of N_s vectors is a float64 CUDA tensor of shape (N_s, N) (or a
row-strided view of a wider (N_s, ld) tensor), row i = state i. This is the
paper's N x N_s block X transposed.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libdgchefsi.so")

PRECISIONS = {"f64": 0, "tf32": 1, "bf16": 2, "bf16x3": 3}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NOT_SPD", 5: "ERR_NONFINITE",
          6: "ERR_NO_CONVERGENCE", 7: "ERR_TIMEOUT", 8: "ERR_UNSUPPORTED"}

EXPORTS = ["dgchefsi_create", "dgchefsi_destroy", "dgchefsi_set_stream", "dgchefsi_dims", "dgchefsi_matvec",
           "dgchefsi_bounds", "dgchefsi_filter", "dgchefsi_rayleigh_ritz", "dgchefsi_occupations",
           "dgchefsi_density_blocks", "dgchefsi_cycle", "dgchefsi_last_error", "dgchefsi_launch_count",
           "dgchefsi_bounds_static", "dgchefsi_gram", "dgchefsi_set_values", "dgchefsi_energy_grad",
           "dgchefsi_filter_graph", "dgchefsi_set_tile_shape", "dgchefsi_get_tile_shape",
           "dgchefsi_selftest_wait", "dgchefsi_selftest_fp64_rate", "dgchefsi_set_orthonormalisation", "dgchefsi_density_pattern",
           "dgchefsi_realign", "dgchefsi_filter_host", "dgchefsi_set_subspace_products",
           "dgchefsi_sliced_gemm", "dgchefsi_sliced_matvec", "dgchefsi_set_unit_order",
           "dgchefsi_get_unit_order", "dgchefsi_sliced_timing", "dgchefsi_set_eigensolver",
           "dgchefsi_subspace_eigh", "dgchefsi_eigensolver_stats", "dgchefsi_set_cholesky",
           "dgchefsi_cholesky_inverse", "dgchefsi_set_refinement_start", "dgchefsi_eigensolver_history"]

# Orthonormalisations of Alg. 1 step 3 (dgchefsi_set_orthonormalisation).
ORTHONORMALISATIONS = {"cholqr": 0, "cholqr2": 1, "shifted_cholqr3": 2}

# Arithmetic of the Rayleigh-Ritz products (dgchefsi_set_subspace_products).
SUBSPACE_PRODUCTS = {"f64": 0, "sliced_bf16": 1}

# Eigensolver of the projected Hamiltonian (dgchefsi_set_eigensolver).
EIGENSOLVERS = {"auto": 0, "syevd": 1, "refined": 2}
EIGENSOLVER_NAMES = {v: k for k, v in EIGENSOLVERS.items()}

# Cholesky form of Alg. 1 step 3 (dgchefsi_set_cholesky).
CHOLESKY_FORMS = {"auto": 0, "cusolver": 1, "products": 2}

# Capacity (doubles) of the library's fixed scratch array for bounds_static.
BOUNDS_STATIC_DOUBLES = 1 << 20


class DGChefsiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = STATUS.get(status, str(status))


def load_library(path: str = _LIBPATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    st = C.c_int
    sig = {
        "dgchefsi_create": (st, [I32, P, P, P, P, P, I64, P, C.POINTER(C.c_void_p)]),
        "dgchefsi_destroy": (None, [P]),
        "dgchefsi_set_stream": (st, [P, P]),
        "dgchefsi_dims": (st, [P, P, P]),
        "dgchefsi_matvec": (st, [P, P, P, I64, I64]),
        "dgchefsi_bounds": (st, [P, P, C.c_int, P, P]),
        "dgchefsi_bounds_static": (st, [P, P, C.c_int, P, P]),
        "dgchefsi_filter": (st, [P, C.c_int, P, P, I64, I64, C.c_int, D, D, D]),
        "dgchefsi_rayleigh_ritz": (st, [P, P, I64, I64, P]),
        "dgchefsi_gram": (st, [P, P, I64, I64, P]),
        "dgchefsi_filter_graph": (st, [P, C.c_int, P, P, I64, I64, C.c_int, D, D, D]),
        "dgchefsi_set_tile_shape": (st, [P, C.c_int, C.c_int, C.c_int, C.c_int]),
        "dgchefsi_get_tile_shape": (st, [P, C.c_int, P, P, P, P]),
        "dgchefsi_selftest_wait": (st, [P, I64]),
        "dgchefsi_selftest_fp64_rate": (st, [P, C.c_int, P]),
        "dgchefsi_set_orthonormalisation": (st, [P, C.c_int]),
        "dgchefsi_set_subspace_products": (st, [P, C.c_int, C.c_int]),
        "dgchefsi_sliced_gemm": (st, [P, C.c_int, C.c_int, I64, I64, I64, P, I64, P, I64, P, I64, C.c_int, I64]),
        "dgchefsi_sliced_matvec": (st, [P, P, P, I64, I64, C.c_int]),
        "dgchefsi_set_unit_order": (st, [P, C.c_int, C.c_int]),
        "dgchefsi_get_unit_order": (st, [P, C.c_int, P]),
        "dgchefsi_sliced_timing": (st, [P, P, P]),
        "dgchefsi_set_eigensolver": (st, [P, C.c_int]),
        "dgchefsi_set_cholesky": (st, [P, C.c_int]),
        "dgchefsi_set_refinement_start": (st, [P, D]),
        "dgchefsi_eigensolver_history": (st, [P, P, P, C.c_int, P]),
        "dgchefsi_cholesky_inverse": (st, [P, P, I64, I64]),
        "dgchefsi_subspace_eigh": (st, [P, P, I64, I64, P]),
        "dgchefsi_eigensolver_stats": (st, [P, P, P, P, P, P, P, P, P, P]),
        "dgchefsi_density_pattern": (st, [P, P, I64, I64, P, P]),
        "dgchefsi_realign": (st, [P, P, P, P, P, P, I64, I64, P, I64]),
        "dgchefsi_filter_host": (st, [P, C.c_int, P, P, I64, I64, C.c_int, D, D, D, I64]),
        "dgchefsi_set_values": (st, [P, P]),
        "dgchefsi_energy_grad": (st, [P, C.c_int, P, I64, I64, C.c_int, D, D, D, D, D, C.c_int, P, P, P, P]),
        "dgchefsi_occupations": (st, [P, P, I64, D, D, P, P]),
        "dgchefsi_density_blocks": (st, [P, P, I64, I64, P, P]),
        "dgchefsi_cycle": (st, [P, C.c_int, P, I64, I64, C.c_int, D, D, P, C.c_int, P, P, C.c_int, P, P, P, P]),
        "dgchefsi_last_error": (C.c_char_p, []),
        "dgchefsi_launch_count": (I64, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def last_error() -> str:
    return _lib.dgchefsi_last_error().decode()


def launch_count() -> int:
    return int(_lib.dgchefsi_launch_count())


def _check(status: int):
    if status != 0:
        raise DGChefsiError(status, last_error())


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _block(X: torch.Tensor, N: int, name: str):
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2):
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor (N_s, N)")
    if X.shape[1] != N or (X.shape[0] > 1 and X.stride(1) != 1) or (X.shape[0] > 0 and X.stride(1) != 1):
        raise ValueError(f"{name} must have shape (N_s, {N}) with unit column stride")
    ld = X.stride(0) if X.shape[0] > 1 else N
    return X.shape[0], max(ld, N)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Context:
    """A device copy of the block-sparse H and the library's workspace.

    ``H`` is any object with the block-CSR fields nb, row_ptr, col, blk_off and
    values (see paper_1606_03416_gb300.inputs.BlockSparse)."""

    def __init__(self, H):
        nb = np.ascontiguousarray(H.nb, dtype=np.int32)
        row_ptr = np.ascontiguousarray(H.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(H.col, dtype=np.int32)
        blk_off = np.ascontiguousarray(H.blk_off, dtype=np.int64)
        values = np.ascontiguousarray(H.values, dtype=np.float64)
        h = C.c_void_p()
        _check(_lib.dgchefsi_create(int(nb.shape[0]), nb.ctypes.data, row_ptr.ctypes.data, col.ctypes.data,
                                    blk_off.ctypes.data, values.ctypes.data, int(values.shape[0]), _stream(),
                                    C.byref(h)))
        self._h = h
        N, M = C.c_int64(), C.c_int32()
        _check(_lib.dgchefsi_dims(h, C.byref(N), C.byref(M)))
        self.N, self.M = int(N.value), int(M.value)
        self.nb = nb
        self.n_values = int(values.shape[0])
        self.density_offsets = np.concatenate([[0], np.cumsum(nb.astype(np.int64) ** 2)])

    def close(self):
        if getattr(self, "_h", None):
            _lib.dgchefsi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _sync_stream(self):
        _check(_lib.dgchefsi_set_stream(self._h, _stream()))

    # -- Eq. matvec_3
    def matvec(self, X: torch.Tensor, Y: torch.Tensor | None = None) -> torch.Tensor:
        Ns, ld = _block(X, self.N, "X")
        if Y is None:
            Y = torch.empty_like(X)
        Ns2, ld2 = _block(Y, self.N, "Y")
        if (Ns2, ld2) != (Ns, ld):
            raise ValueError("X and Y need the same shape and stride")
        self._sync_stream()
        _check(_lib.dgchefsi_matvec(self._h, _ptr(X), _ptr(Y), Ns, ld))
        return Y

    # -- Alg. 1 step 1
    def bounds(self, v0: torch.Tensor, k: int = 10):
        if not (v0.is_cuda and v0.dtype == torch.float64 and v0.numel() == self.N and v0.is_contiguous()):
            raise ValueError("v0 must be a contiguous float64 CUDA vector of length N")
        b, t = C.c_double(), C.c_double()
        self._sync_stream()
        _check(_lib.dgchefsi_bounds(self._h, _ptr(v0), int(k), C.byref(b), C.byref(t)))
        return b.value, t.value

    def bounds_static(self, v0: torch.Tensor, k: int = 10):
        """Same as ``bounds`` but without any device allocation: the Krylov basis
        lives in a fixed array inside the library (see include/dgchefsi.h)."""
        if not (v0.is_cuda and v0.dtype == torch.float64 and v0.numel() == self.N and v0.is_contiguous()):
            raise ValueError("v0 must be a contiguous float64 CUDA vector of length N")
        b, t = C.c_double(), C.c_double()
        self._sync_stream()
        _check(_lib.dgchefsi_bounds_static(self._h, _ptr(v0), int(k), C.byref(b), C.byref(t)))
        return b.value, t.value

    # -- Alg. 1 step 2
    def filter(self, X: torch.Tensor, m: int, a: float, b: float, a0: float, prec: str = "f64",
               Y: torch.Tensor | None = None) -> torch.Tensor:
        Ns, ld = _block(X, self.N, "X")
        if Y is None:
            Y = torch.empty_like(X)
        Ns2, ld2 = _block(Y, self.N, "Y")
        if (Ns2, ld2) != (Ns, ld):
            raise ValueError("X and Y need the same shape and stride")
        self._sync_stream()
        _check(_lib.dgchefsi_filter(self._h, PRECISIONS[prec], _ptr(X), _ptr(Y), Ns, ld, int(m), float(a),
                                    float(b), float(a0)))
        return Y

    # -- Alg. 1 step 3, first product
    def gram(self, Y: torch.Tensor, S: torch.Tensor | None = None) -> torch.Tensor:
        Ns, ld = _block(Y, self.N, "Y")
        if S is None:
            S = torch.empty((Ns, Ns), dtype=torch.float64, device=Y.device)
        self._sync_stream()
        _check(_lib.dgchefsi_gram(self._h, _ptr(Y), Ns, ld, _ptr(S)))
        return S

    def filter_host(self, X: torch.Tensor, m: int, a: float, b: float, a0: float, prec: str = "bf16x3",
                    Y: torch.Tensor | None = None, chunk: int = 0) -> torch.Tensor:
        """The filter on host (CPU) float64 blocks, (N_s, N) with unit column
        stride; copies in, filters and copies out in overlapping chunks. Pinned
        tensors (``pin_memory()``) let the copies overlap the filter."""
        if not (isinstance(X, torch.Tensor) and X.device.type == "cpu" and X.dtype == torch.float64 and X.dim() == 2):
            raise TypeError("X must be a 2-D float64 CPU tensor (N_s, N)")
        if X.shape[1] != self.N or (X.shape[0] > 0 and X.stride(1) != 1):
            raise ValueError(f"X must have shape (N_s, {self.N}) with unit column stride")
        ld = max(X.stride(0) if X.shape[0] > 1 else self.N, self.N)
        if Y is None:
            Y = torch.empty(X.shape, dtype=torch.float64, pin_memory=X.is_pinned())
        if Y.device.type != "cpu" or Y.dtype != torch.float64 or Y.shape != X.shape or \
                (Y.shape[0] > 1 and Y.stride(0) != ld) or (Y.shape[0] > 0 and Y.stride(1) != 1):
            raise ValueError("Y must be a CPU float64 tensor laid out like X")
        self._sync_stream()
        _check(_lib.dgchefsi_filter_host(self._h, PRECISIONS[prec], _ptr(X), _ptr(Y), X.shape[0], ld, int(m),
                                         float(a), float(b), float(a0), int(chunk)))
        return Y

    def filter_graph(self, X: torch.Tensor, m: int, a: float, b: float, a0: float, prec: str = "bf16x3",
                     Y: torch.Tensor | None = None) -> torch.Tensor:
        """The filter replayed from a CUDA graph (captured on first use); any precision."""
        Ns, ld = _block(X, self.N, "X")
        if Y is None:
            Y = torch.empty_like(X)
        self._sync_stream()
        _check(_lib.dgchefsi_filter_graph(self._h, PRECISIONS[prec], _ptr(X), _ptr(Y), Ns, ld, int(m), float(a),
                                          float(b), float(a0)))
        return Y

    def selftest_wait(self, limit_ns: int = 50_000_000):
        """Run the bounded-wait self-test; returns the status name (ERR_TIMEOUT expected)."""
        st = _lib.dgchefsi_selftest_wait(self._h, int(limit_ns))
        return STATUS.get(st, str(st)), last_error()

    def fp64_rate(self, reps: int = 10) -> float:
        """Best FP64 DFMA rate of the GPU's CUDA cores over `reps` probe launches (flop/s)."""
        r = C.c_double()
        self._sync_stream()
        _check(_lib.dgchefsi_selftest_fp64_rate(self._h, int(reps), C.byref(r)))
        return r.value

    def set_tile_shape(self, prec: str, G: int, T: int, layout: int = 0):
        _check(_lib.dgchefsi_set_tile_shape(self._h, PRECISIONS[prec], int(G), int(T), int(layout)))

    def set_unit_order(self, prec: str, tgb: int = -1):
        """State tiles per pass over the element groups (0: a group's tiles back to back; -1: tune)."""
        _check(_lib.dgchefsi_set_unit_order(self._h, PRECISIONS[prec], int(tgb)))

    def unit_order(self, prec: str) -> int:
        v = C.c_int()
        _check(_lib.dgchefsi_get_unit_order(self._h, PRECISIONS[prec], C.byref(v)))
        return v.value

    def tile_shape(self, prec: str):
        """(G, T, ACC, layout) of the tensor-core filter for this precision."""
        g, t, acc, lay = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(_lib.dgchefsi_get_tile_shape(self._h, PRECISIONS[prec], C.byref(g), C.byref(t), C.byref(acc),
                                            C.byref(lay)))
        return g.value, t.value, acc.value, lay.value

    # -- Alg. 1 steps 3-5 (in place: Y becomes X_new)
    def rayleigh_ritz(self, Y: torch.Tensor, ritz: torch.Tensor | None = None) -> torch.Tensor:
        Ns, ld = _block(Y, self.N, "Y")
        if ritz is None:
            ritz = torch.empty(Ns, dtype=torch.float64, device=Y.device)
        self._sync_stream()
        _check(_lib.dgchefsi_rayleigh_ritz(self._h, _ptr(Y), Ns, ld, _ptr(ritz)))
        return ritz

    def occupations(self, ritz: torch.Tensor, Ne: float, kT: float):
        f = torch.empty_like(ritz)
        mu = torch.empty(1, dtype=torch.float64, device=ritz.device)
        self._sync_stream()
        _check(_lib.dgchefsi_occupations(self._h, _ptr(ritz), ritz.numel(), float(Ne), float(kT), _ptr(f), _ptr(mu)))
        return f, mu

    def density_blocks(self, X: torch.Tensor, f: torch.Tensor, P: torch.Tensor | None = None) -> torch.Tensor:
        Ns, ld = _block(X, self.N, "X")
        if P is None:
            P = torch.empty(int(self.density_offsets[-1]), dtype=torch.float64, device=X.device)
        self._sync_stream()
        _check(_lib.dgchefsi_density_blocks(self._h, _ptr(X), Ns, ld, _ptr(f), _ptr(P)))
        return P

    def density_pattern(self, X: torch.Tensor, f: torch.Tensor, P: torch.Tensor | None = None) -> torch.Tensor:
        """P_KK' = sum_i f_i x_{i;K} x_{i;K'}^T on every stored block of H, laid
        out like H's values."""
        Ns, ld = _block(X, self.N, "X")
        if P is None:
            P = torch.empty(self.n_values, dtype=torch.float64, device=X.device)
        self._sync_stream()
        _check(_lib.dgchefsi_density_pattern(self._h, _ptr(X), Ns, ld, _ptr(f), _ptr(P)))
        return P

    def set_orthonormalisation(self, mode: str):
        """"cholqr" (Alg. 1 step 3 as in the paper), "cholqr2" or "shifted_cholqr3"."""
        _check(_lib.dgchefsi_set_orthonormalisation(self._h, ORTHONORMALISATIONS[mode]))

    def set_subspace_products(self, mode: str, slices: int = 10):
        """"f64" (FP64 cores) or "sliced_bf16" (FP64 products rebuilt from
        `slices` exact BF16 slices per operand on the tensor cores) for the
        Gram, Y U^-1, projected-H and rotation products of Rayleigh-Ritz."""
        _check(_lib.dgchefsi_set_subspace_products(self._h, SUBSPACE_PRODUCTS[mode], int(slices)))

    def sliced_gemm(self, A: torch.Tensor, B: torch.Tensor, b_rows: bool = True, a_lower: bool = False,
                    slices: int = 10, out: torch.Tensor | None = None, tri: int = 0) -> torch.Tensor:
        """A @ B.T (b_rows) or A @ B in FP64 from exact BF16 slices. A, B: 2-D
        float64 CUDA tensors, rows contiguous; a_lower treats A as lower
        triangular; tri > 0 computes only the entries (r, c) with c <= r % tri."""
        for name, T in (("A", A), ("B", B)):
            if not (T.is_cuda and T.dtype == torch.float64 and T.dim() == 2 and T.stride(1) == 1):
                raise TypeError(f"{name} must be a 2-D float64 CUDA tensor with contiguous rows")
        M, K = A.shape
        Nc = B.shape[0] if b_rows else B.shape[1]
        if (B.shape[1] if b_rows else B.shape[0]) != K:
            raise ValueError("inner dimensions differ")
        if out is None:
            out = torch.empty((M, Nc), dtype=torch.float64, device=A.device)
        if not (out.is_cuda and out.dtype == torch.float64 and out.shape == (M, Nc) and out.stride(1) == 1):
            raise TypeError("out must be a float64 CUDA tensor of shape (M, Nc) with contiguous rows")
        self._sync_stream()
        _check(_lib.dgchefsi_sliced_gemm(self._h, int(b_rows), int(a_lower), M, Nc, K, _ptr(A), A.stride(0),
                                         _ptr(B), B.stride(0), _ptr(out), out.stride(0), int(slices), int(tri)))
        return out

    def set_cholesky(self, mode: str):
        """"auto", "cusolver" (potrf + trtri) or "products" (recursive blocked
        form on dense products) for the Cholesky factorisation of Alg. 1 step 3."""
        _check(_lib.dgchefsi_set_cholesky(self._h, CHOLESKY_FORMS[mode]))

    def cholesky_inverse(self, S: torch.Tensor) -> torch.Tensor:
        """In place: the lower triangle of S (n x n float64 CUDA, rows
        contiguous, symmetric positive definite) is replaced by L^{-1} for
        S = L L^T; returns S."""
        if not (S.is_cuda and S.dtype == torch.float64 and S.dim() == 2 and S.shape[0] == S.shape[1]
                and S.stride(1) == 1):
            raise TypeError("S must be a square float64 CUDA tensor with contiguous rows")
        self._sync_stream()
        _check(_lib.dgchefsi_cholesky_inverse(self._h, _ptr(S), S.shape[0], S.stride(0)))
        return S

    def set_eigensolver(self, mode: str):
        """"auto", "syevd" (cuSOLVER FP64) or "refined" (FP32 start refined to
        FP64 by dense sliced products) for the eigensolve of Alg. 1 step 4."""
        _check(_lib.dgchefsi_set_eigensolver(self._h, EIGENSOLVERS[mode]))

    def subspace_eigh(self, A: torch.Tensor, w: torch.Tensor | None = None):
        """Eigen-decomposition of the symmetric matrix whose lower triangle is
        in A (n x n float64 CUDA, rows contiguous), in place: returns (w, A)
        with w ascending and row i of A the eigenvector of w[i]."""
        if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2 and A.shape[0] == A.shape[1]
                and A.stride(1) == 1):
            raise TypeError("A must be a square float64 CUDA tensor with contiguous rows")
        n = A.shape[0]
        if w is None:
            w = torch.empty(n, dtype=torch.float64, device=A.device)
        if not (w.is_cuda and w.dtype == torch.float64 and w.numel() == n and w.is_contiguous()):
            raise TypeError("w must be a contiguous float64 CUDA vector of length n")
        self._sync_stream()
        _check(_lib.dgchefsi_subspace_eigh(self._h, _ptr(A), n, A.stride(0), _ptr(w)))
        return w, A

    def eigensolver_stats(self) -> dict:
        """What the last eigensolve did (see dgchefsi_eigensolver_stats)."""
        i = [C.c_int() for _ in range(4)]
        d = [C.c_double() for _ in range(3)]
        order = C.c_int64()
        solver = C.c_int()
        _check(_lib.dgchefsi_eigensolver_stats(self._h, *[C.byref(x) for x in i], *[C.byref(x) for x in d],
                                               C.byref(order), C.byref(solver)))
        hist = (C.c_double * 16)()
        cnt = C.c_int()
        sl = (C.c_int * 16)()
        _check(_lib.dgchefsi_eigensolver_history(self._h, hist, sl, 16, C.byref(cnt)))
        return {"used": EIGENSOLVER_NAMES.get(i[0].value, i[0].value), "steps": i[1].value,
                "max_cluster": i[2].value, "fallback": i[3].value, "update": d[0].value,
                "start_ms": d[1].value, "refine_ms": d[2].value, "start_order": order.value,
                "start_solver": {0: "none", 1: "jacobi", 2: "cusolver_fp32"}.get(solver.value, solver.value),
                "history": [hist[k] for k in range(cnt.value)],
                "update_slices": [sl[k] for k in range(cnt.value)]}

    def set_refinement_start(self, coupling: float = 0.001):
        """First-order coupling at which a row joins the FP32 start block of
        the refined eigensolve (default 0.001)."""
        _check(_lib.dgchefsi_set_refinement_start(self._h, float(coupling)))

    def sliced_timing(self):
        """(ms, launches) of the slice-pair kernel in the last dense sliced product."""
        ms, n = C.c_double(), C.c_int64()
        _check(_lib.dgchefsi_sliced_timing(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def sliced_matvec(self, X: torch.Tensor, Y: torch.Tensor | None = None, slices: int = 10) -> torch.Tensor:
        """Y = H X (Eq. matvec_3) in FP64 from exact BF16 slices on the tensor cores."""
        Ns, ld = _block(X, self.N, "X")
        if Y is None:
            Y = torch.empty_like(X)
        Ns2, ld2 = _block(Y, self.N, "Y")
        if Ns2 != Ns or ld2 != ld:
            raise ValueError("X and Y must have the same shape and row stride")
        self._sync_stream()
        _check(_lib.dgchefsi_sliced_matvec(self._h, _ptr(X), _ptr(Y), Ns, ld, int(slices)))
        return Y

    # -- Sec. III.B.3: coefficients carried to the next SCF step's basis
    def realign(self, X_old: torch.Tensor, nb_old, nr, V_old: torch.Tensor, V_new: torch.Tensor,
                X_new: torch.Tensor | None = None) -> torch.Tensor:
        """X_new_K = (V_K^new)^T V_K^old X_old_K for every element. X_old is
        (N_s, sum nb_old) state-major; V_old / V_new are the packed per-element
        R_K x J_K sample blocks (float64 CUDA); this context's H is the new one."""
        nb_old = np.ascontiguousarray(nb_old, dtype=np.int32)
        nr = np.ascontiguousarray(nr, dtype=np.int32)
        if nb_old.shape != (self.M,) or nr.shape != (self.M,):
            raise ValueError("nb_old and nr need one entry per element")
        Ns, ld_old = _block(X_old, int(nb_old.astype(np.int64).sum()), "X_old")
        for name, V in (("V_old", V_old), ("V_new", V_new)):
            if not (V.is_cuda and V.dtype == torch.float64 and V.is_contiguous()):
                raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
        if V_old.numel() != int((nr.astype(np.int64) * nb_old).sum()) or \
                V_new.numel() != int((nr.astype(np.int64) * self.nb).sum()):
            raise ValueError("V_old / V_new sizes do not match nr x element sizes")
        if X_new is None:
            X_new = torch.empty((Ns, self.N), dtype=torch.float64, device=X_old.device)
        _, ld = _block(X_new, self.N, "X_new")
        self._sync_stream()
        _check(_lib.dgchefsi_realign(self._h, nb_old.ctypes.data, nr.ctypes.data, _ptr(V_old), _ptr(V_new),
                                     _ptr(X_old), Ns, ld_old, _ptr(X_new), ld))
        return X_new

    # -- differentiation of one cycle (band energy)
    def set_values(self, values: torch.Tensor):
        """Replace H's stored values from a float64 CUDA tensor [n_values]."""
        if not (values.is_cuda and values.dtype == torch.float64 and values.is_contiguous()):
            raise TypeError("values must be a contiguous float64 CUDA tensor")
        self._sync_stream()
        _check(_lib.dgchefsi_set_values(self._h, _ptr(values)))

    def energy_grad(self, X: torch.Tensor, m: int, a: float, b: float, a0: float, Ne: float, kT: float,
                    grad: bool = True, stride: int = 0, n_values: int | None = None, prec: str = "f64"):
        """(E, ritz, H_bar, X_bar) of one cycle's band energy; H_bar and X_bar are
        None when grad is False. H_bar is per stored entry (entries independent)."""
        Ns, ld = _block(X, self.N, "X")
        dev = X.device
        ritz = torch.empty(Ns, dtype=torch.float64, device=dev)
        Hb = torch.empty(int(n_values if n_values is not None else self.n_values), dtype=torch.float64,
                         device=dev) if grad else None
        Xb = torch.empty_like(X) if grad else None
        E = C.c_double()
        self._sync_stream()
        _check(_lib.dgchefsi_energy_grad(self._h, PRECISIONS[prec], _ptr(X), Ns, ld, int(m), float(a), float(b), float(a0),
                                         float(Ne), float(kT), int(stride), C.byref(E), _ptr(ritz),
                                         _ptr(Hb) if grad else None, _ptr(Xb) if grad else None))
        return E.value, ritz, Hb, Xb

    def unpack_density(self, P: torch.Tensor):
        o = self.density_offsets
        return [P[o[K]:o[K + 1]].view(int(self.nb[K]), int(self.nb[K])) for K in range(self.M)]

    # -- one full cycle (Alg. 1 + occupations + density), X updated in place
    def cycle(self, X: torch.Tensor, m: int, Ne: float, kT: float, v0: torch.Tensor | None = None,
              prev_ritz=None, bounds=None, prec: str = "f64", k_lanczos: int = 10, out=None):
        Ns, ld = _block(X, self.N, "X")
        dev = X.device
        if out is None:
            out = dict(ritz=torch.empty(Ns, dtype=torch.float64, device=dev),
                       f=torch.empty(Ns, dtype=torch.float64, device=dev),
                       mu=torch.empty(1, dtype=torch.float64, device=dev),
                       P=torch.empty(int(self.density_offsets[-1]), dtype=torch.float64, device=dev))
        bnd = (C.c_double * 3)(*(bounds if bounds is not None else (0.0, 0.0, 0.0)))
        prev = None
        if prev_ritz is not None:
            prev = np.ascontiguousarray(np.asarray(prev_ritz, dtype=np.float64))
        self._sync_stream()
        _check(_lib.dgchefsi_cycle(self._h, PRECISIONS[prec], _ptr(X), Ns, ld, int(m), float(Ne), float(kT),
                                   _ptr(v0) if v0 is not None else None, int(k_lanczos),
                                   prev.ctypes.data if prev is not None else None, bnd,
                                   1 if bounds is not None else 0, _ptr(out["ritz"]), _ptr(out["f"]),
                                   _ptr(out["mu"]), _ptr(out["P"])))
        out["bounds"] = (bnd[0], bnd[1], bnd[2])
        return out


def create(H) -> Context:
    return Context(H)
