"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point the header declares, and rejects malformed
block-sparse input before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_03416_gb300 import build as B
    path = B.build()
    return C.CDLL(path)


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dgchefsi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dgchefsi_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "dgchefsi_filter" in names and "dgchefsi_cycle" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_exports_match_header():
    from paper_1606_03416_gb300 import dgchefsi as D
    assert sorted(D.EXPORTS) == declared_symbols()


def _create(lib, nb, row_ptr, col, blk_off, values):
    nb = np.ascontiguousarray(nb, dtype=np.int32)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    blk_off = np.ascontiguousarray(blk_off, dtype=np.int64)
    values = np.ascontiguousarray(values, dtype=np.float64)
    out = C.c_void_p()
    f = lib.dgchefsi_create
    f.restype = C.c_int
    st = f(C.c_int32(len(nb)), C.c_void_p(nb.ctypes.data), C.c_void_p(row_ptr.ctypes.data),
           C.c_void_p(col.ctypes.data), C.c_void_p(blk_off.ctypes.data), C.c_void_p(values.ctypes.data),
           C.c_int64(len(values)), None, C.byref(out))
    lib.dgchefsi_last_error.restype = C.c_char_p
    return st, lib.dgchefsi_last_error().decode()


def two_element(sym=True):
    A = np.arange(4.0).reshape(2, 2)
    d = np.array([[1.0, 0.5], [0.5, 2.0]])
    B = A.T.copy() if sym else A.copy()
    vals = np.concatenate([d.ravel(), A.ravel(), B.ravel(), d.ravel()])
    return [2, 2], [0, 2, 4], [0, 1, 0, 1], [0, 4, 8, 12], vals


def test_create_rejects_asymmetric_blocks(lib):
    st, msg = _create(lib, *two_element(sym=False))
    assert st == 1 and "symmetric" in msg


def test_create_rejects_bad_structure(lib):
    nb, rp, col, off, vals = two_element()
    assert _create(lib, nb, [0, 2, 3], [0, 1, 0], off[:3], vals)[0] == 1           # pattern asymmetric
    assert _create(lib, nb, rp, [1, 0, 0, 1], off, vals)[0] == 1                   # unsorted row
    assert _create(lib, nb, [0, 1, 2], [1, 0], [4, 8], vals)[0] == 1               # no diagonal block
    assert _create(lib, nb, rp, col, [0, 4, 8, 14], vals)[0] == 1                  # block outside values
    bad = vals.copy()
    bad[0] = np.nan
    assert _create(lib, nb, rp, col, off, bad)[0] == 1                             # non-finite value
    assert _create(lib, [0, 2], rp, col, off, vals)[0] == 1                        # empty element
