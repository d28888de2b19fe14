"""The boundary is a plain C ABI. CPU: include/dgchefsi.h compiles as strict
C99, C11 and C++17 on its own. GPU: a C program (tests/c/cycle_from_c.c) that
allocates with the CUDA runtime and calls only the library's entry points runs
one FP64 cycle of the tiny workload and reproduces, bit for bit, the Ritz
values, mu and density trace the Python binding gets from the same calls."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from paper_1606_03416_gb300 import inputs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")


def _cc():
    return shutil.which("gcc") or shutil.which("cc")


@pytest.mark.parametrize("std,compiler", [("c99", "gcc"), ("c11", "gcc"), ("c++17", "g++")])
def test_header_compiles_standalone(tmp_path, std, compiler):
    exe = shutil.which(compiler)
    if exe is None:
        pytest.skip(f"{compiler} not available")
    src = tmp_path / ("h.cpp" if compiler == "g++" else "h.c")
    src.write_text('#include "dgchefsi.h"\nint main(void) { return (int)DGCHEFSI_OK + DGCHEFSI_F64; }\n')
    r = subprocess.run([exe, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only", "-I", INC,
                        str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def write_problem(path, H, X0, v0, Ns, m, Ne, kT):
    with open(path, "wb") as fh:
        np.array([H.nb.shape[0], H.col.shape[0], H.values.shape[0], X0.shape[1], Ns, m], dtype=np.int64).tofile(fh)
        np.asarray(H.nb, dtype=np.int32).tofile(fh)
        np.asarray(H.row_ptr, dtype=np.int64).tofile(fh)
        np.asarray(H.col, dtype=np.int32).tofile(fh)
        np.asarray(H.blk_off, dtype=np.int64).tofile(fh)
        np.asarray(H.values, dtype=np.float64).tofile(fh)
        np.ascontiguousarray(X0, dtype=np.float64).tofile(fh)
        np.asarray(v0, dtype=np.float64).tofile(fh)
        np.array([Ne, kT], dtype=np.float64).tofile(fh)


@pytest.mark.gpu
def test_c_program_matches_python_binding(tmp_path):
    D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi")
    cc = _cc()
    if cc is None:
        pytest.skip("no C compiler")
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc")))
    pkg = os.path.dirname(D._LIBPATH)
    exe = tmp_path / "cycle_from_c"
    r = subprocess.run([cc, "-std=c11", "-O2", os.path.join(ROOT, "tests", "c", "cycle_from_c.c"), "-o", str(exe),
                        "-I", INC, "-I", os.path.join(cuda, "include"), "-L", pkg, "-ldgchefsi",
                        "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{pkg}:{os.path.join(cuda, 'lib64')}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    cfg = G.CONFIGS["tiny_2x2x2"]
    H, X0, v0, Ns, Ne = G.make_problem(cfg)
    prob = tmp_path / "tiny.bin"
    write_problem(prob, H, X0, v0, Ns, cfg.m, Ne, cfg.kT)
    out = subprocess.run([str(exe), str(prob)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    vals = {line.split()[0]: np.array([float(x) for x in line.split()[1:]]) for line in out.stdout.splitlines()}
    dev = torch.device("cuda:0")
    with D.Context(H) as ctx:
        b, tmin = ctx.bounds(torch.from_numpy(v0).to(dev), 10)
        a0, a = tmin, tmin + (b - tmin) * Ns / H.N
        Y = ctx.filter(torch.from_numpy(X0).to(dev), cfg.m, a, b, a0, prec="f64")
        ritz = ctx.rayleigh_ritz(Y)
        f, mu = ctx.occupations(ritz, Ne, cfg.kT)
        P = ctx.density_blocks(Y, f)
        tr = sum(float(torch.trace(p)) for p in ctx.unpack_density(P))
        ritz = ritz.cpu().numpy()
        mu = float(mu.item())
    assert np.array_equal(vals["BOUNDS"], np.array([a, b, a0]))
    assert np.array_equal(vals["RITZ"], ritz)
    assert vals["MU"][0] == mu
    assert abs(vals["TRACE_P"][0] - tr) <= 1e-12 * abs(tr)
