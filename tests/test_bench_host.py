"""Host logic of bench.py (no GPU): the algorithmic flop and byte counts the
roofline uses, checked against the workload's stated figures, and the lookup
of profiled DRAM traffic, which must return a number only for a summary taken
on the current kernel source and the right layout."""
import importlib.util
import os
import sys

import pytest

from paper_1606_03416_gb300 import inputs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


@pytest.fixture(scope="module")
def bulk():
    cfg = G.CONFIGS["bulk3d_8x8x8"]
    return cfg, G.make_blocks(cfg)


def test_filter_flops_match_workload_figures(bench, bulk):
    cfg, H = bulk
    # 2 * 27 blocks of 64 x 64 per element * 512 elements * N_s per mat-vec: 4.64e11; m = 20 steps
    assert bench.filter_flops(H, cfg.Ns, 1) == 2.0 * 27 * 64 * 64 * 512 * 4096
    assert abs(bench.filter_flops(H, cfg.Ns, cfg.m) - 9.28e12) / 9.28e12 < 1e-3


def test_filter_bytes_per_step(bench, bulk):
    cfg, H = bulk
    N, Ns = H.N, cfg.Ns
    # BF16: read BF16 Y_k and FP32 Y_{k-1}, write FP32 Y_{k+1} and its BF16 copy, read BF16 H
    assert abs(bench.filter_bytes_per_step(H, Ns, "bf16") - 1.72e9) / 1.72e9 < 0.01
    assert bench.filter_bytes_per_step(H, Ns, "bf16x3") > bench.filter_bytes_per_step(H, Ns, "bf16")
    assert bench.filter_bytes_per_step(H, Ns, "f64") == 8.0 * N * Ns * 3 + 8.0 * H.values.shape[0]


def test_profiled_traffic_keyed_on_source_and_layout(bench):
    t = bench.profiled_traffic("bf16x3", 4096, 2)
    if t is not None:  # present only while the summary matches the kernel source
        assert t > bench.filter_bytes_per_step(G.make_blocks(G.CONFIGS["bulk3d_8x8x8"]), 4096, "bf16x3") * 0.5
        assert bench.profiled_traffic("bf16x3", 2048, 2) == pytest.approx(t / 2)
    assert bench.profiled_traffic("bf16x3", 4096, 0) is None   # no summary for layout 0 on this source
    assert bench.profiled_traffic("tf32", 4096, 1) is None


def test_profiled_gram_traffic_exact_size_only(bench):
    assert bench.profiled_gram_traffic(1234) is None
    t = bench.profiled_gram_traffic(4096)
    assert t is None or t > 1e9
