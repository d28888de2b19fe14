"""The allocation-free Lanczos bound (dgchefsi_bounds_static) against the
regular one (dgchefsi_bounds), through the C ABI.

It exists for callers that cannot allocate device memory while they run (GPU
memory already reserved by another framework's caching allocator, or loops
that cannot take the device-wide synchronisation of cudaMalloc). Its Krylov
basis lives in a fixed array inside the library, shared by every call, so the
test makes two calls in a row (the second sees the first one's leftovers) and
uses two different problems. Tolerance: the bound's 1e-10 relative parity
used by the other GPU tests (both paths run the same kernels in the same order).
This file is collected last so that a stop at its first failure has already
run every other test."""
import numpy as np
import pytest
import torch

from paper_1606_03416_gb300 import inputs as G

pytestmark = pytest.mark.gpu

D = pytest.importorskip("paper_1606_03416_gb300.dgchefsi") if torch.cuda.is_available() else None


def _bound_pair(ctx, v, k):
    return ctx.bounds(v, k), ctx.bounds_static(v, k)


def _device_memory():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()


@pytest.mark.parametrize("grid,nb,k", [((4, 4, 4), 64, 10), ((2, 2, 2), 32, 6)])
def test_bounds_static_allocates_nothing_and_matches_bounds(grid, nb, k):
    """On a fresh context, with no call of the allocating bound before it: two
    calls in a row leave the device's free memory (cudaMemGetInfo) and torch's
    reserved memory unchanged (the library allocates through the CUDA runtime,
    so the free-memory figure is the one that would move), and both match
    dgchefsi_bounds."""
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=grid, nb=nb, Ns=16)
    H = G.make_blocks(cfg)
    dev = torch.device("cuda:0")
    v = torch.from_numpy(G.make_start_vector(H.N, 7)).to(dev)
    with D.Context(H) as ctx:
        mem0 = _device_memory()
        first = ctx.bounds_static(v, k)
        mem1 = _device_memory()
        second = ctx.bounds_static(v, k)
        mem2 = _device_memory()
        assert mem1 == mem0, f"first call changed (free, reserved) from {mem0} to {mem1}"
        assert mem2 == mem1, f"second call changed (free, reserved) from {mem1} to {mem2}"
        b, t = ctx.bounds(v, k)
        for bs, ts in (first, second):
            assert abs(bs - b) <= 1e-10 * abs(b)
            assert abs(ts - t) <= 1e-10 * max(abs(t), abs(b))
            assert np.isfinite(bs) and bs > ts


@pytest.mark.parametrize("grid,nb,k", [((4, 4, 4), 64, 10), ((2, 2, 2), 32, 6)])
def test_bounds_static_matches_bounds_twice(grid, nb, k):
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=grid, nb=nb, Ns=16)
    H = G.make_blocks(cfg)
    dev = torch.device("cuda:0")
    v = torch.from_numpy(G.make_start_vector(H.N, 7)).to(dev)
    with D.Context(H) as ctx:
        for _ in range(2):
            (b, t), (bs, ts) = _bound_pair(ctx, v, k)
            assert abs(bs - b) <= 1e-10 * abs(b)
            assert abs(ts - t) <= 1e-10 * max(abs(t), abs(b))
            assert np.isfinite(bs) and bs > ts


def test_bounds_static_rejects_oversize_request():
    cfg = G.scaled_copy(G.CONFIGS["bulk3d_8x8x8"], grid=(8, 8, 4), nb=64, Ns=16)
    H = G.make_blocks(cfg)
    assert (64 + 2) * H.N + 72 > D.BOUNDS_STATIC_DOUBLES
    dev = torch.device("cuda:0")
    v = torch.from_numpy(G.make_start_vector(H.N, 1)).to(dev)
    with D.Context(H) as ctx:
        with pytest.raises(D.DGChefsiError) as e:
            ctx.bounds_static(v, 64)
        assert e.value.status == "ERR_ARG" and "fixed scratch" in str(e.value)
        (b, t), (bs, ts) = _bound_pair(ctx, v, 10)     # a size that fits still works
        assert abs(bs - b) <= 1e-10 * abs(b)
