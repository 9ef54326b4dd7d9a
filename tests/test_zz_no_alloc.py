"""gbt_recv_order_noalloc: the receiver order without any device allocation.

Some callers cannot allocate device memory when they need the order (a host
that owns every device allocation, or a latency-critical loop that must not
call an allocator); this entry point uses a fixed scratch array inside the
library instead.  The test calls it through the C ABI twice in a row and
checks that it returns exactly the permutation of the allocating entry point
(index work: bit-exact), and that an oversized request is rejected before any
work.  It runs last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2501_13382_gb300 import build, gbt
    build.build()
    lib = gbt.load()
    torch.cuda.init()
    return torch, gbt, lib


def _orders(torch, gbt, lib, recv_np):
    recv = torch.as_tensor(recv_np, device="cuda")
    n = recv.shape[0]
    ref = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    got = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    stream = gbt._stream_ptr()
    gbt.gbt_recv_order(recv.data_ptr(), n, ref.data_ptr(), stream)
    st = lib.gbt_recv_order_noalloc(ctypes.c_void_p(recv.data_ptr()), ctypes.c_int64(n),
                                    ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(stream))
    assert st == 0, lib.gbt_last_error()
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_order_matches_allocating_entry_point_twice(env):
    torch, gbt, lib = env
    rng = np.random.default_rng(2501)
    # two calls in a row: a large set, then a smaller one (the scratch keeps the
    # first call's contents; the second must not see them)
    for n in (300_000, 4097):
        recv = (rng.random((n, 3)) * [1000.0, 700.0, 30.0] - [500.0, 350.0, 0.0]).astype(np.float32)
        ref, got = _orders(torch, gbt, lib, recv)
        assert np.array_equal(got, ref)
        assert np.array_equal(np.sort(got), np.arange(n, dtype=np.int32))
    gbt.gbt_sync()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, gbt, lib = env
    n = (1 << 20) + 1
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    st = lib.gbt_recv_order_noalloc(ctypes.c_void_p(out.data_ptr()), ctypes.c_int64(n),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert st == 1                                   # GBT_ERR_INVALID_ARG, nothing launched
    assert b"1048576" in lib.gbt_last_error()
