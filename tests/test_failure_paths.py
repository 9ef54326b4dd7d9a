"""Failure detection, all provoked on the host or through a bounded wait:
invalid arguments, a failing allocator, a device wait that runs out."""
import ctypes

import numpy as np
import pytest

from paper_2501_13382_gb300 import gbt as G
from paper_2501_13382_gb300 import inputs as I


@pytest.fixture(scope="module")
def lib():
    import os
    if not os.path.exists(G.LIB_PATH):
        from paper_2501_13382_gb300 import build
        build.build()
    return G.load()


def test_failing_allocator_reports_oom_before_any_launch(lib):
    calls = []
    G.gbt_set_allocator(lambda n, s: calls.append(n) or 0, lambda p, s: None)
    try:
        sc = I._ground_scene(1.0)
        d = G.gbt_scene_desc(343.0, 1, 0, 0.0, 0, 0, 0, 0, 1)
        with pytest.raises(G.GBTError) as e:
            G.gbt_scene_create(d, 0)
        assert e.value.status == 2 and b"allocator" in lib.gbt_last_error()
        assert calls and calls[0] > 0
    finally:
        G.gbt_set_allocator(None)


def test_invalid_scene_rejected_on_host(lib):
    d = G.gbt_scene_desc(-1.0, 1, 0, 0.0, 0, 0, 0, 0, 1)
    with pytest.raises(G.GBTError) as e:
        G.gbt_scene_create(d, 0)
    assert e.value.status == 1 and b"speed of sound" in lib.gbt_last_error()
    tri = np.zeros((1, 9))
    mat = np.array([5], np.int32)
    d = G.gbt_scene_desc(343.0, 0, 0, 0.0, 1, tri.ctypes.data, mat.ctypes.data, 0, 2)
    with pytest.raises(G.GBTError) as e:
        G.gbt_scene_create(d, 0)
    assert e.value.status == 1 and b"tri_material" in lib.gbt_last_error()


def test_unknown_accel_rejected_on_host(lib):
    d = G.gbt_scene_desc(343.0, 1, 0, 0.0, 0, 0, 0, 0, 1, 7)
    with pytest.raises(G.GBTError) as e:
        G.gbt_scene_create(d, 0)
    assert e.value.status == 1 and b"accel" in lib.gbt_last_error()


def test_null_handles_rejected(lib):
    st = lib.gbt_sum(None, None, None)
    assert st == 1
    assert lib.gbt_trace_destroy(None) == 0 and lib.gbt_scene_destroy(None) == 0


def test_unknown_batch_form_rejected_on_host(lib):
    traces = (ctypes.c_void_p * 1)(None)
    args = (G.gbt_sum_args * 1)()
    d = G.gbt_batch_desc(1, ctypes.cast(traces, ctypes.c_void_p).value,
                         ctypes.cast(args, ctypes.c_void_p).value, 1, 0, 7)
    with pytest.raises(G.GBTError) as e:
        G.gbt_batch_create(d, 0)
    assert e.value.status == 1 and b"form" in lib.gbt_last_error()


@pytest.mark.gpu
def test_bounded_device_wait_times_out_and_context_survives(lib):
    import torch
    torch.cuda.init()
    G.gbt_sync()                                # clean state
    G.gbt_selftest_timeout(20000)
    with pytest.raises(G.GBTError) as e:
        G.gbt_sync()
    assert e.value.status == 4                  # GBT_ERR_TIMEOUT
    G.gbt_sync()                                # flag cleared, context fine
    w = I.open_plane_small()
    sc = G.Scene(w.scene)
    tr = G.Trace(sc, w.sources[0])
    r = torch.as_tensor(w.receivers, device="cuda")
    p = G.gbs_sum(tr, r, list(w.freqs), list(w.beam_b[0]), torch.as_tensor(w.scene.gamma, device="cuda"))
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(p)).all()
    G.gbt_sync()


@pytest.mark.gpu
def test_torch_caching_allocator_as_library_allocator(lib):
    import torch
    w = I.open_plane_small()
    r = torch.as_tensor(w.receivers, device="cuda")
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    sc = G.Scene(w.scene)
    ref = G.gbs_sum(G.Trace(sc, w.sources[0]), r, list(w.freqs), list(w.beam_b[0]), gam).cpu()
    G.use_torch_allocator()
    try:
        sc2 = G.Scene(w.scene)
        tr2 = G.Trace(sc2, w.sources[0])
        got = G.gbs_sum(tr2, r, list(w.freqs), list(w.beam_b[0]), gam).cpu()
        torch.cuda.synchronize()
        tr2.close()
        sc2.close()
    finally:
        G.gbt_set_allocator(None)
    assert torch.equal(ref, got)


def test_binding_checks_tensors_before_any_call():
    """The binding rejects tensors the library would read out of bounds or cannot use
    (host tensors, wrong dtypes, gamma or ray_weight of the wrong length) before any
    library call: the C ABI cannot see the sizes of device arrays."""
    import torch
    from types import SimpleNamespace
    tr = SimpleNamespace(scene=SimpleNamespace(n_materials=2), n_fan=8, handle=0)
    recv = torch.zeros(4, 3)
    with pytest.raises(ValueError, match="recv"):
        G.gbs_sum(tr, recv, [500.0], [10.0], torch.ones(2))
    with pytest.raises(ValueError, match="recv"):
        G._check_tensors(torch.zeros(4, 2), torch.ones(2), None, None)
    if not torch.cuda.is_available():
        return
    r = torch.zeros(4, 3, device="cuda")
    with pytest.raises(ValueError, match="gamma must hold 2"):
        G._check_tensors(r, torch.ones(3, device="cuda"), None, None, 2, 8)
    with pytest.raises(ValueError, match="ray_weight must hold 8"):
        G._check_tensors(r, torch.ones(2, device="cuda"), torch.ones(7, device="cuda"), None, 2, 8)
    with pytest.raises(ValueError, match="order"):
        G._check_tensors(r, torch.ones(2, device="cuda"), None,
                         torch.zeros(3, dtype=torch.int32, device="cuda"), 2, 8)


def test_synthesis_rejects_bad_arguments_on_host(lib):
    fr = (ctypes.c_double * 17)(*([500.0] * 17))
    am = (ctypes.c_double * 34)(*([1.0] * 34))
    for nf, n_t in ((0, 10), (17, 10), (4, 0), (4, (1 << 20) + 1)):
        assert lib.gbt_synthesize(None, nf, 0, fr, am, 0.0, 1e-4, n_t, None, 0, None) == 1
    assert lib.gbt_synthesize(None, 4, 10, fr, am, 0.0, 1e-4, 10, None, 0, None) == 1   # NULL p
