"""Batches (gbt_batch_*, fused persistent and concurrent forms) vs one gbt_sum per
instance, and vs the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13382_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2501_13382_gb300 import build, gbt
    build.build()
    gbt.load()
    torch.cuda.init()
    return gbt


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _batch_setup(G, n_src=6, side=40, seed=44):
    import torch
    w = I.batched_city(n_sources=n_src)
    rng = np.random.default_rng(seed)
    sc = G.Scene(w.scene)
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    insts, srcs = [], []
    for i, s in enumerate(w.sources):
        n = int(rng.integers(1024, 12000))              # uneven ray counts
        src = I.Source(s.pos, n, s.max_reflections, s.max_path)
        recv_np = I.receiver_grid(side + 4 * i, 250.0, 1.5)  # uneven receiver counts
        recv = torch.as_tensor(recv_np, device="cuda")
        freqs = list(w.freqs[i % 3:i % 3 + 3 + (i % 2)])
        b = [I.beam_b_rule(n, f) for f in freqs]
        tr = G.Trace(sc, src)
        insts.append(dict(trace=tr, recv=recv, freqs=freqs, beam_b=b, gamma=gam,
                          order=G.recv_order(recv)))
        srcs.append((src, recv_np, freqs, b))
    return w, sc, gam, insts, srcs


@pytest.mark.parametrize("form,use_graph", [(1, True), (1, False), (2, True), (2, False)])
def test_batch_equals_per_instance_sums(G, form, use_graph):
    """FUSED: one persistent launch over all instances' items (other splits than a
    single sum, so equal up to rounding).  CONCURRENT: the single-sum kernels with
    the single sum's splits on branch streams, so bit-identical."""
    import torch
    w, sc, gam, insts, _ = _batch_setup(G)
    batch = G.Batch(insts, window=w.window, use_graph=use_graph, form=form)
    for rep in range(2):                               # capture, then replay
        batch.submit()
        torch.cuda.synchronize()
        G.gbt_sync()
        for d, out in zip(batch.instances, batch.outputs):
            ref = G.gbs_sum(d["trace"], d["recv"], d["freqs"], d["beam_b"], gam, order=d["order"],
                            window=w.window)
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.complex128)
            ref = ref.cpu().numpy().astype(np.complex128)
            if form == G.BATCH_CONCURRENT:
                assert np.array_equal(got, ref), rep
            else:
                e = rel_l2(got, ref)
                assert e < 1e-6, (rep, e)
    batch.close()


@pytest.mark.parametrize("form", [0, 1, 2])
def test_batch_graph_replay_sees_new_gamma(G, form):
    import torch
    w, sc, gam, insts, srcs = _batch_setup(G, n_src=3, side=32, seed=3)
    batch = G.Batch(insts, window=w.window, use_graph=True, autotune=True, form=form)
    batch.submit()
    torch.cuda.synchronize()
    new_gamma = np.linspace(0.5, 0.99, w.scene.n_materials).astype(np.float32)
    gam.copy_(torch.as_tensor(new_gamma, device="cuda"))   # same buffer, new contents
    batch.submit()
    torch.cuda.synchronize()
    src, recv_np, freqs, b = srcs[1]
    otr = O.trace(w.scene, src)
    po = O.gbs_sum(otr, recv_np, freqs, b, w.scene.c, new_gamma, window=w.window)
    got = batch.outputs[1].cpu().numpy().astype(np.complex128)
    assert rel_l2(got, po) < 1e-4


@pytest.mark.parametrize("form", [1, 2])
def test_batch_with_tile_cull_equals_per_instance_sums(G, form):
    """Both batch forms with the pre-cull (per-instance tile lists in one workspace) against
    one pre-culled gbt_sum per instance."""
    import torch
    w, sc, gam, insts, _ = _batch_setup(G, n_src=4, side=48, seed=8)
    batch = G.Batch(insts, window=w.window, use_graph=True, form=form, tile_cull=True)
    for rep in range(2):
        batch.submit()
        torch.cuda.synchronize()
        G.gbt_sync()
        for d, out in zip(batch.instances, batch.outputs):
            ref = G.gbs_sum(d["trace"], d["recv"], d["freqs"], d["beam_b"], gam, order=d["order"],
                            window=w.window, tile_cull=True)
            torch.cuda.synchronize()
            e = rel_l2(out.cpu().numpy().astype(np.complex128),
                       ref.cpu().numpy().astype(np.complex128))
            assert e < 1e-6, (rep, e)
    batch.close()


@pytest.mark.parametrize("form", [1, 2])
def test_batch_with_latlong_fans_against_oracle(G, form):
    """Instances traced with the paper's take-off grid (cell solid-angle weights, no
    per-ray weights passed) mixed with Fibonacci ones: each batch output against the
    oracle."""
    import torch
    w = I.batched_city(n_sources=4)
    sc = G.Scene(w.scene)
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    recv_np = I.receiver_grid(24, 250.0, 1.5)
    recv = torch.as_tensor(recv_np, device="cuda")
    order = G.recv_order(recv)
    freqs = [500.0, 1000.0]
    insts, srcs = [], []
    for i, s in enumerate(w.sources):
        if i % 2 == 0:
            src = I.Source(s.pos, 48 * 96, s.max_reflections, s.max_path, I.FAN_LATLONG, 48)
        else:
            src = I.Source(s.pos, 4096, s.max_reflections, s.max_path)
        b = [I.beam_b_rule(src.n_rays, f) for f in freqs]
        insts.append(dict(trace=G.Trace(sc, src), recv=recv, freqs=freqs, beam_b=b, gamma=gam,
                          order=order))
        srcs.append((src, b))
    batch = G.Batch(insts, window=w.window, use_graph=True, form=form)
    batch.submit()
    torch.cuda.synchronize()
    G.gbt_sync()
    for (src, b), out in zip(srcs, batch.outputs):
        po = O.gbs_sum(O.trace(w.scene, src), recv_np, freqs, b, w.scene.c, w.scene.gamma,
                       window=w.window)
        assert rel_l2(out.cpu().numpy().astype(np.complex128), po) <= 1e-4
    batch.close()


@pytest.mark.parametrize("form", [1, 2])
def test_batch_instances_with_more_than_eight_frequencies(G, form):
    """Instances of 12 and 16 frequencies next to one of 3: the batch splits them into groups
    of 8 consecutive frequencies; every output row against gbt_sum on the whole instance."""
    import torch
    w, sc, gam, insts, _ = _batch_setup(G, n_src=3, side=32, seed=8)
    rng = np.random.default_rng(8)
    for d, nf in zip(insts, (12, 3, 16)):
        d["freqs"] = list(rng.permutation(125.0 * 2.0 ** (np.arange(nf) / 3.0)))
        d["beam_b"] = [I.beam_b_rule(4096, f) for f in d["freqs"]]
    batch = G.Batch(insts, window=w.window, use_graph=True, form=form)
    batch.submit()
    torch.cuda.synchronize()
    G.gbt_sync()
    for d, out in zip(batch.instances, batch.outputs):
        ref = G.gbs_sum(d["trace"], d["recv"], d["freqs"], d["beam_b"], gam, order=d["order"],
                        window=w.window).cpu().numpy().astype(np.complex128)
        got = out.cpu().numpy().astype(np.complex128)
        assert got.shape == ref.shape
        for f in range(ref.shape[0]):
            assert rel_l2(got[f], ref[f]) < 1e-6, f
    batch.close()
