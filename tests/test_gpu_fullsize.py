"""The differentiable-city adjoint and the batched city at their configured sizes against
the FP64 oracle, on seeded receiver samples the oracle evaluates one by one.

* Differentiable city: 262,144 rays, <= 6 reflections, 128 x 128 receivers, 4 bands;
  the loss gradient g is nonzero only on 64 seeded receivers, so the oracle adjoint over
  those receivers is the whole adjoint.  Gradients in gamma, b and every ray weight
  within 1e-3 (the derivatives of Eq. 1 under the uneven per-ray work of Sec. 3.4).
* Batched city: 32 sources (log-uniform 4,096-262,144 rays), 8 bands, 512 x 512
  receivers, with the tile pre-cull; 3 sources x 128 seeded receivers within 1e-4.
"""
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def diff_city_full():
    w = I.diff_city()
    src = w.sources[0]
    otr = O.trace(w.scene, src)
    idx = I.receiver_subset(w.receivers, 64, 91)
    po = O.gbs_sum(otr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                   window=w.window, cutoff=w.cutoff)
    rng = np.random.default_rng(92)
    g_sub = (rng.normal(size=po.shape) + 1j * rng.normal(size=po.shape)) * np.abs(po).mean()
    ref = O.gbs_adjoint(otr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                        g_sub, window=w.window, cutoff=w.cutoff)
    return w, idx, g_sub, ref


@pytest.mark.parametrize("tile_cull", [False, True])
def test_diff_city_backward_at_full_size(G, diff_city_full, tile_cull):
    import torch
    w, idx, g_sub, (dgo, dwo, dbo) = diff_city_full
    nr = w.receivers.shape[0]
    assert w.sources[0].n_rays == 262144 and nr == 128 * 128 and len(w.freqs) == 4
    g = np.zeros((len(w.freqs), nr), np.complex64)
    g[:, idx] = g_sub
    sc = G.Scene(w.scene)
    tr = G.Trace(sc, w.sources[0])
    r = torch.as_tensor(w.receivers, device="cuda")
    dg, dw, db = G.gbs_sum_backward(tr, r, list(w.freqs), list(w.beam_b[0]),
                                    torch.as_tensor(w.scene.gamma, device="cuda"),
                                    torch.as_tensor(g, device="cuda"), order=G.recv_order(r),
                                    window=w.window, cutoff=w.cutoff, tile_cull=tile_cull)
    torch.cuda.synchronize()
    G.gbt_sync()
    assert rel_l2(dg.cpu().numpy(), dgo) < 1e-3, (dg.cpu().numpy(), dgo)
    assert rel_l2(db.cpu().numpy(), dbo) < 1e-3, (db.cpu().numpy(), dbo)
    assert rel_l2(dw.cpu().numpy(), dwo) < 1e-3


@pytest.fixture(scope="module")
def batched_city_full():
    w = I.batched_city()
    picks = [0, 13, 27]
    refs = {}
    for i in picks:
        idx = I.receiver_subset(w.receivers, 128, 100 + i)
        otr = O.trace(w.scene, w.sources[i])
        refs[i] = (idx, O.gbs_sum(otr, w.receivers[idx], w.freqs, w.beam_b[i], w.scene.c,
                                  w.scene.gamma, window=w.window, cutoff=w.cutoff))
    return w, refs


@pytest.mark.parametrize("form", [0, 1])        # GBT_BATCH_AUTO, GBT_BATCH_FUSED
def test_batched_city_at_full_size(G, batched_city_full, form):
    import torch
    w, refs = batched_city_full
    assert len(w.sources) == 32 and w.receivers.shape[0] == 512 * 512 and len(w.freqs) == 8
    sc = G.Scene(w.scene)
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    recv = torch.as_tensor(w.receivers, device="cuda")
    order = G.recv_order(recv)
    insts = [dict(trace=G.Trace(sc, s), recv=recv, freqs=list(w.freqs), beam_b=list(w.beam_b[i]),
                  gamma=gam, order=order) for i, s in enumerate(w.sources)]
    batch = G.Batch(insts, window=w.window, use_graph=True, autotune=False, form=form,
                    tile_cull=True)
    batch.submit()
    torch.cuda.synchronize()
    G.gbt_sync()
    for i, (idx, po) in refs.items():
        pg = batch.outputs[i].cpu().numpy().astype(np.complex128)[:, idx]
        for f in range(len(w.freqs)):
            assert rel_l2(pg[f], po[f]) < 1e-4, (i, f, rel_l2(pg[f], po[f]))
    batch.close()
