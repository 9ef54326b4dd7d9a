"""Adjoint on the GPU (gbt_sum_backward, torch autograd) vs the FP64 oracle's adjoint,
which is itself pinned to central differences (test_oracle_pins).  Bar: 1e-3 relative."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13382_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_2501_13382_gb300 import build, gbt
    build.build()
    gbt.load()
    torch.cuda.init()
    return gbt


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _problem(n_rays=16384, side=40, window=I.WINDOW_SEGMENT, seed=5):
    w = I.diff_city()
    src = I.Source(w.sources[0].pos, n_rays, 6, 1000.0)
    recv = I.receiver_grid(side, 250.0, 1.5)
    freqs = w.freqs
    b = np.array([I.beam_b_rule(n_rays, f) for f in freqs])
    rng = np.random.default_rng(seed)
    gamma = w.scene.gamma.copy()
    gamma[1:] = rng.uniform(0.6, 0.95, gamma.shape[0] - 1).astype(np.float32)
    return w.scene, src, recv, freqs, b, gamma, window


def test_backward_matches_oracle_adjoint(G):
    import torch
    sc0, src, recv, freqs, b, gamma, win = _problem()
    otr = O.trace(sc0, src)
    rng = np.random.default_rng(9)
    wt = (4 * np.pi / src.n_rays) * rng.uniform(0.7, 1.3, src.n_rays)
    wt32 = wt.astype(np.float32)
    po = O.gbs_sum(otr, recv, freqs, b, sc0.c, gamma, weight=wt32.astype(np.float64), window=win)
    g = (rng.normal(size=po.shape) + 1j * rng.normal(size=po.shape)) * np.abs(po).mean()
    dg_o, dw_o, db_o = O.gbs_adjoint(otr, recv, freqs, b, sc0.c, gamma, g,
                                     weight=wt32.astype(np.float64), window=win)
    sc = G.Scene(sc0)
    tr = G.Trace(sc, src)
    r = torch.as_tensor(recv, device="cuda")
    dg, dw, db = G.gbs_sum_backward(tr, r, list(freqs), list(b),
                                    torch.as_tensor(gamma, device="cuda"),
                                    torch.as_tensor(g.astype(np.complex64), device="cuda"),
                                    ray_weight=torch.as_tensor(wt32, device="cuda"),
                                    order=G.recv_order(r), window=win)
    torch.cuda.synchronize()
    G.gbt_sync()
    assert _rel(dg.cpu().numpy(), dg_o) < TOL, (dg.cpu().numpy(), dg_o)
    assert _rel(db.cpu().numpy(), db_o) < TOL, (db.cpu().numpy(), db_o)
    assert _rel(dw.cpu().numpy(), dw_o) < TOL


def test_backward_line_window_open_plane(G):
    import torch
    w = I.open_plane_small()
    otr = O.trace(w.scene, w.sources[0])
    po = O.gbs_sum(otr, w.receivers, w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma, window=1)
    g = np.conj(po) * 3.0 + 0.5j * po
    gamma = np.array([0.7], np.float32)
    dg_o, dw_o, db_o = O.gbs_adjoint(otr, w.receivers, w.freqs, w.beam_b[0], w.scene.c, gamma, g,
                                     window=1)
    sc = G.Scene(w.scene)
    tr = G.Trace(sc, w.sources[0])
    r = torch.as_tensor(w.receivers, device="cuda")
    dg, dw, db = G.gbs_sum_backward(tr, r, list(w.freqs), list(w.beam_b[0]),
                                    torch.as_tensor(gamma, device="cuda"),
                                    torch.as_tensor(g.astype(np.complex64), device="cuda"),
                                    window=1)
    torch.cuda.synchronize()
    assert _rel(dg.cpu().numpy(), dg_o) < TOL
    assert _rel(db.cpu().numpy(), db_o) < TOL
    assert _rel(dw.cpu().numpy(), dw_o) < TOL


@pytest.mark.parametrize("tile_cull", [False, True])
def test_autograd_loss_gradients(G, tile_cull):
    """L = sum |p - p_target|^2 through torch autograd (testing every pair, and with the
    tile pre-cull); gradients vs the oracle adjoint (pinned to central differences)."""
    import torch
    from paper_2501_13382_gb300.autograd import gbs_field
    sc0, src, recv, freqs, b, gamma_t, win = _problem(n_rays=8192, side=32, seed=7)
    gamma0 = np.full_like(gamma_t, 0.8)
    gamma0[0] = 1.0
    otr = O.trace(sc0, src)
    target = O.gbs_sum(otr, recv, freqs, b, sc0.c, gamma_t, window=win)
    sc = G.Scene(sc0)
    tr = G.Trace(sc, src)
    r = torch.as_tensor(recv, device="cuda")
    gam = torch.tensor(gamma0, device="cuda", requires_grad=True)
    bt = torch.tensor(b, device="cuda", dtype=torch.float64, requires_grad=True)
    p = gbs_field(tr, r, freqs, bt, gam, order=G.recv_order(r), window=win, tile_cull=tile_cull)
    tt = torch.as_tensor(target.astype(np.complex64), device="cuda")
    loss = (p - tt).abs().pow(2).sum()
    loss.backward()
    po = O.gbs_sum(otr, recv, freqs, b, sc0.c, gamma0, window=win)
    dg_o, _, db_o = O.gbs_adjoint(otr, recv, freqs, b, sc0.c, gamma0, 2 * (po - target), window=win)
    assert _rel(gam.grad.cpu().numpy(), dg_o) < TOL
    assert _rel(bt.grad.cpu().numpy(), db_o) < TOL
    assert math.isclose(float(loss.detach()), float(np.sum(np.abs(po - target) ** 2)), rel_tol=1e-3)


def test_backward_tile_cull_matches_dense(G):
    import torch
    sc0, src, recv, freqs, b, gamma, win = _problem(n_rays=8192, side=48, seed=12)
    sc = G.Scene(sc0)
    tr = G.Trace(sc, src)
    r = torch.as_tensor(recv, device="cuda")
    rng = np.random.default_rng(4)
    g = torch.as_tensor((rng.normal(size=(len(freqs), recv.shape[0])) +
                         1j * rng.normal(size=(len(freqs), recv.shape[0]))).astype(np.complex64),
                        device="cuda")
    gam = torch.as_tensor(gamma, device="cuda")
    d = G.gbs_sum_backward(tr, r, list(freqs), list(b), gam, g, window=win)
    c = G.gbs_sum_backward(tr, r, list(freqs), list(b), gam, g, window=win, tile_cull=True)
    torch.cuda.synchronize()
    for x, y in zip(d, c):
        assert _rel(y.cpu().numpy(), x.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("nf", [11, 16])
def test_backward_more_than_eight_frequencies(G, nf):
    """The adjoint in frequency groups of at most 8: dL/dgamma, dL/dW and every dL/db_f
    against the oracle's adjoint (frequencies unsorted, b per frequency and uniform)."""
    import torch
    sc0, src, recv, _, _, gamma, win = _problem(n_rays=4096, side=24, seed=nf)
    rng = np.random.default_rng(nf)
    freqs = rng.permutation(125.0 * 2.0 ** (np.arange(nf) / 3.0))
    if nf == 16:
        b = np.full(nf, I.beam_b_rule(src.n_rays, 700.0))
    else:
        b = np.array([I.beam_b_rule(src.n_rays, f) for f in freqs])
    otr = O.trace(sc0, src)
    po = O.gbs_sum(otr, recv, freqs, b, sc0.c, gamma, window=win)
    g = (rng.normal(size=po.shape) + 1j * rng.normal(size=po.shape)) * np.abs(po).mean()
    dg_o, dw_o, db_o = O.gbs_adjoint(otr, recv, freqs, b, sc0.c, gamma, g, window=win)
    sc = G.Scene(sc0)
    tr = G.Trace(sc, src)
    r = torch.as_tensor(recv, device="cuda")
    dg, dw, db = G.gbs_sum_backward(tr, r, list(freqs), list(b),
                                    torch.as_tensor(gamma, device="cuda"),
                                    torch.as_tensor(g.astype(np.complex64), device="cuda"),
                                    order=G.recv_order(r), window=win)
    torch.cuda.synchronize()
    G.gbt_sync()
    assert _rel(dg.cpu().numpy(), dg_o) < TOL
    assert _rel(dw.cpu().numpy(), dw_o) < TOL
    db = db.cpu().numpy()
    for f in range(nf):
        assert abs(db[f] - db_o[f]) < TOL * np.abs(db_o).max(), (f, db[f], db_o[f])


def test_backward_latlong_fan_default_weights(G):
    """Adjoint on the paper's take-off grid with the cells' solid angles as the default
    ray weights: dL/dgamma, dL/dW and dL/db against the oracle's adjoint."""
    import torch
    sc0, _, recv, freqs, b, gamma, win = _problem(n_rays=4096, side=24, seed=21)
    src = I.Source(np.array([0.0, 0.0, 5.0]), 64 * 96, 6, 1000.0, I.FAN_LATLONG, 64)
    b = np.array([I.beam_b_rule(src.n_rays, f) for f in freqs])
    otr = O.trace(sc0, src)
    po = O.gbs_sum(otr, recv, freqs, b, sc0.c, gamma, window=win)
    rng = np.random.default_rng(21)
    g = (rng.normal(size=po.shape) + 1j * rng.normal(size=po.shape)) * np.abs(po).mean()
    dg_o, dw_o, db_o = O.gbs_adjoint(otr, recv, freqs, b, sc0.c, gamma, g, window=win)
    sc = G.Scene(sc0)
    tr = G.Trace(sc, src)
    r = torch.as_tensor(recv, device="cuda")
    dg, dw, db = G.gbs_sum_backward(tr, r, list(freqs), list(b),
                                    torch.as_tensor(gamma, device="cuda"),
                                    torch.as_tensor(g.astype(np.complex64), device="cuda"),
                                    order=G.recv_order(r), window=win)
    torch.cuda.synchronize()
    G.gbt_sync()
    assert _rel(dg.cpu().numpy(), dg_o) < TOL
    assert _rel(db.cpu().numpy(), db_o) < TOL
    assert _rel(dw.cpu().numpy(), dw_o) < TOL


def test_backward_over_an_imported_trace(G):
    """The adjoint over a trace imported from the oracle's segment list (gbt_trace_import)
    against the oracle's adjoint."""
    import torch
    sc0, src, recv, freqs, b, gamma, win = _problem(n_rays=4096, side=20, seed=31)
    otr = O.trace(sc0, src)
    po = O.gbs_sum(otr, recv, freqs, b, sc0.c, gamma, window=win)
    rng = np.random.default_rng(31)
    g = (rng.normal(size=po.shape) + 1j * rng.normal(size=po.shape)) * np.abs(po).mean()
    dg_o, dw_o, db_o = O.gbs_adjoint(otr, recv, freqs, b, sc0.c, gamma, g, window=win)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    seg = {"ray_off": dev(otr.ray_off.astype(np.int32)), "o": dev(otr.o), "t": dev(otr.t),
           "L": dev(otr.L), "s0": dev(otr.s0), "bmat": dev(otr.bmat.astype(np.int32))}
    sc = G.Scene(sc0)
    tr = G.Trace(sc, src, segments=seg)
    r = torch.as_tensor(recv, device="cuda")
    dg, dw, db = G.gbs_sum_backward(tr, r, list(freqs), list(b),
                                    torch.as_tensor(gamma, device="cuda"),
                                    torch.as_tensor(g.astype(np.complex64), device="cuda"),
                                    order=G.recv_order(r), window=win)
    torch.cuda.synchronize()
    G.gbt_sync()
    assert _rel(dg.cpu().numpy(), dg_o) < TOL
    assert _rel(db.cpu().numpy(), db_o) < TOL
    assert _rel(dw.cpu().numpy(), dw_o) < TOL
