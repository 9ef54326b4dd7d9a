"""Propagation losses on the GPU against the FP64 oracle: air absorption (ISO 9613-1 rate,
exp(-a s) over the unfolded arclength) and porous surfaces (Delany-Bazley impedance,
plane-wave reflection factor at each reflection's incidence), as the oracle defines them
for the atmosphere and flow-impedance settings of the paper's Sec. 4.5 (Tables 2-3).

Bars as for the lossless path: fields within relative L2 1e-4 (F32) and 1e-6 (F64) of the
oracle, gradients within 1e-3."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13382_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-4


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


def _dev(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)


def _lossy_open_plane(n_rays=16384, n_side=48, freqs=(125.0, 250.0, 500.0, 1000.0, 2000.0, 4000.0)):
    """Ground with the flow resistivity of grass (200 kPa s m^-2) under a source at 2 m, the
    paper's atmosphere (20 C, 70 %, 1 atm)."""
    sc = I.Scene(343.0, True, 0.0, 0, np.zeros((0, 3, 3)), np.zeros(0, np.int32),
                 np.zeros(0, np.int32), np.array([0.95], np.float32))
    src = I.Source(np.array([0.0, 0.0, 2.0]), n_rays, 3, 1000.0)
    recv = I.receiver_grid(n_side, 400.0, 1.5)
    freqs = np.array(freqs)
    b = np.array([I.beam_b_rule(n_rays, f) for f in freqs])
    return sc, src, recv, freqs, b, np.array([200.0])


def _lossy_city(n_rays=16384, n_side=40, freqs=(250.0, 1000.0)):
    """The synthetic city with a porous ground, hard buildings except every third one
    (porous, 50 kPa s m^-2), and the paper's atmosphere."""
    sc, _ = I.city_scene(I.SEED_BASE + 3)
    src = I.Source(np.array([0.0, 0.0, 5.0]), n_rays, 6, 1000.0)
    recv = I.receiver_grid(n_side, 250.0, 1.5)
    freqs = np.array(freqs)
    b = np.array([I.beam_b_rule(n_rays, f) for f in freqs])
    sigma = np.full(sc.n_materials, -10.0)
    sigma[0] = 200.0
    sigma[1::3] = 50.0
    return sc, src, recv, freqs, b, sigma


def _run(G, sc, src, recv, freqs, b, sigma, absorb, window, precision=0, tile_cull=False,
         order=True, seg_split=0):
    import torch
    gsc = G.Scene(sc)
    tr = G.Trace(gsc, src)
    r = _dev(recv, torch.float32)
    p = G.gbs_sum(tr, r, list(freqs), list(b), _dev(sc.gamma, torch.float32),
                  order=G.recv_order(r) if order else None, window=window,
                  precision=precision, tile_cull=tile_cull, seg_split=seg_split,
                  absorption=None if absorb is None else list(absorb),
                  flow_resistivity=None if sigma is None else _dev(sigma, torch.float32))
    torch.cuda.synchronize()
    G.gbt_sync()
    return p.cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def open_plane_case():
    sc, src, recv, freqs, b, sigma = _lossy_open_plane()
    absorb = O.air_absorption(freqs, 20.0, 70.0, 101.325)
    tr = O.trace(sc, src)
    po = O.gbs_sum(tr, recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_LINE, absorption=absorb,
                   sigma=sigma, scene=sc)
    p0 = O.gbs_sum(tr, recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_LINE)
    return sc, src, recv, freqs, b, sigma, absorb, po, p0


@pytest.mark.parametrize("tile_cull", [False, True])
def test_open_plane_porous_ground_and_absorption_f32(G, open_plane_case, tile_cull):
    sc, src, recv, freqs, b, sigma, absorb, po, p0 = open_plane_case
    assert rel_l2(p0, po) > 0.1            # the losses matter here
    pg = _run(G, sc, src, recv, freqs, b, sigma, absorb, I.WINDOW_LINE, tile_cull=tile_cull)
    for f in range(len(freqs)):
        assert rel_l2(pg[f], po[f]) < TOL_L2, (f, rel_l2(pg[f], po[f]))


def test_open_plane_losses_f64_path(G, open_plane_case):
    sc, src, recv, freqs, b, sigma, absorb, po, p0 = open_plane_case
    pg = _run(G, sc, src, recv, freqs, b, sigma, absorb, I.WINDOW_LINE, precision=1)
    assert rel_l2(pg, po) < 1e-6


@pytest.mark.parametrize("only", ["absorption", "porous"])
def test_each_loss_alone(G, open_plane_case, only):
    sc, src, recv, freqs, b, sigma, absorb, _, _ = open_plane_case
    a = absorb if only == "absorption" else None
    s = sigma if only == "porous" else None
    po = O.gbs_sum(O.trace(sc, src), recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_LINE,
                   absorption=a, sigma=s, scene=sc)
    pg = _run(G, sc, src, recv, freqs, b, s, a, I.WINDOW_LINE)
    assert rel_l2(pg, po) < TOL_L2


@pytest.fixture(scope="module")
def city_case():
    sc, src, recv, freqs, b, sigma = _lossy_city()
    absorb = O.air_absorption(freqs, 20.0, 70.0, 101.325)
    tr = O.trace(sc, src)
    po = O.gbs_sum(tr, recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_SEGMENT,
                   absorption=absorb, sigma=sigma, scene=sc)
    return sc, src, recv, freqs, b, sigma, absorb, tr, po


@pytest.mark.parametrize("tile_cull,seg_split", [(False, 0), (True, 0), (False, 7)])
def test_city_porous_surfaces_against_oracle(G, city_case, tile_cull, seg_split):
    sc, src, recv, freqs, b, sigma, absorb, tr, po = city_case
    pg = _run(G, sc, src, recv, freqs, b, sigma, absorb, I.WINDOW_SEGMENT, tile_cull=tile_cull,
              seg_split=seg_split)
    for f in range(len(freqs)):
        assert rel_l2(pg[f], po[f]) < TOL_L2, (f, rel_l2(pg[f], po[f]))


def test_city_losses_f64_path(G, city_case):
    sc, src, recv, freqs, b, sigma, absorb, tr, po = city_case
    pg = _run(G, sc, src, recv, freqs, b, sigma, absorb, I.WINDOW_SEGMENT, precision=1)
    assert rel_l2(pg, po) < 1e-6


def test_losses_with_more_than_eight_frequencies(G):
    """Twelve bands (two pair launches) with absorption and a porous ground."""
    freqs = tuple(125.0 * 2.0 ** (i / 2.0) for i in range(12))
    sc, src, recv, freqs, b, sigma = _lossy_open_plane(n_rays=8192, n_side=24, freqs=freqs)
    absorb = O.air_absorption(freqs, 10.0, 40.0, 95.0)
    po = O.gbs_sum(O.trace(sc, src), recv, freqs, b, sc.c, sc.gamma, window=I.WINDOW_LINE,
                   absorption=absorb, sigma=sigma, scene=sc)
    pg = _run(G, sc, src, recv, freqs, b, sigma, absorb, I.WINDOW_LINE)
    for f in range(len(freqs)):
        assert rel_l2(pg[f], po[f]) < TOL_L2, (f, rel_l2(pg[f], po[f]))


def test_adjoint_with_losses_against_oracle(G, city_case):
    import torch
    sc, src, recv, freqs, b, sigma, absorb, tr, po = city_case
    rng = np.random.default_rng(11)
    g = (rng.normal(size=po.shape) + 1j * rng.normal(size=po.shape)) * 1e3
    gsc = G.Scene(sc)
    gtr = G.Trace(gsc, src)
    r = _dev(recv, torch.float32)
    for cull in (False, True):
        dg, dw, db = G.gbs_sum_backward(gtr, r, list(freqs), list(b),
                                        _dev(sc.gamma, torch.float32),
                                        _dev(g.astype(np.complex64)), order=G.recv_order(r),
                                        window=I.WINDOW_SEGMENT, tile_cull=cull,
                                        absorption=list(absorb),
                                        flow_resistivity=_dev(sigma, torch.float32))
        torch.cuda.synchronize()
        G.gbt_sync()
        dgo, dwo, dbo = O.gbs_adjoint(tr, recv, freqs, b, sc.c, sc.gamma, g,
                                      window=I.WINDOW_SEGMENT, absorption=absorb, sigma=sigma,
                                      scene=sc)
        assert rel_l2(dg.cpu().numpy(), dgo) < 1e-3
        assert rel_l2(dw.cpu().numpy(), dwo) < 1e-3
        assert rel_l2(db.cpu().numpy(), dbo) < 1e-3


def test_chunked_solve_with_losses_equals_one_pass(G):
    import torch
    sc, src, recv, freqs, b, sigma = _lossy_city(n_rays=8192, n_side=24)
    absorb = O.air_absorption(freqs)
    gsc = G.Scene(sc)
    r = _dev(recv, torch.float32)
    gam = _dev(sc.gamma, torch.float32)
    sg = _dev(sigma, torch.float32)
    kw = dict(order=G.recv_order(r), window=I.WINDOW_SEGMENT, absorption=list(absorb),
              flow_resistivity=sg)
    one = G.gbs_solve(gsc, src, r, list(freqs), list(b), gam, **kw)
    many = G.gbs_solve(gsc, src, r, list(freqs), list(b), gam, max_device_bytes=2 << 20, **kw)
    torch.cuda.synchronize()
    G.gbt_sync()
    assert rel_l2(many.cpu().numpy(), one.cpu().numpy()) < 1e-6


def test_batch_with_losses_runs_concurrent_and_matches_single_sums(G):
    import torch
    sc, src, recv, freqs, b, sigma = _lossy_city(n_rays=8192, n_side=24)
    gsc = G.Scene(sc)
    r = _dev(recv, torch.float32)
    gam = _dev(sc.gamma, torch.float32)
    order = G.recv_order(r)
    sg = _dev(sigma, torch.float32)
    insts = []
    for k, pos in enumerate(([0.0, 0.0, 5.0], [62.5, -62.5, 12.0])):    # street corners
        s = I.Source(np.array(pos), 8192 >> k, 5, 1000.0)
        insts.append(dict(trace=G.Trace(gsc, s), recv=r, freqs=list(freqs), beam_b=list(b),
                          gamma=gam, order=order, absorption=list(O.air_absorption(freqs)),
                          flow_resistivity=sg))
    ref = [G.gbs_sum(d["trace"], r, d["freqs"], d["beam_b"], gam, order=order,
                     window=I.WINDOW_SEGMENT, absorption=d["absorption"], flow_resistivity=sg)
           for d in insts]
    batch = G.Batch(insts, window=I.WINDOW_SEGMENT, use_graph=True, autotune=True)
    batch.submit()
    batch.submit()
    torch.cuda.synchronize()
    G.gbt_sync()
    for a, o in zip(batch.outputs, ref):
        assert torch.equal(a, o)
    batch.close()
    with pytest.raises(G.GBTError) as e:
        G.Batch(insts, window=I.WINDOW_SEGMENT, form=G.BATCH_FUSED)
    assert e.value.status == 6                      # GBT_ERR_UNSUPPORTED


def test_invalid_absorption_is_rejected(G):
    import torch
    sc, src, recv, freqs, b, sigma = _lossy_open_plane(n_rays=1024, n_side=4)
    gsc = G.Scene(sc)
    tr = G.Trace(gsc, src)
    r = _dev(recv, torch.float32)
    with pytest.raises(G.GBTError):
        G.gbs_sum(tr, r, list(freqs), list(b), _dev(sc.gamma, torch.float32),
                  absorption=[-0.1] * len(freqs))
    with pytest.raises(ValueError):
        G.gbs_sum(tr, r, list(freqs), list(b), _dev(sc.gamma, torch.float32),
                  flow_resistivity=_dev(np.array([1.0, 2.0]), torch.float32))
