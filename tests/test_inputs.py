"""The synthetic input recipe (paper_2501_13382_gb300/inputs.py): sizes, seeds and the
structural properties the workloads are meant to have, so that they cannot drift from
what the documentation states.  Pure data; no GPU, no oracle."""
import math

import numpy as np

from paper_2501_13382_gb300 import inputs as I


def test_workload_sizes():
    w = I.open_plane_small()
    assert w.sources[0].n_rays == 1024 and w.receivers.shape == (64 * 64, 3) and list(w.freqs) == [500.0]
    w = I.open_plane_large()
    assert w.sources[0].n_rays == 65536 and w.receivers.shape == (256 * 256, 3)
    assert np.allclose(w.freqs, 125.0 * 2.0 ** np.arange(6)) and w.scene.n_tri == 0
    w = I.city(n_rays=4096, n_recv_side=16)
    assert w.scene.n_tri == 64 * 12 and w.sources[0].max_reflections == 8
    assert w.scene.n_materials == 65                              # ground + one per building
    w = I.diff_city()
    assert w.sources[0].n_rays == 262144 and w.receivers.shape == (128 * 128, 3)
    assert w.scene.n_materials == 9 and w.extra["target_gamma"].shape == (9,)
    assert np.all((w.extra["target_gamma"][1:] >= 0.6) & (w.extra["target_gamma"][1:] <= 0.95))
    w = I.big_city(n_rays=1024, n_recv_side=8)
    assert w.scene.n_tri == 32 * 32 * 12
    w = I.open_plane_latlong()
    s = w.sources[0]
    assert s.fan == I.FAN_LATLONG and s.n_rays == 128 * 256 and s.n_theta == 128


def test_workloads_are_seeded():
    a, b = I.city(n_rays=1024, n_recv_side=8), I.city(n_rays=1024, n_recv_side=8)
    assert np.array_equal(a.scene.tri_xyz, b.scene.tri_xyz) and np.array_equal(a.scene.gamma, b.scene.gamma)
    a, b = I.batched_city(), I.batched_city()
    assert [s.n_rays for s in a.sources] == [s.n_rays for s in b.sources]


def test_city_buildings_leave_streets_and_the_source_outside():
    tris, faces, bidx, foot, heights, gam = I.synthetic_city(I.SEED_BASE + 3)
    assert np.all((heights >= 10) & (heights <= 60)) and np.all((gam >= 0.7) & (gam <= 0.95))
    side = np.stack([foot[:, 1] - foot[:, 0], foot[:, 3] - foot[:, 2]], 1)
    assert np.all((side >= 20) & (side <= 60))
    # footprints do not overlap and keep streets of at least 2.5 m between neighbours
    for i in range(len(foot)):
        for j in range(i + 1, len(foot)):
            gx = max(foot[j, 0] - foot[i, 1], foot[i, 0] - foot[j, 1])
            gy = max(foot[j, 2] - foot[i, 3], foot[i, 2] - foot[j, 3])
            assert max(gx, gy) >= 2.5 - 1e-9, (i, j)
    # the city source at (0, 0) stands in a street
    assert all(not (f[0] <= 0.0 <= f[1] and f[2] <= 0.0 <= f[3]) for f in foot)


def test_batched_city_sources():
    w = I.batched_city()
    assert len(w.sources) == 32 and len(w.freqs) == 8
    n = np.array([s.n_rays for s in w.sources])
    assert n.min() >= 4096 and n.max() <= 262144
    assert np.log(n).std() > 0.5                                   # log-uniform spread
    foot = w.extra["footprints"]
    for s in w.sources:
        x, y, z = s.pos
        assert 1.0 <= z <= 30.0
        dist = min(math.hypot(max(f[0] - x, 0, x - f[1]), max(f[2] - y, 0, y - f[3])) for f in foot)
        assert dist >= 1.0                                          # in the open streets

