"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with an
independent statement (closed forms, the matrix form of Eq. 1 / Eq. 2, the
exact image construction, a different intersection algorithm, finite
differences, hand-traced geometry).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13382_gb300 import inputs as I

C = 343.0


def _scene(ground=False, gamma=1.0, tris=None, faces=None, mats=None, gammas=None):
    tris = np.zeros((0, 3, 3)) if tris is None else np.asarray(tris, np.float64)
    nt = tris.shape[0]
    faces = np.arange(nt, dtype=np.int32) if faces is None else np.asarray(faces, np.int32)
    mats = np.zeros(nt, np.int32) if mats is None else np.asarray(mats, np.int32)
    gam = np.array([gamma] if gammas is None else gammas, np.float32)
    return I.Scene(C, ground, 0.0, 0, tris, mats, faces, gam)


def _one_segment_trace(o, t, L=1e4, s0=0.0):
    return O.Trace(1, np.array([0, 1]), np.array([1], np.int32), np.array([o], float),
                   np.array([t], float), np.array([L]), np.array([s0]), np.array([0], np.int32),
                   np.array([0], np.int32), np.array([-1], np.int32), np.array([-1], np.int32))


# ----------------------------------------------------------------- fan --

def test_fan_fibonacci_properties():
    n = 4096
    d = O.fan_fibonacci(n)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    # equal-area bands in z: z_i = 1 - (2i+1)/n
    assert np.allclose(d[:, 2], 1.0 - (2.0 * np.arange(n) + 1.0) / n, atol=0, rtol=0)
    # balanced: centroid of a uniform sphere sampling ~ 0
    assert np.linalg.norm(d.mean(axis=0)) < 2.0 / n
    # nearest-neighbour spacing close to the mean angular spacing sqrt(4 pi / n)
    sub = d[::37]
    cosang = np.clip(sub @ d.T, -1, 1)
    cosang[cosang > 1 - 1e-15] = -2
    nn = np.arccos(cosang.max(axis=1))
    dth = math.sqrt(4 * math.pi / n)
    assert 0.6 * dth < nn.min() and nn.max() < 1.3 * dth


@pytest.mark.parametrize("nt,nph,th,ph", [(16, 32, (0.0, 180.0), (0.0, 360.0)),
                                          (7, 5, (30.0, 150.0), (10.0, 100.0)),
                                          (1, 1, (80.0, 100.0), (0.0, 360.0))])
def test_fan_latlong_cells(nt, nph, th, ph):
    """Take-off grid of elevation x azimuth angles: each ray at its cell's centre,
    theta-major, weighted by the cell's solid angle (checked by quadrature of sin(theta),
    not by the closed form the oracle uses), the weights adding up to the solid angle of
    the whole range."""
    from scipy.integrate import quad
    d, w = O.fan_latlong(nt, nph, th, ph)
    assert d.shape == (nt * nph, 3) and w.shape == (nt * nph,)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    rad = math.pi / 180.0
    dth, dph = (th[1] - th[0]) / nt, (ph[1] - ph[0]) / nph
    it, ip = np.divmod(np.arange(nt * nph), nph)
    theta = np.arccos(np.clip(d[:, 2], -1, 1)) / rad
    phi = np.mod(np.arctan2(d[:, 1], d[:, 0]) / rad - ph[0], 360.0) + ph[0]
    assert np.allclose(theta, th[0] + (it + 0.5) * dth, atol=1e-9)
    assert np.allclose(phi, ph[0] + (ip + 0.5) * dph, atol=1e-9)
    for g in range(0, nt * nph, max(1, nph // 2)):
        lo = (th[0] + it[g] * dth) * rad
        cell = quad(math.sin, lo, lo + dth * rad, epsabs=0, epsrel=1e-13)[0] * dph * rad
        assert math.isclose(w[g], cell, rel_tol=1e-12), g
    total = (ph[1] - ph[0]) * rad * (math.cos(th[0] * rad) - math.cos(th[1] * rad))
    assert math.isclose(w.sum(), total, rel_tol=1e-13)


def test_fan_latlong_full_sphere_is_balanced():
    d, w = O.fan_latlong(64, 128)
    assert math.isclose(w.sum(), 4 * math.pi, rel_tol=1e-13)
    # the solid-angle-weighted mean direction of a full sphere vanishes, and the weighted
    # second moment is isotropic: integral of d d^T over the sphere = (4 pi / 3) I
    assert np.linalg.norm((w[:, None] * d).sum(0)) < 1e-12
    m2 = (w[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0)
    assert np.allclose(m2, 4 * math.pi / 3 * np.eye(3), atol=2e-3)


def test_free_field_point_source_latlong_fan():
    """The paper's take-off grid with cell weights reproduces exp(ikr)/(4 pi r) with the
    same paraxial residual law as the Fibonacci fan away from the poles.  Near a pole
    the beams' Gaussian reaches across theta = 0, where the integrand over theta does not
    vanish, so the grid keeps the midpoint rule's endpoint error: it falls as dtheta^2
    (a factor 4 per halving)."""
    f, b = 500.0, 70.0
    k = 2 * math.pi * f / C
    rng = np.random.default_rng(7)
    dirs = rng.normal(size=(6, 3))
    dirs = dirs[np.abs(dirs[:, 2]) < 0.8 * np.linalg.norm(dirs, axis=1)]
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pole = np.array([[0.05, 0.0, 0.99875], [0.0, 0.0, 1.0]])
    pole /= np.linalg.norm(pole, axis=1, keepdims=True)

    def resid(tr, d, r):
        recv = (d * r).astype(np.float32)
        rr = np.linalg.norm(recv.astype(float), axis=1)
        p = O.gbs_sum(tr, recv, [f], [b], C, [1.0], window=1)[0]
        law = 1j * rr / (k * b * b)
        return p / (np.exp(1j * k * rr) / (4 * math.pi * rr)) - 1 - law, law

    errs = []
    for nt in (64, 128, 256):
        tr = O.trace(_scene(), I.Source(np.zeros(3), nt * 2 * nt, 0, 1e4, I.FAN_LATLONG, nt))
        if nt == 128:
            for r in (40.0, 120.0, 300.0):
                res, law = resid(tr, dirs, r)
                assert np.all(np.abs(res) <= 0.05 * np.abs(law) + np.abs(law) ** 2 + 2e-5), r
        errs.append(np.abs(resid(tr, pole, 40.0)[0]))
    for coarse, fine in zip(errs[:-1], errs[1:]):
        assert np.all((3.5 < coarse / fine) & (coarse / fine < 4.6)), coarse / fine


# --------------------------------------------------------------- trace --

def test_trace_ground_plane_is_image_construction():
    sc = _scene(ground=True)
    src = I.Source(np.array([3.0, -2.0, 2.0]), 2048, 2, 200.0)
    tr = O.trace(sc, src)
    d = O.fan_fibonacci(2048)
    for i in range(2048):
        a, b = tr.ray_off[i], tr.ray_off[i + 1]
        if d[i, 2] >= 0 or (-2.0 / d[i, 2]) >= 200.0:
            assert b - a == 1 and tr.hit[a] == -1 and tr.L[a] == 200.0
            continue
        assert b - a == 2
        assert tr.hit[a] == 0 and tr.hit[a + 1] == -1
        assert math.isclose(tr.L[a], -2.0 / d[i, 2], rel_tol=1e-15)
        # reflected direction is the mirror image, exactly
        assert np.array_equal(tr.t[a + 1], d[i] * [1, 1, -1])
        assert abs(tr.o[a + 1, 2]) < 1e-13
        # unfolding the reflected segment back by s0 reaches the image source
        img = tr.o[a + 1] - tr.s0[a + 1] * tr.t[a + 1]
        assert np.allclose(img, [3.0, -2.0, -2.0], atol=1e-12)
        assert math.isclose(tr.L[a] + tr.L[a + 1], 200.0, rel_tol=1e-14)


def _box(x0, x1, y0, y1, h, base_face=0):
    t, f = I.box_triangles(x0, x1, y0, y1, h)
    return t, f + base_face


def test_trace_box_hand_cases():
    # corridor between two boxes: walls at x = -10 and x = +10
    ta, fa = _box(-20, -10, -50, 50, 40, 0)
    tb, fb = _box(10, 20, -50, 50, 40, 6)
    tris = np.concatenate([ta, tb])
    faces = np.concatenate([fa, fb])
    mats = np.array([1] * 12 + [2] * 12, np.int32)
    sc = _scene(ground=True, tris=tris, faces=faces, mats=mats, gammas=[1.0, 0.5, 0.7])
    src = I.Source(np.array([0.0, 0.0, 5.0]), 1, 3, 500.0)
    tr = O.trace(sc, src, dirs=np.array([[1.0, 0.0, 0.0]]))
    # +x: 10 to the right wall, then 20, 20, 20 across; the 4th hit ends the ray (R = 3)
    assert tr.n_seg == 4
    assert np.allclose(tr.L, [10, 20, 20, 20]) and np.allclose(tr.s0, [0, 10, 30, 50])
    assert np.allclose(tr.t[:, 0], [1, -1, 1, -1])
    hit_face = faces[tr.hit - 1]
    assert list(hit_face) == [6, 1, 6, 1]               # box B face x=x0, box A face x=x1
    assert list(tr.bmat) == [-1, 2, 1, 2]
    # 45 degrees down: ground at (5,0,0), wall x=10 at (10,0,5), wall x=-10 at (-10,0,25),
    # then it passes over box B (height 40) and runs free to the path limit
    s2 = math.sqrt(2.0)
    tr = O.trace(sc, I.Source(np.array([0.0, 0.0, 5.0]), 1, 3, 100.0),
                 dirs=np.array([[1 / s2, 0.0, -1 / s2]]))
    assert tr.n_seg == 4
    assert tr.hit[0] == 0 and tr.hit[3] == -1
    assert faces[tr.hit[1] - 1] == 6 and faces[tr.hit[2] - 1] == 1
    assert np.allclose(tr.o[1:], [[5, 0, 0], [10, 0, 5], [-10, 0, 25]], atol=1e-12)
    assert np.allclose(tr.s0, [0, 5 * s2, 10 * s2, 30 * s2], rtol=1e-14)
    assert math.isclose(tr.s0[3] + tr.L[3], 100.0, rel_tol=1e-14)
    assert np.allclose(tr.t[3], [1 / s2, 0, 1 / s2])
    assert list(tr.bmat) == [-1, 0, 2, 1]


def _independent_nearest_hit(o, d, tris, faces, last_face, ground, tmin=1e-9):
    """Plane intersection + same-side point-in-triangle test (not Moller-Trumbore)."""
    best_t, best = np.inf, []
    cands = []
    if ground and last_face != -2 and d[2] != 0:
        t = -o[2] / d[2]
        if t > tmin:
            cands.append((t, 0))
    for k in range(tris.shape[0]):
        if faces[k] == last_face:
            continue
        v0, v1, v2 = tris[k]
        n = np.cross(v1 - v0, v2 - v0)
        den = n @ d
        if den == 0:
            continue
        t = (n @ (v0 - o)) / den
        if t <= tmin:
            continue
        p = o + t * d
        ok = True
        for a, b in ((v0, v1), (v1, v2), (v2, v0)):
            if np.cross(b - a, p - a) @ n < -1e-9 * np.linalg.norm(n) * np.linalg.norm(b - a):
                ok = False
        if ok:
            cands.append((t, k + 1))
    if not cands:
        return np.inf, []
    tb = min(c[0] for c in cands)
    return tb, [c[1] for c in cands if abs(c[0] - tb) <= 1e-9 * max(1.0, tb)]


def test_trace_city_against_independent_intersection():
    sc, _ = I.city_scene(I.SEED_BASE + 3)
    src = I.Source(np.array([0.0, 0.0, 5.0]), 96, 6, 600.0)
    tr = O.trace(sc, src)
    tris = sc.tri_xyz
    faces = sc.tri_face
    for i in range(src.n_rays):
        a, b = tr.ray_off[i], tr.ray_off[i + 1]
        last = -1
        for j in range(a, b):
            o, d = tr.o[j], tr.t[j]
            tb, hits = _independent_nearest_hit(o, d, tris, faces, last, True)
            remaining = 600.0 - tr.s0[j]
            if tr.hit[j] == -1:
                assert not hits or tb >= remaining * (1 - 1e-12)
                assert math.isclose(tr.L[j], remaining, rel_tol=1e-12)
            else:
                assert tr.hit[j] in hits and tr.hit[j] == min(hits)
                assert math.isclose(tr.L[j], tb, rel_tol=1e-9, abs_tol=1e-9)
                # chain continuity and the law of reflection
                if j + 1 < b:
                    assert np.allclose(tr.o[j + 1], o + tr.L[j] * d, atol=1e-9)
                    if tr.hit[j] == 0:
                        n = np.array([0.0, 0.0, 1.0])
                        last = -2
                    else:
                        v0, v1, v2 = tris[tr.hit[j] - 1]
                        n = np.cross(v1 - v0, v2 - v0)
                        n /= np.linalg.norm(n)
                        last = faces[tr.hit[j] - 1]
                    assert np.allclose(tr.t[j + 1], d - 2 * (d @ n) * n, atol=1e-14)
                    assert tr.bmat[j + 1] == (0 if tr.hit[j] == 0 else sc.tri_material[tr.hit[j] - 1])
        assert b - a <= src.max_reflections + 1
        assert tr.L[a:b].sum() <= 600.0 * (1 + 1e-12)


# ------------------------------------------------------- beam summand --

def _eq1_matrix_form(x, o, t, s0, k, b, W, Gam):
    """Eq. 1 evaluated literally with 2x2 matrices, Q from Eq. 2 (dQ/ds = c P).

    P = I / c (constant), Q(s) = Q0 + c P s with Q0 = -i b I; amplitude
    A0 sqrt(det Q0 / det Q) (branch continuous from 1 at s = 0); weighting
    constant Phi = i k W / (8 pi^2)."""
    t = np.asarray(t, float)
    a = np.array([1.0, 0.0, 0.0]) if abs(t[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(t, a); e1 /= np.linalg.norm(e1)
    e2 = np.cross(t, e1)
    dx = np.asarray(x, float) - o
    q = np.array([dx @ e1, dx @ e2])
    s = s0 + dx @ t
    P = np.eye(2) / C
    Q0 = -1j * b * np.eye(2)
    Q = Q0 + C * P * s
    ratio = np.linalg.det(Q0) / np.linalg.det(Q)
    amp = np.sqrt(ratio + 0j)
    assert amp.real > 0       # principal branch is the continuous one for s >= 0
    omega = k * C
    phase = 1j * k * s + 0.5j * omega * (q @ P @ np.linalg.inv(Q) @ q)
    Phi = 1j * k * W / (8 * math.pi ** 2)
    return Phi * Gam * amp * np.exp(phase)


def _brute_force_mismatches():
    """Eq. 3 as a plain triple loop on a tiny traced scene (8 rays off a box and the ground,
    12 receivers, 2 frequencies, per-ray weights, two materials): every (receiver,
    segment, frequency) term from the matrix form of Eq. 1 with Gamma_path the product of
    the coefficients of the reflections before the segment, kept where the segment's
    window holds and the beam's Gaussian factor is at least exp(-C); summed exactly."""
    tris, faces = I.box_triangles(10.0, 16.0, -5.0, 5.0, 12.0)
    sc = _scene(ground=True, tris=tris, faces=faces, mats=np.ones(12, np.int32),
                gammas=[0.9, 0.7])
    dirs = np.array([[1, 0, 0.1], [1, 0.3, -0.2], [1, -0.2, 0.4], [0.2, 1, -0.5],
                     [1, 0.1, -0.6], [-1, 0.2, -0.3], [0.9, -0.4, 0.05], [0.5, 0.5, -1]], float)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    src = I.Source(np.array([0.0, 0.0, 3.0]), len(dirs), 3, 120.0)
    tr = O.trace(sc, src, dirs=dirs)
    assert tr.hit.max() >= 1 and (tr.hit == 0).any()             # box and ground both hit
    rng = np.random.default_rng(4)
    recv = np.concatenate([rng.uniform([-20, -15, 0.5], [8, 15, 10], (9, 3)),
                           [[20.0, 0.0, 2.0], [5.0, 8.0, 1.0], [-8.0, -4.0, 6.0]]]).astype(np.float32)
    w = rng.uniform(0.5, 1.5, len(dirs)) * 4 * math.pi / len(dirs)
    freqs, bb, cutoff = [400.0, 900.0], [20.0, 35.0], 16.0
    got = O.gbs_sum(tr, recv, freqs, bb, C, sc.gamma, weight=w, window=0, cutoff=cutoff)
    bad = []
    for fi, (f, b) in enumerate(zip(freqs, bb)):
        k = 2 * math.pi * f / C
        for r, x in enumerate(recv.astype(float)):
            re, im = [], []
            for j in range(tr.n_seg):
                o, t = tr.o[j], tr.t[j]
                s_loc = (x - o) @ t
                if not (0.0 <= s_loc < tr.L[j]):
                    continue
                first = j - tr.depth[j]
                gam = math.prod(float(sc.gamma[tr.bmat[q]]) for q in range(first + 1, j + 1))
                c = _eq1_matrix_form(x, o, t, tr.s0[j], k, b, w[tr.ray[j]], gam)
                s = tr.s0[j] + s_loc
                gauss = abs(c) * abs(s - 1j * b) / (w[tr.ray[j]] * gam * k * b / (8 * math.pi ** 2))
                if gauss < math.exp(-cutoff):
                    continue
                re.append(c.real)
                im.append(c.imag)
            ref = math.fsum(re) + 1j * math.fsum(im)
            if not abs(got[fi, r] - ref) <= 1e-12 * max(abs(ref), 1e-30) + 1e-18:
                bad.append((fi, r, got[fi, r], ref))
    assert np.count_nonzero(got) > 10
    return bad


def test_sum_brute_force_on_tiny_inputs():
    assert _brute_force_mismatches() == []


def test_summand_matches_matrix_form_of_eq1():
    rng = np.random.default_rng(1)
    for _ in range(40):
        t = rng.normal(size=3); t /= np.linalg.norm(t)
        o = rng.uniform(-50, 50, 3)
        s0 = rng.uniform(0, 300)
        f = rng.uniform(100, 4000); k = 2 * math.pi * f / C
        b = rng.uniform(5, 150)
        W = rng.uniform(0.01, 1.0)
        s_loc = rng.uniform(0, 400)
        nv = np.cross(t, rng.normal(size=3)); nv *= rng.uniform(0, 1) * math.sqrt(
            2 * (s0 + s_loc) ** 2 / (k * b) + b / k) / np.linalg.norm(nv)
        x = (o + s_loc * t + nv).astype(np.float32)
        tr = _one_segment_trace(o, t, L=1e6, s0=s0)
        gam = 0.7
        tr.bmat[0] = -1
        p = O.gbs_sum(tr, x[None], [f], [b], C, [gam], weight=[W], window=1, cutoff=1e9)[0, 0]
        ref = _eq1_matrix_form(x.astype(float), o, t, s0, k, b, W, 1.0)
        assert abs(p - ref) <= 1e-10 * abs(ref)       # |phase| ~ 1e4 rad in FP64


def _cutoff_window_case(cutoff=16.0):
    """One segment along +x (s0 = 20 m, L = 50 m) and receivers at s_loc in {-5, 0, 25, 50,
    60} m times normal offsets 0 .. 60 m: for each receiver the culled SEGMENT-window sum
    and the unculled LINE-window beam.  Returns (kept?, expected?, undecided?)."""
    f, b, s0, L = 800.0, 40.0, 20.0, 50.0
    k = 2 * math.pi * f / C
    tr = _one_segment_trace([0, 0, 0], [1.0, 0, 0], L=L, s0=s0)
    xs = np.array([-5.0, 0.0, 25.0, 50.0, 60.0])
    ns = np.linspace(0.0, 60.0, 241)
    recv = np.array([[x, n, 0.0] for x in xs for n in ns], np.float32)
    cut = O.gbs_sum(tr, recv, [f], [b], C, [1.0], weight=[1.0], window=0, cutoff=cutoff)[0]
    full = O.gbs_sum(tr, recv, [f], [b], C, [1.0], weight=[1.0], window=1, cutoff=1e30)[0]
    x = recv[:, 0].astype(float)
    s = s0 + x
    # the beam's Gaussian factor, read from the unculled field: |c| |E| / (k b / (8 pi^2))
    gauss = np.abs(full) * np.abs(s - 1j * b) / (k * b / (8 * math.pi ** 2))
    in_window = (x >= 0.0) & (x < L)
    expect = in_window & (gauss >= math.exp(-cutoff))
    undecided = np.abs(np.log(np.maximum(gauss, 1e-300)) + cutoff) < 1e-9
    return cut != 0, expect, undecided, cut, full, tr, recv, f, b


def test_cutoff_and_window_against_the_beam_amplitude():
    """A pair is kept iff its beam's Gaussian factor exp(-k n^2 b / (2 (s^2 + b^2))), taken
    from the magnitude of the unculled field, is at least exp(-C), and (SEGMENT window) its
    projection lies in [0, L): half-open, so a receiver abreast of the segment's end belongs
    to the next segment.  Kept pairs contribute exactly the unculled beam."""
    kept, expect, undecided, cut, full, tr, recv, f, b = _cutoff_window_case()
    assert np.array_equal(kept[~undecided], expect[~undecided])
    assert np.array_equal(cut[kept], full[kept])
    assert kept.sum() > 50 and (~kept & (recv[:, 0] >= 0) & (recv[:, 0] < 50)).sum() > 50
    assert not kept[recv[:, 0] == 50.0].any() and kept[recv[:, 0] == 0.0].any()
    assert O.count_kept(tr, recv, [f], [b], C, window=0) == int(kept.sum())


def test_single_beam_profile_closed_form():
    """On-axis |c| = W k b / (8 pi^2 sqrt(s^2+b^2)); 1/e half-width w^2 = 2(s^2+b^2)/(k b);
    on-axis phase advances at k per metre (plus the Gouy term atan(s/b))."""
    k = 2 * math.pi * 1000 / C
    b = 40.0
    tr = _one_segment_trace([0, 0, 0], [1.0, 0, 0])
    for s in (0.0, 10.0, 55.5, 300.0):
        w = math.sqrt(2 * (s * s + b * b) / (k * b))
        x = np.array([[s, 0, 0], [s, w, 0], [s, 0, 2 * w]], np.float32)
        xs = x.astype(float)
        p = O.gbs_sum(tr, x, [1000.0], [b], C, [1.0], weight=[1.0], window=1, cutoff=1e9)[0]
        ws = np.hypot(xs[:, 1], xs[:, 2])
        sx = xs[:, 0]
        amp0 = k * b / (8 * math.pi ** 2 * math.sqrt(sx[0] ** 2 + b * b))
        assert math.isclose(abs(p[0]), amp0, rel_tol=1e-12)
        assert math.isclose(abs(p[1]) / abs(p[0]), math.exp(-(ws[1] / w) ** 2), rel_tol=1e-6)
        assert math.isclose(abs(p[2]) / abs(p[0]), math.exp(-(ws[2] / w) ** 2), rel_tol=1e-6)
        # phase on axis: k s + atan(s / b)   (arg 1/(s - i b) = atan2(b, s))
        ph = (k * sx[0] + math.atan2(b, sx[0])) % (2 * math.pi)
        assert abs(((np.angle(p[0]) - ph + math.pi) % (2 * math.pi)) - math.pi) < 1e-9


# ------------------------------------------------------------- physics --

def _free_trace(n):
    return O.trace(_scene(), I.Source(np.zeros(3), n, 0, 1e4))


@pytest.fixture(scope="module")
def free65k():
    return _free_trace(65536)


@pytest.mark.parametrize("f,b", [(500.0, 70.0), (250.0, 100.0), (1000.0, 100.0), (1000.0, 50.0)])
def test_free_field_point_source(free65k, f, b):
    """A dense fan reproduces exp(ikr)/(4 pi r).  The residual is the known paraxial
    error of Gaussian beam summation: expanding the exact phase k r cos(th) +
    k r^2 sin^2(th) / (2 (r cos(th) - i b)) to fourth order in the take-off angle and
    averaging th^4 over the Gaussian gives p/p_exact - 1 = i r / (k b^2) + o(.)."""
    rng = np.random.default_rng(7)
    dirs = rng.normal(size=(6, 3)); dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    k = 2 * math.pi * f / C
    for r in (40.0, 120.0, 300.0):
        recv = (dirs * r).astype(np.float32)
        rr = np.linalg.norm(recv.astype(float), axis=1)
        p = O.gbs_sum(free65k, recv, [f], [b], C, [1.0], window=1)[0]
        exact = np.exp(1j * k * rr) / (4 * math.pi * rr)
        law = 1j * rr / (k * b * b)
        resid = p / exact - 1 - law
        assert np.all(np.abs(law) <= 0.01)            # leading-order regime
        assert np.all(np.abs(resid) <= 0.05 * np.abs(law) + np.abs(law) ** 2 + 2e-5), (r, np.abs(resid))


def test_broadband_synthesis_of_the_free_field_arrives_at_r_over_c(free65k):
    """Time synthesis of the oracle's GBS fields: 16 equally weighted frequencies of a
    free-field point source superpose to a pulse that peaks at the travel time r / c with
    the height sum_f 1 / (4 pi r) (to the paraxial error of the beams), the arrival the
    exp(-i omega t) convention fixes (the other sign would put it at -r / c)."""
    freqs = np.linspace(250.0, 4000.0, 16)
    recv = np.array([[40.0, 20.0, -10.0], [-30.0, 50.0, 25.0]], np.float32)
    rr = np.linalg.norm(recv.astype(float), axis=1)
    b = [min(100.0, I.beam_b_rule(65536, f)) for f in freqs]
    p = O.gbs_sum(free65k, recv, freqs, b, C, [1.0], window=1)
    dt = 1e-6
    for r in range(2):
        # the 250 Hz comb repeats the pulse every 4 ms: look within +-1.8 ms of r / c
        t0 = rr[r] / C - 1.8e-3
        h = O.synthesize(p[:, r:r + 1], freqs, np.ones(16), t0, dt, 3600)[:, 0]
        n = int(np.argmax(h))
        assert abs(t0 + n * dt - rr[r] / C) <= 2 * dt, (r, t0 + n * dt, rr[r] / C)
        assert math.isclose(h[n], 16 / (4 * math.pi * rr[r]), rel_tol=2e-2)
    # one frequency: a cosine of the field's phase running backwards in time
    h1 = O.synthesize(p[:1], freqs[:1], [0.5 - 0.25j], 0.0, 1e-4, 50)
    t = 1e-4 * np.arange(50)
    a = (0.5 - 0.25j) * p[0]
    assert np.allclose(h1, np.abs(a)[None, :] * np.cos(np.angle(a)[None, :] - 2 * np.pi * freqs[0] * t[:, None]),
                       rtol=0, atol=1e-14 * np.abs(a).max())


def test_free_field_error_does_not_depend_on_fan_once_resolved():
    recv = np.array([[60.0, 20.0, -30.0], [-100.0, 5.0, 40.0]], np.float32)
    k = 2 * math.pi * 500 / C
    rr = np.linalg.norm(recv.astype(float), axis=1)
    exact = np.exp(1j * k * rr) / (4 * math.pi * rr)
    errs = []
    for n in (16384, 65536):
        p = O.gbs_sum(_free_trace(n), recv, [500.0], [100.0], C, [1.0], window=1)[0]
        errs.append(p / exact - 1)
    assert np.allclose(errs[0], errs[1], atol=2e-5)


@pytest.mark.parametrize("gam", [1.0, 0.9, 0.5])
def test_two_image_sources(gam):
    """Rigid/absorbing infinite plane (the paper's verification case, Sec. 4.1): the
    field is the direct source plus gamma times its mirror image."""
    sc = _scene(ground=True, gamma=gam)
    zs = 5.0
    tr = O.trace(sc, I.Source(np.array([0.0, 0.0, zs]), 65536, 1, 1e4))
    xs = np.array([-100, -60, -30, -15, 15, 30, 60, 100.0])
    f, b = 2000.0, 100.0
    k = 2 * math.pi * f / C
    for z in (10.0, 40.0):
        recv = np.stack([xs, np.full_like(xs, 7.0), np.full_like(xs, z)], 1).astype(np.float32)
        x = recv.astype(float)
        p = O.gbs_sum(tr, recv, [f], [b], C, sc.gamma, window=1)[0]
        r1 = np.linalg.norm(x - [0, 0, zs], axis=1)
        r2 = np.linalg.norm(x - [0, 0, -zs], axis=1)
        d = np.exp(1j * k * r1) / (4 * math.pi * r1) * (1 + 1j * r1 / (k * b * b))
        im = gam * np.exp(1j * k * r2) / (4 * math.pi * r2) * (1 + 1j * r2 / (k * b * b))
        err = np.abs(p - d - im) / np.abs(d + im).max()
        assert err.max() < 2e-4, err
    # close to the plane, where the reflected beams must extend back to the image
    recv = np.array([[40.0, 7.0, 0.5], [-25.0, 3.0, 1.0], [60.0, -10.0, 2.0]], np.float32)
    x = recv.astype(float)
    p = O.gbs_sum(tr, recv, [f], [b], C, sc.gamma, window=1)[0]
    r1 = np.linalg.norm(x - [0, 0, zs], axis=1)
    r2 = np.linalg.norm(x - [0, 0, -zs], axis=1)
    d = np.exp(1j * k * r1) / (4 * math.pi * r1) * (1 + 1j * r1 / (k * b * b))
    im = gam * np.exp(1j * k * r2) / (4 * math.pi * r2) * (1 + 1j * r2 / (k * b * b))
    assert np.max(np.abs(p - d - im) / np.abs(d + im).max()) < 5e-4


def test_reciprocity_over_ground():
    """Swapping source and receiver leaves the field unchanged (up to GBS error)."""
    sc = _scene(ground=True, gamma=0.8)
    A = np.array([0.0, 0.0, 6.0])
    B = np.array([70.0, -40.0, 25.0], np.float32)
    f, b = 1000.0, 100.0
    pa = O.gbs_sum(O.trace(sc, I.Source(A, 65536, 1, 1e4)), B[None], [f], [b], C,
                   sc.gamma, window=1)[0, 0]
    Bd = B.astype(np.float64)
    pb = O.gbs_sum(O.trace(sc, I.Source(Bd, 65536, 1, 1e4)), A[None].astype(np.float32),
                   [f], [b], C, sc.gamma, window=1)[0, 0]
    assert abs(pa - pb) <= 1e-3 * abs(pa)


# ------------------------------------------------------------- adjoint --

@pytest.fixture(scope="module")
def small_city_problem():
    ta, fa = _box(20, 40, -30, 10, 25, 0)
    tb, fb = _box(-45, -25, 5, 40, 35, 6)
    tris = np.concatenate([ta, tb]); faces = np.concatenate([fa, fb])
    mats = np.array([1] * 12 + [2] * 12, np.int32)
    sc = _scene(ground=True, tris=tris, faces=faces, mats=mats, gammas=[0.9, 0.8, 0.6])
    src = I.Source(np.array([0.0, 0.0, 4.0]), 2048, 4, 300.0)
    tr = O.trace(sc, src)
    rng = np.random.default_rng(3)
    recv = I.random_receivers(rng, 24, [-60, -60, 1], [60, 60, 20])
    freqs = np.array([300.0, 700.0])
    b = np.array([30.0, 45.0])
    pt = (rng.normal(size=(2, 24)) + 1j * rng.normal(size=(2, 24))) * 1e-3
    return sc, tr, recv, freqs, b, pt


def _loss(prob, gamma, w, b, b_mask):
    sc, tr, recv, freqs, _, pt = prob
    p = O.gbs_sum(tr, recv, freqs, b, C, gamma, weight=w, window=0, b_mask=b_mask)
    return float(np.sum(np.abs(p - pt) ** 2)), p


def test_adjoint_matches_central_differences(small_city_problem):
    sc, tr, recv, freqs, b, pt = small_city_problem
    gamma = sc.gamma.astype(float)
    w = O.default_weight(tr.n_rays) * (1 + 0.1 * np.sin(np.arange(tr.n_rays)))
    L0, p = _loss(small_city_problem, gamma, w, b, b)
    g = 2 * (p - pt)
    dg, dw, db = O.gbs_adjoint(tr, recv, freqs, b, C, gamma, g, weight=w, window=0)
    h = 1e-6
    for m in range(3):
        e = np.zeros(3); e[m] = h
        fd = (_loss(small_city_problem, gamma + e, w, b, b)[0] -
              _loss(small_city_problem, gamma - e, w, b, b)[0]) / (2 * h)
        assert math.isclose(dg[m], fd, rel_tol=1e-6, abs_tol=1e-12 * abs(L0) / h), (m, dg[m], fd)
    for f in range(2):
        e = np.zeros(2); e[f] = h * b[f]
        fd = (_loss(small_city_problem, gamma, w, b + e, b)[0] -
              _loss(small_city_problem, gamma, w, b - e, b)[0]) / (2 * e[f])
        assert math.isclose(db[f], fd, rel_tol=1e-5), (f, db[f], fd)
    top = np.argsort(-np.abs(dw))[:4]
    for i in top:
        e = np.zeros_like(w); e[i] = h * w[i]
        fd = (_loss(small_city_problem, gamma, w + e, b, b)[0] -
              _loss(small_city_problem, gamma, w - e, b, b)[0]) / (2 * e[i])
        assert math.isclose(dw[i], fd, rel_tol=1e-5), (i, dw[i], fd)


# --------------------------------------------------------- b rule, grid --

def test_beam_b_rule_width():
    for n, f in ((1024, 500.0), (4096, 250.0), (65536, 125.0), (1 << 20, 1000.0)):
        b = I.beam_b_rule(n, f)
        k = 2 * math.pi * f / C
        w2 = 2 * (100.0 ** 2 + b * b) / (k * b)       # 1/e half-width^2 at 100 m
        target = (math.sqrt(4 * math.pi / n) * 100.0) ** 2
        if b != 100.0:
            assert math.isclose(w2, target, rel_tol=1e-12)
            assert b < 100.0
        else:
            assert w2 >= target        # diffraction limited: no b reaches the target
    assert abs(I.beam_b_rule(1024, 500.0) - 18.4) < 0.05


def test_receiver_grid_endpoints():
    g = I.receiver_grid(64, 50.0, 1.5)
    assert g.shape == (4096, 3) and g.dtype == np.float32
    assert g[0, 0] == -50 and g[63, 0] == 50 and g[-1, 1] == 50 and np.all(g[:, 2] == 1.5)
