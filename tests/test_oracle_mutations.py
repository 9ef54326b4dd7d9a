"""Planted mistakes: each plausible slip in the oracle must fail at least one pin.

Every case edits a private copy of the oracle's C source (on the CPU), builds
it, and runs a compact battery of the independent pins against it.  The
committed oracle itself passes the same battery.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13382_gb300 import inputs as I

C = 343.0

MUTATIONS = {
    "phase_sign": ("cexp(I * k * s + I * k * n2 / (2.0 * E))",
                   "cexp(-I * k * s + I * k * n2 / (2.0 * E))"),
    "dropped_1_over_E": ("(8.0 * ORC_PI * ORC_PI)) / E * cexp", "(8.0 * ORC_PI * ORC_PI)) * cexp"),
    "normalisation": ("(k * b / (8.0 * ORC_PI * ORC_PI))", "(k * b / (4.0 * ORC_PI * ORC_PI))"),
    "E_sign": ("double complex E = s - I * b;\n    return", "double complex E = s + I * b;\n    return"),
    "cross_transposed": ("double cx = dy * t[2] - dz * t[1];", "double cx = dy * t[1] - dz * t[2];"),
    "reflection_factor": ("d[2] = d[2] - 2.0 * dn * nrm[2];", "d[2] = d[2] - dn * nrm[2];"),
    "gamma_path_sum": ("for (int64_t q = first + 1; q <= j; ++q) g *= gamma[S->bmat[q]];",
                       "for (int64_t q = first + 1; q <= j; ++q) g += gamma[S->bmat[q]];"),
    "line_window_local": ("if (!(s >= 0.0)) return 0;", "if (!(s_loc >= 0.0)) return 0;"),
    "adjoint_b_sign": ("1.0 / b + I / E - k * n2", "1.0 / b - I / E - k * n2"),
    "fan_offset": ("double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;",
                   "double z = 1.0 - (2.0 * (double)i) / (double)n;"),
    "gaussian_exponent_half": ("I * k * n2 / (2.0 * E)", "I * k * n2 / E"),
    "adjoint_weight_without_gamma_path": ("mw[ray] += creal(gc * gpath[j] * cu);",
                                          "mw[ray] += creal(gc * cu);"),
    "adjoint_gamma_product_includes_self": ("if (q2 != q) other *= gamma[S->bmat[q2]];",
                                            "other *= gamma[S->bmat[q2]];"),
    "adjoint_gamma_without_weight": ("mg[S->bmat[q]] += creal(gc * weight[ray] * other * cu);",
                                     "mg[S->bmat[q]] += creal(gc * other * cu);"),
    "cutoff_without_b": ("return k * n2 * bm / (2.0 * (s * s + bm * bm)) <= A->cutoff;",
                         "return k * n2 / (2.0 * (s * s + bm * bm)) <= A->cutoff;"),
    "segment_window_closed_end": ("if (!(s_loc >= 0.0 && s_loc < S->L[j])) return 0;",
                                  "if (!(s_loc >= 0.0 && s_loc <= S->L[j])) return 0;"),
    "latlong_midpoint_weight": ("const double cell = dph * (cos(lo) - cos(hi));",
                                "const double cell = dph * dth * sin(th);"),
    "latlong_cell_edge": ("const double th = th0 + ((double)it + 0.5) * dth;",
                          "const double th = th0 + (double)it * dth;"),
    "latlong_sin_cos_swapped": ("dirs[3 * g + 0] = sin(th) * cos(ph);",
                                "dirs[3 * g + 0] = cos(th) * cos(ph);"),
    # propagation losses (the loss battery below)
    "absorption_local_arclength": ("orc_acc_add(&acc, w * orc_losses(S, A, f, j, s) * orc_beam",
                                   "orc_acc_add(&acc, w * orc_losses(S, A, f, j, s - S->s0[j]) * orc_beam"),
    "absorption_sign": ("if (A->absorb) L *= exp(-A->absorb[f] * s);",
                        "if (A->absorb) L *= exp(A->absorb[f] * s);"),
    "absorption_db_not_np": ("return orc_air_absorption_db(f, T_c, rh, p_kpa) / (20.0 / log(10.0));",
                             "return orc_air_absorption_db(f, T_c, rh, p_kpa);"),
    "iso_oxygen_humidity": ("h * (0.02 + h) / (0.391 + h)", "h * (0.2 + h) / (0.391 + h)"),
    "iso_nitrogen_temperature": ("pow(T / T0, -1.0 / 3.0) - 1.0", "pow(T / T0, 1.0 / 3.0) - 1.0"),
    "reflection_inverted": ("return (Z * cos_theta - 1.0) / (Z * cos_theta + 1.0);",
                            "return (Z - cos_theta) / (Z + cos_theta);"),
    "delany_bazley_imag_sign": ("+ I * 11.9 * pow(x, -0.73)", "- I * 11.9 * pow(x, -0.73)"),
    "incidence_sine": ("cosi[j] = fabs(t[3 * j] * nrm[0] + t[3 * j + 1] * nrm[1] + t[3 * j + 2] * nrm[2]);",
                       "cosi[j] = sqrt(1.0 - pow(t[3 * j] * nrm[0] + t[3 * j + 1] * nrm[1] + "
                       "t[3 * j + 2] * nrm[2], 2.0));"),
    "path_factor_skips_first_bounce": ("for (int64_t q = first + 1; q <= j; ++q) {\n                const double sg",
                                       "for (int64_t q = first + 2; q <= j; ++q) {\n                const double sg"),
    "adjoint_without_losses": ("double complex cu = orc_losses(S, A, f, j, s) * orc_beam(k, b, s, n2);",
                               "double complex cu = orc_beam(k, b, s, n2);"),
}


def _battery():
    """Independent checks (closed forms, images, FD); True iff all pass."""
    ok = True
    # fan: equal-area z bands
    d = O.fan_fibonacci(1024)
    ok &= bool(np.allclose(d[:, 2], 1.0 - (2.0 * np.arange(1024) + 1.0) / 1024, atol=1e-15))
    # lat-long fan: cell centres and cell solid angles (quadrature of sin(theta))
    from scipy.integrate import quad
    dl, wl = O.fan_latlong(6, 4, (20.0, 140.0), (0.0, 360.0))
    ok &= bool(np.allclose(np.linalg.norm(dl, axis=1), 1.0, atol=1e-15))
    ok &= bool(np.allclose(np.degrees(np.arccos(dl[::4, 2])), 20.0 + 20.0 * (np.arange(6) + 0.5)))
    cells = [quad(math.sin, math.radians(20.0 + 20.0 * i), math.radians(40.0 + 20.0 * i))[0] *
             math.pi / 2 for i in range(6)]
    ok &= bool(np.allclose(wl[::4], cells, rtol=1e-12))
    # free field, point source with the paraxial law p/p_exact - 1 = i r / (k b^2)
    sc = I.Scene(C, False, 0.0, 0, np.zeros((0, 3, 3)), np.zeros(0, np.int32),
                 np.zeros(0, np.int32), np.array([1.0], np.float32))
    tr = O.trace(sc, I.Source(np.zeros(3), 16384, 0, 1e4))
    recv = np.array([[60.0, 20.0, -30.0], [-80.0, 5.0, 40.0]], np.float32)
    f, b = 500.0, 100.0
    k = 2 * math.pi * f / C
    rr = np.linalg.norm(recv.astype(float), axis=1)
    p = O.gbs_sum(tr, recv, [f], [b], C, [1.0], window=1)[0]
    ex = np.exp(1j * k * rr) / (4 * math.pi * rr)
    ok &= bool(np.all(np.abs(p / ex - 1 - 1j * rr / (k * b * b)) < 1e-4))
    # ground plane with gamma = 0.6: direct + 0.6 x image
    sg = I.Scene(C, True, 0.0, 0, np.zeros((0, 3, 3)), np.zeros(0, np.int32),
                 np.zeros(0, np.int32), np.array([0.6], np.float32))
    tg = O.trace(sg, I.Source(np.array([0.0, 0.0, 5.0]), 65536, 1, 1e4))
    recv = np.array([[30.0, 7.0, 10.0], [-60.0, 7.0, 40.0], [15.0, -7.0, 25.0],
                     [40.0, 7.0, 0.5], [-25.0, 3.0, 1.0]], np.float32)
    f = 2000.0
    k = 2 * math.pi * f / C
    x = recv.astype(float)
    r1 = np.linalg.norm(x - [0, 0, 5], axis=1); r2 = np.linalg.norm(x - [0, 0, -5], axis=1)
    exg = (np.exp(1j * k * r1) / (4 * math.pi * r1) * (1 + 1j * r1 / (k * b * b)) +
           0.6 * np.exp(1j * k * r2) / (4 * math.pi * r2) * (1 + 1j * r2 / (k * b * b)))
    pg = O.gbs_sum(tg, recv, [f], [b], C, sg.gamma, window=1)[0]
    ok &= bool(np.all(np.abs(pg - exg) < 5e-4 * np.abs(exg).max()))
    # off-axis single beam against Eq. 1 in matrix form
    from tests.test_oracle_pins import _eq1_matrix_form, _one_segment_trace
    t = np.array([0.3, -0.5, 0.81]); t /= np.linalg.norm(t)
    o = np.array([1.0, 2.0, 3.0])
    tr1 = _one_segment_trace(o, t, L=1e6, s0=12.0)
    xs = (o + 80 * t + np.array([3.0, 1.0, 0.5]) - (np.array([3.0, 1.0, 0.5]) @ t) * t)
    xs = xs.astype(np.float32)
    p1 = O.gbs_sum(tr1, xs[None], [700.0], [30.0], C, [1.0], weight=[0.5], window=1,
                   cutoff=1e9)[0, 0]
    ref = _eq1_matrix_form(xs.astype(float), o, t, 12.0, 2 * math.pi * 700 / C, 30.0, 0.5, 1.0)
    ok &= bool(abs(p1 - ref) < 1e-9 * abs(ref))
    # adjoint in b against central differences (mask frozen)
    recv = np.array([[30.0, 7.0, 10.0], [-20.0, 3.0, 12.0]], np.float32)
    g = np.array([[1.0 + 0.5j, -0.3 + 1j]])
    bb = np.array([40.0])
    _, _, db = O.gbs_adjoint(tg, recv, [800.0], bb, C, [0.6], g, window=1)
    h = 1e-4
    lp = np.real(np.conj(g) * O.gbs_sum(tg, recv, [800.0], bb + h, C, [0.6], window=1,
                                        b_mask=bb)).sum()
    lm = np.real(np.conj(g) * O.gbs_sum(tg, recv, [800.0], bb - h, C, [0.6], window=1,
                                        b_mask=bb)).sum()
    ok &= bool(math.isclose(db[0], (lp - lm) / (2 * h), rel_tol=1e-5))
    # Eq. 3 as a plain triple loop on a tiny traced scene
    from tests.test_oracle_pins import _brute_force_mismatches
    ok &= not _brute_force_mismatches()
    # cutoff and window against the beam amplitude (one segment, a grid of receivers)
    from tests.test_oracle_pins import _cutoff_window_case
    kept, expect, undecided = _cutoff_window_case()[:3]
    ok &= bool(np.array_equal(kept[~undecided], expect[~undecided]))
    # adjoint in gamma and in the ray weights against central differences (the field is
    # linear in both over a single reflection, so the differences are exact up to rounding)
    rng = np.random.default_rng(3)
    w0 = (4 * math.pi / tg.n_rays) * rng.uniform(0.5, 1.5, tg.n_rays)
    dg, dw, _ = O.gbs_adjoint(tg, recv, [800.0], bb, C, [0.6], g, weight=w0, window=1)
    loss = lambda gam, w: np.real(np.conj(g) * O.gbs_sum(tg, recv, [800.0], bb, C, [gam],
                                                          weight=w, window=1)).sum()
    hg = 1e-3
    ok &= bool(math.isclose(dg[0], (loss(0.6 + hg, w0) - loss(0.6 - hg, w0)) / (2 * hg),
                            rel_tol=1e-6))
    v = rng.normal(size=tg.n_rays) * (4 * math.pi / tg.n_rays)
    fd = (loss(0.6, w0 + v) - loss(0.6, w0 - v)) / 2
    ok &= bool(math.isclose(float(dw @ v), fd, rel_tol=1e-6))
    return ok


def _loss_battery():
    """The loss pins (tests/test_oracle_losses.py) on small cases; True iff all pass."""
    from tests import test_oracle_losses as TL
    ok = not TL.iso_table_mismatches()
    sc0 = I.Scene(C, False, 0.0, 0, np.zeros((0, 3, 3)), np.zeros(0, np.int32),
                  np.zeros(0, np.int32), np.array([1.0], np.float32))
    tr = O.trace(sc0, I.Source(np.zeros(3), 16384, 0, 1e4))
    res, corr = TL.free_field_absorption_residual(tr, 500.0, 100.0, 0.01, 120.0)
    ok &= bool(res <= 0.05 * corr + corr ** 2 + 1e-6)
    # the level drop of the paper's atmosphere at 4 kHz over 300 m
    a = O.air_absorption([4000.0])[0]
    alpha = O.air_absorption_db([4000.0])[0]
    recv = np.array([[300.0, 0.0, 0.0]], np.float32)
    p0 = O.gbs_sum(tr, recv, [4000.0], [100.0], C, [1.0], window=1)[0, 0]
    pa = O.gbs_sum(tr, recv, [4000.0], [100.0], C, [1.0], window=1, absorption=[a])[0, 0]
    ok &= bool(abs(20 * math.log10(abs(p0) / abs(pa)) - alpha * 300.0) < 2e-3 * alpha * 300.0)
    ok &= bool(TL.image_field_with_absorption_error() < 3e-4)
    # reflection factor against the impedance boundary condition
    Z, th, k = 5.57 + 6.1j, 0.7, 2.0
    R = O.plane_wave_reflection(Z, math.cos(th))
    pz = lambda z: np.exp(-1j * k * z * math.cos(th)) + R * np.exp(1j * k * z * math.cos(th))
    h = 1e-5
    ok &= bool(abs(pz(0.0) / (-(pz(h) - pz(-h)) / (2 * h) / (1j * k)) - Z) < 1e-6 * abs(Z))
    # Delany-Bazley against the Rayleigh model's sign and size
    zd = O.delany_bazley(500.0, 200.0)
    zr = np.sqrt(1 + 1j * 200e3 / (2 * math.pi * 500.0 * 1.2))
    ok &= bool(zd.real > 1 and zd.imag > 0 and 0.6 < abs(zd) / abs(zr) < 1.6 and
               abs(np.angle(zd) - np.angle(zr)) < math.radians(12.0))
    ok &= not TL.hand_traced_path_factor_errors()
    for f, sig, z, e0, e1, c in TL.porous_ground_image_errors(((1000.0, 200.0),)):
        ok &= bool(e1 < e0 and e1 <= 0.35 * c + 2e-4)
    from tests.test_oracle_pins import _box
    ta, fa = _box(20, 40, -30, 10, 25, 0)
    sc = I.Scene(C, True, 0.0, 0, ta, np.ones(12, np.int32), fa, np.array([0.9, 0.7], np.float32))
    trc = O.trace(sc, I.Source(np.array([0.0, 0.0, 4.0]), 512, 3, 300.0))
    rng = np.random.default_rng(5)
    prob = (sc, trc, I.random_receivers(rng, 8, [-60, -60, 1], [60, 60, 20]),
            np.array([400.0]), np.array([35.0]),
            (rng.normal(size=(1, 8)) + 1j * rng.normal(size=(1, 8))) * 1e-3,
            np.array([150.0, 40.0]), np.array([0.015]))
    errs = TL.lossy_adjoint_errors(prob)
    ok &= bool(max(errs) < 1e-5)
    return ok


def test_unmutated_oracle_passes_battery():
    assert _battery()
    assert _loss_battery()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = O.source_text()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    lib = O.compile_source(src.replace(old, new), str(tmp_path / f"liboracle_{name}.so"))
    with O.use_library(lib):
        assert not (_battery() and _loss_battery()), f"planted mistake {name} went undetected"
