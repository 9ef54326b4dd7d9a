"""Seeded synthetic inputs for Gaussian beam summation (GBS) workloads.

This module only builds input arrays: scene geometry, source descriptions,
receiver grids, frequency lists and beam parameters.  It holds none of the
method's arithmetic (no fan, no tracing, no beam summation), so both the FP64
oracle and the CUDA library consume exactly the same inputs.

The five workloads stand in for the paper's free-field and city cases
(Sec. 4.5, Tables 2 and 3): the paper's city geometry is not published, so the
city is a seeded grid of axis-aligned box buildings on a ground plane.

Conventions
-----------
* Primitive ids: 0 is the ground plane z = ground_z (normal +z), 1..T are the
  triangles in the order given.
* Face ids group coplanar triangles of one planar facet (two per box face);
  a reflected ray may not hit the facet it just left.
* Materials index the per-material reflection coefficients ``gamma``.
* Seeds are ``13382 + workload index`` (workloads numbered 1..5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

C_AIR = 343.0          # m/s, homogeneous air
SEED_BASE = 13382

WINDOW_SEGMENT = 0     # 0 <= s_loc < L
WINDOW_LINE = 1        # s >= 0 (unfolded full line; exact images for infinite planes)


@dataclass
class Scene:
    c: float
    ground: bool
    ground_z: float
    ground_material: int
    tri_xyz: np.ndarray          # (T, 3, 3) float64 vertices
    tri_material: np.ndarray     # (T,) int32
    tri_face: np.ndarray         # (T,) int32 facet id (coplanar triangles share one)
    gamma: np.ndarray            # (M,) float32 per-material reflection coefficient

    @property
    def n_tri(self) -> int:
        return int(self.tri_xyz.shape[0])

    @property
    def n_materials(self) -> int:
        return int(self.gamma.shape[0])


FAN_FIBONACCI, FAN_LATLONG = 0, 2


@dataclass
class Source:
    pos: np.ndarray              # (3,) float64
    n_rays: int
    max_reflections: int
    max_path: float              # m
    fan: int = FAN_FIBONACCI     # FAN_LATLONG: n_theta rows of n_rays / n_theta azimuths
    n_theta: int = 0
    theta_deg: tuple = (0.0, 180.0)   # polar angle range from +z, degrees
    phi_deg: tuple = (0.0, 360.0)     # azimuth range, degrees


@dataclass
class Workload:
    name: str
    scene: Scene
    sources: List[Source]
    receivers: np.ndarray        # (Nr, 3) float32
    freqs: np.ndarray            # (F,) float64 Hz (per source when batched: same list)
    window: int
    cutoff: float = 16.0
    beam_b: Optional[List[np.ndarray]] = None   # per source, (F,) float64 metres
    extra: dict = field(default_factory=dict)


def receiver_grid(n: int, half: float, z: float, center=(0.0, 0.0)) -> np.ndarray:
    """n x n receivers on [-half, half]^2 (+center), endpoints included, row-major (y outer)."""
    xs = np.linspace(-half, half, n) + center[0]
    ys = np.linspace(-half, half, n) + center[1]
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel(), np.full(n * n, z)], axis=1)
    return pts.astype(np.float32)


def beam_b_rule(n_rays: int, freq_hz: float, c: float = C_AIR, s_ref: float = 100.0) -> float:
    """Beam parameter b (metres) for a fan of n_rays at one frequency.

    The paper fixes the beam's imaginary parameter only as a bare number with no
    units (Tables 2-3), so this is a configuration choice: pick b so that the
    1/e amplitude half-width w(s)^2 = 2 (s^2 + b^2) / (k b) at s_ref equals the
    fan's angular spacing times s_ref.  When no real b reaches that width (the
    beam is diffraction limited), b = s_ref.
    """
    k = 2.0 * math.pi * freq_hz / c
    dtheta = math.sqrt(4.0 * math.pi / n_rays)
    w_ref = dtheta * s_ref
    a = 0.5 * k * w_ref * w_ref          # b^2 - a b + s_ref^2 = 0
    disc = a * a - 4.0 * s_ref * s_ref
    if disc >= 0.0:
        return 2.0 * s_ref * s_ref / (a + math.sqrt(disc))
    return s_ref


def _ground_scene(gamma_ground: float) -> Scene:
    return Scene(c=C_AIR, ground=True, ground_z=0.0, ground_material=0,
                 tri_xyz=np.zeros((0, 3, 3)), tri_material=np.zeros(0, np.int32),
                 tri_face=np.zeros(0, np.int32),
                 gamma=np.array([gamma_ground], np.float32))


def box_triangles(x0, x1, y0, y1, h):
    """12 triangles (2 per face, bottom included) of the box [x0,x1]x[y0,y1]x[0,h].

    Returns (tris (12,3,3), local face index (12,)) with faces ordered
    x=x0, x=x1, y=y0, y=y1, z=0, z=h.
    """
    P = lambda x, y, z: (x, y, z)
    quads = [
        (P(x0, y0, 0), P(x0, y1, 0), P(x0, y1, h), P(x0, y0, h)),
        (P(x1, y0, 0), P(x1, y0, h), P(x1, y1, h), P(x1, y1, 0)),
        (P(x0, y0, 0), P(x0, y0, h), P(x1, y0, h), P(x1, y0, 0)),
        (P(x0, y1, 0), P(x1, y1, 0), P(x1, y1, h), P(x0, y1, h)),
        (P(x0, y0, 0), P(x1, y0, 0), P(x1, y1, 0), P(x0, y1, 0)),
        (P(x0, y0, h), P(x0, y1, h), P(x1, y1, h), P(x1, y0, h)),
    ]
    tris, faces = [], []
    for fi, (a, b, c, d) in enumerate(quads):
        tris.append((a, b, c))
        tris.append((a, c, d))
        faces += [fi, fi]
    return np.array(tris, np.float64), np.array(faces, np.int32)


def synthetic_city(seed: int, n_side: int = 8, extent: float = 500.0):
    """Seeded city: an n_side x n_side jittered grid of box buildings on a ground plane.

    Cells are extent/n_side wide on [-extent/2, extent/2]^2; footprint sides are
    U(20, 60) per axis, centres jittered so streets stay >= 2.5 m wide; heights
    U(10, 60).  Returns (triangles, face ids, building index per triangle,
    footprints (B,4) [x0,x1,y0,y1], heights (B,), building gamma (B,)).
    """
    rng = np.random.default_rng(seed)
    nb = n_side * n_side
    cell = extent / n_side
    sides = rng.uniform(20.0, 60.0, size=(nb, 2))
    jit_u = rng.uniform(-1.0, 1.0, size=(nb, 2))
    heights = rng.uniform(10.0, 60.0, size=nb)
    gammas = rng.uniform(0.70, 0.95, size=nb)
    tris, faces, bidx, foot = [], [], [], []
    for b in range(nb):
        i, j = b % n_side, b // n_side
        cx = -extent / 2 + cell * (i + 0.5)
        cy = -extent / 2 + cell * (j + 0.5)
        jmax = np.maximum(0.0, (cell - sides[b]) / 2 - 1.25)
        cx += jit_u[b, 0] * jmax[0]
        cy += jit_u[b, 1] * jmax[1]
        x0, x1 = cx - sides[b, 0] / 2, cx + sides[b, 0] / 2
        y0, y1 = cy - sides[b, 1] / 2, cy + sides[b, 1] / 2
        t, f = box_triangles(x0, x1, y0, y1, heights[b])
        tris.append(t)
        faces.append(f + 6 * b)
        bidx.append(np.full(12, b, np.int32))
        foot.append((x0, x1, y0, y1))
    return (np.concatenate(tris), np.concatenate(faces).astype(np.int32),
            np.concatenate(bidx), np.array(foot), heights, gammas)


def city_scene(seed: int, material_of_building=None, gamma_buildings=None, n_side: int = 8,
               extent: float = 500.0) -> Scene:
    """Ground (material 0, gamma 1.0: hard surface) plus the synthetic city.

    By default each building is its own material 1+b with its seeded gamma.
    ``material_of_building`` (B,) maps building -> material index >= 1 and
    ``gamma_buildings`` gives gamma per such material (index 1..).
    """
    tris, faces, bidx, foot, heights, gam = synthetic_city(seed, n_side, extent)
    nb = foot.shape[0]
    if material_of_building is None:
        mat = (1 + bidx).astype(np.int32)
        gamma = np.concatenate([[1.0], gam]).astype(np.float32)
    else:
        mob = np.asarray(material_of_building, np.int32)
        mat = mob[bidx].astype(np.int32)
        gamma = np.concatenate([[1.0], np.asarray(gamma_buildings)]).astype(np.float32)
    sc = Scene(c=C_AIR, ground=True, ground_z=0.0, ground_material=0,
               tri_xyz=tris, tri_material=mat, tri_face=faces, gamma=gamma)
    sc_extra = {"footprints": foot, "heights": heights, "n_buildings": nb}
    return sc, sc_extra


def _with_b(w: Workload) -> Workload:
    w.beam_b = [np.array([beam_b_rule(s.n_rays, f, w.scene.c) for f in w.freqs])
                for s in w.sources]
    return w


def open_plane_small() -> Workload:
    """Open plane, plain GBS: 1,024 rays, <=2 reflections, 200 m, 64x64 receivers, 500 Hz."""
    sc = _ground_scene(1.0)
    src = Source(np.array([0.0, 0.0, 2.0]), 1024, 2, 200.0)
    return _with_b(Workload("open_plane_1k_rays_64x64_500Hz", sc, [src],
                            receiver_grid(64, 50.0, 1.5), np.array([500.0]),
                            WINDOW_LINE))


def open_plane_large() -> Workload:
    """Open plane, large: 65,536 rays, <=3 reflections, 1 km, 256x256 receivers, 6 octave bands."""
    sc = _ground_scene(0.9)
    src = Source(np.array([0.0, 0.0, 2.0]), 65536, 3, 1000.0)
    freqs = 125.0 * 2.0 ** np.arange(6)
    return _with_b(Workload("open_plane_64k_rays_256x256_6f", sc, [src],
                            receiver_grid(256, 500.0, 1.5), freqs, WINDOW_LINE))


def open_plane_latlong(n_theta: int = 128, n_phi: int = 256) -> Workload:
    """Open plane with the take-off grid of the paper's input tables (polar angle 0-180,
    azimuth 0-360 degrees): 128 x 256 rays, <=2 reflections, 400 m, 96x96 receivers,
    two bands."""
    sc = _ground_scene(0.9)
    src = Source(np.array([0.0, 0.0, 10.0]), n_theta * n_phi, 2, 400.0, FAN_LATLONG, n_theta)
    return _with_b(Workload(f"open_plane_latlong_{n_theta}x{n_phi}_96x96_2f", sc, [src],
                            receiver_grid(96, 150.0, 1.5), np.array([250.0, 500.0]),
                            WINDOW_LINE))


CITY_MAX_PATH = 1000.0


def _count_name(n: int) -> str:
    """1048576 -> '1M', 262144 -> '256k', 1000 -> '1000'."""
    if n % (1 << 20) == 0:
        return f"{n >> 20}M"
    if n % 1024 == 0:
        return f"{n >> 10}k"
    return str(n)


def city(n_rays: int = 1 << 20, n_recv_side: int = 512) -> Workload:
    """Synthetic city: 64 boxes, 1,048,576 rays from (0,0,5), <=8 reflections, 512^2 receivers, 1 kHz."""
    sc, ex = city_scene(SEED_BASE + 3)
    src = Source(np.array([0.0, 0.0, 5.0]), n_rays, 8, CITY_MAX_PATH)
    w = Workload(f"city_{_count_name(n_rays)}_rays_{n_recv_side}x{n_recv_side}_1kHz", sc, [src],
                 receiver_grid(n_recv_side, 250.0, 1.5), np.array([1000.0]),
                 WINDOW_SEGMENT, extra=ex)
    return _with_b(w)


def big_city(n_rays: int = 1 << 18, n_recv_side: int = 256) -> Workload:
    """Large synthetic city for the BVH: 32 x 32 boxes over 2 km (12,288 triangles),
    262,144 rays from (0,0,5), <=8 reflections, 1 km paths, 256^2 receivers, 1 kHz."""
    sc, ex = city_scene(SEED_BASE + 6, n_side=32, extent=2000.0)
    src = Source(np.array([0.0, 0.0, 5.0]), n_rays, 8, CITY_MAX_PATH)
    w = Workload("big_city_12k_tris_256k_rays_256x256_1kHz", sc, [src],
                 receiver_grid(n_recv_side, 1000.0, 1.5), np.array([1000.0]),
                 WINDOW_SEGMENT, extra=ex)
    return _with_b(w)


def _dist_to_rect(x, y, r):
    dx = max(r[0] - x, 0.0, x - r[1])
    dy = max(r[2] - y, 0.0, y - r[3])
    return math.hypot(dx, dy)


def batched_city(n_sources: int = 32) -> Workload:
    """32 sources in the open streets at 1-30 m, log-uniform 4,096-262,144 rays each, 8 freqs."""
    sc, ex = city_scene(SEED_BASE + 3)
    rng = np.random.default_rng(SEED_BASE + 4)
    foot = ex["footprints"]
    srcs = []
    while len(srcs) < n_sources:
        x, y = rng.uniform(-250.0, 250.0, size=2)
        z = rng.uniform(1.0, 30.0)
        n = int(round(math.exp(rng.uniform(math.log(4096), math.log(262144)))))
        if min(_dist_to_rect(x, y, r) for r in foot) < 1.0:
            continue
        srcs.append(Source(np.array([x, y, z]), n, 8, CITY_MAX_PATH))
    freqs = 125.0 * 2.0 ** (5.0 * np.arange(8) / 7.0)
    w = Workload("batched_city_32src_8f_512x512", sc, srcs,
                 receiver_grid(512, 250.0, 1.5), freqs, WINDOW_SEGMENT, extra=ex)
    return _with_b(w)


def diff_city():
    """Differentiable city: buildings in 8 material groups (gamma init 0.8), 262,144 rays,
    <=6 reflections, 128^2 receivers, 4 frequencies; target gammas U(0.6, 0.95) seeded."""
    nb = 64
    group = (np.arange(nb) % 8 + 1).astype(np.int32)
    sc, ex = city_scene(SEED_BASE + 3, material_of_building=group,
                        gamma_buildings=np.full(8, 0.8))
    rng = np.random.default_rng(SEED_BASE + 5)
    target = np.concatenate([[1.0], rng.uniform(0.6, 0.95, size=8)]).astype(np.float32)
    src = Source(np.array([0.0, 0.0, 5.0]), 262144, 6, CITY_MAX_PATH)
    w = Workload("diff_city_256k_rays_128x128_4f", sc, [src],
                 receiver_grid(128, 250.0, 1.5), np.array([250.0, 500.0, 1000.0, 2000.0]),
                 WINDOW_SEGMENT, extra=dict(ex, target_gamma=target))
    return _with_b(w)


WORKLOADS = {
    1: open_plane_small,
    2: open_plane_large,
    3: city,
    4: batched_city,
    5: diff_city,
}


def random_receivers(rng: np.random.Generator, n: int, lo, hi) -> np.ndarray:
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)


def receiver_subset(receivers: np.ndarray, n: int, seed: int) -> np.ndarray:
    """Seeded subset of receiver indices (sorted) for sampled parity and CPU timing."""
    rng = np.random.default_rng(seed)
    n = min(n, receivers.shape[0])
    return np.sort(rng.choice(receivers.shape[0], size=n, replace=False))
