"""Python front end of the FP64 CPU oracle (``gbt_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this module; the library never does.  It
shares no code with the CUDA path.  Inputs come from
``paper_2501_13382_gb300.inputs`` (pure data), outputs are numpy arrays.

Functions and the passages they follow (arXiv 2501.13382):
  fan_fibonacci  -- the ray fan over take-off angles (Sec. 3.3, Eq. 3's gamma1, gamma2)
  fan_latlong    -- the paper's grid of elevation x azimuth take-off angles, with
                    each ray's cell solid angle as its weight
  trace          -- straight-ray tracing with specular reflection (Sec. 2, Sec. 3.1)
  gbs_sum        -- Gaussian beam summation, Eq. 3 with the beam of Eq. 1 / Eq. 2
  gbs_adjoint    -- gradient of a real loss through gbs_sum
  synthesize     -- time signals from per-frequency fields (superposition of the
                    time-harmonic fields of Eq. 1 under the exp(-i omega t) convention)
  air_absorption, delany_bazley, plane_wave_reflection, incidence_cos, path_factor
                 -- propagation losses for the atmospheric conditions and surface flow
                    impedance of the paper's input tables (Sec. 4.5, Tables 2-3), which
                    give no formula: ISO 9613-1 absorption of air, Delany-Bazley impedance
                    and the plane-wave reflection factor of a locally reacting surface
Parity unpinned (definitions with no external check): the Fibonacci variant,
the beam-parameter rule, the cutoff C and the window choice.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

T_MIN = 1e-9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _open(path):
    lib = C.CDLL(path)
    lib.orc_count_kept.restype = C.c_int64
    lib.orc_num_threads.restype = C.c_int
    for fn in ("orc_air_absorption_db", "orc_air_absorption_np"):
        getattr(lib, fn).restype = C.c_double
        getattr(lib, fn).argtypes = [C.c_double] * 4
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _open(_LIB)
    return _lib


class use_library:
    """Context manager: route this module's calls to another build of the oracle
    source (the mutation tests compile deliberately broken copies on the CPU)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        _lib = _open(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_source(src_text: str, out_path: str) -> str:
    """Compile oracle C source text with the oracle's flags (used by mutation tests)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", c_path, "-o", out_path, "-lm"], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class _Scene(C.Structure):
    _fields_ = [("ground", C.c_int), ("ground_z", C.c_double), ("ground_material", C.c_int),
                ("n_tri", C.c_int64), ("tri", C.c_void_p), ("tri_material", C.c_void_p),
                ("tri_face", C.c_void_p)]


class _Segs(C.Structure):
    _fields_ = [("n_seg", C.c_int64), ("o", C.c_void_p), ("t", C.c_void_p), ("L", C.c_void_p),
                ("s0", C.c_void_p), ("ray", C.c_void_p), ("depth", C.c_void_p),
                ("bmat", C.c_void_p)]


class _SumArgs(C.Structure):
    _fields_ = [("c", C.c_double), ("n_freq", C.c_int), ("freq", C.c_void_p), ("b", C.c_void_p),
                ("b_mask", C.c_void_p), ("cutoff", C.c_double), ("window", C.c_int),
                ("absorb", C.c_void_p), ("seg_factor", C.c_void_p)]


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else C.c_void_p(0)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def fan_fibonacci(n: int) -> np.ndarray:
    d = np.empty((n, 3), np.float64)
    _load().orc_fan_fibonacci(C.c_int64(n), _p(d))
    return d


FAN_FIBONACCI, FAN_LATLONG = 0, 2


def fan_latlong(n_theta: int, n_phi: int, theta_deg=(0.0, 180.0), phi_deg=(0.0, 360.0)):
    """Grid of take-off angles (Sec. 3.3; the input tables' elevation and azimuth
    ranges): directions (N, 3) at the cell centres and per-ray cell solid angles (N,)."""
    n = int(n_theta) * int(n_phi)
    d = np.empty((n, 3), np.float64)
    w = np.empty(n, np.float64)
    _load().orc_fan_latlong(C.c_int64(n_theta), C.c_int64(n_phi), C.c_double(theta_deg[0]),
                            C.c_double(theta_deg[1]), C.c_double(phi_deg[0]),
                            C.c_double(phi_deg[1]), _p(d), _p(w))
    return d, w


def fan(source):
    """Directions and weights of a source's fan: Fibonacci (4 pi / N each) or the
    latitude-longitude grid (n_theta rows of n_rays / n_theta azimuths)."""
    n = int(source.n_rays)
    if getattr(source, "fan", FAN_FIBONACCI) == FAN_LATLONG:
        nt = int(source.n_theta)
        assert nt >= 1 and n % nt == 0, "n_rays must be a multiple of n_theta"
        return fan_latlong(nt, n // nt, source.theta_deg, source.phi_deg)
    return fan_fibonacci(n), default_weight(n)


@dataclass
class Trace:
    n_rays: int
    ray_off: np.ndarray   # (N+1,) int64
    cnt: np.ndarray       # (N,) int32
    o: np.ndarray         # (S,3)
    t: np.ndarray         # (S,3)
    L: np.ndarray         # (S,)
    s0: np.ndarray        # (S,)
    ray: np.ndarray       # (S,) int32
    depth: np.ndarray     # (S,) int32
    bmat: np.ndarray      # (S,) int32
    hit: np.ndarray       # (S,) int32  0 ground, 1+k triangle k, -1 none
    w: np.ndarray | None = None   # (N_fan,) the fan's ray weights (None: 4 pi / N)

    @property
    def n_seg(self) -> int:
        return int(self.L.shape[0])

    def subset_rays(self, lo: int, hi: int) -> "Trace":
        a, b = int(self.ray_off[lo]), int(self.ray_off[hi])
        return Trace(hi - lo, self.ray_off[lo:hi + 1] - a, self.cnt[lo:hi], self.o[a:b],
                     self.t[a:b], self.L[a:b], self.s0[a:b], self.ray[a:b], self.depth[a:b],
                     self.bmat[a:b], self.hit[a:b], self.w)


def _scene_struct(scene):
    tri = np.ascontiguousarray(scene.tri_xyz.reshape(-1, 9), np.float64)
    mat = np.ascontiguousarray(scene.tri_material, np.int32)
    face = np.ascontiguousarray(scene.tri_face, np.int32)
    s = _Scene(int(scene.ground), float(scene.ground_z), int(scene.ground_material),
               int(tri.shape[0]), _p(tri), _p(mat), _p(face))
    return s, (tri, mat, face)


def trace(scene, source, dirs: np.ndarray | None = None) -> Trace:
    lib = _load()
    n = int(source.n_rays)
    w = None
    if dirs is None:
        dirs, w = fan(source)
    dirs = np.ascontiguousarray(dirs, np.float64)
    R = int(source.max_reflections)
    cap = n * (R + 1)
    cnt = np.zeros(n, np.int32)
    o = np.zeros((cap, 3)); t = np.zeros((cap, 3)); L = np.zeros(cap); s0 = np.zeros(cap)
    bm = np.zeros(cap, np.int32); hit = np.zeros(cap, np.int32)
    sc, keep = _scene_struct(scene)
    src = np.ascontiguousarray(source.pos, np.float64)
    lib.orc_trace(C.byref(sc), _p(src), _p(dirs), C.c_int64(n), C.c_int(R),
                  C.c_double(source.max_path), C.c_double(T_MIN), _p(cnt), _p(o), _p(t),
                  _p(L), _p(s0), _p(bm), _p(hit))
    rows = (np.arange(n)[:, None] * (R + 1) + np.arange(R + 1)[None, :])
    valid = np.arange(R + 1)[None, :] < cnt[:, None]
    idx = rows[valid]
    ray_off = np.zeros(n + 1, np.int64)
    ray_off[1:] = np.cumsum(cnt)
    ray = np.repeat(np.arange(n, dtype=np.int32), cnt)
    depth = (np.arange(idx.shape[0]) - ray_off[ray]).astype(np.int32)
    return Trace(n, ray_off, cnt, o[idx], t[idx], L[idx], s0[idx], ray, depth, bm[idx], hit[idx], w)


def _segs_struct(tr: Trace):
    arrs = [np.ascontiguousarray(a) for a in
            (tr.o, tr.t, tr.L, tr.s0, tr.ray.astype(np.int32), tr.depth.astype(np.int32),
             tr.bmat.astype(np.int32))]
    s = _Segs(tr.n_seg, *[_p(a) for a in arrs])
    return s, arrs


def _args_struct(c, freqs, b, cutoff, window, b_mask, absorption=None, seg_factor=None):
    fr = np.ascontiguousarray(freqs, np.float64)
    bb = np.ascontiguousarray(b, np.float64)
    bmk = None if b_mask is None else np.ascontiguousarray(b_mask, np.float64)
    ab = None if absorption is None else np.ascontiguousarray(absorption, np.float64)
    sf = None
    if seg_factor is not None:
        sf = np.ascontiguousarray(np.stack([np.real(seg_factor), np.imag(seg_factor)], -1),
                                  np.float64)
    a = _SumArgs(float(c), int(fr.shape[0]), _p(fr), _p(bb), _p(bmk), float(cutoff), int(window),
                 _p(ab), _p(sf))
    return a, (fr, bb, bmk, ab, sf)


# ------------------------------------------------------- propagation losses --

def air_absorption_db(freqs, temperature_c: float = 20.0, humidity_pct: float = 70.0,
                      pressure_kpa: float = 101.325) -> np.ndarray:
    """Pure-tone attenuation coefficient of air, dB per metre (ISO 9613-1)."""
    lib = _load()
    return np.array([lib.orc_air_absorption_db(float(f), float(temperature_c),
                                               float(humidity_pct), float(pressure_kpa))
                     for f in np.atleast_1d(freqs)])


def air_absorption(freqs, temperature_c: float = 20.0, humidity_pct: float = 70.0,
                   pressure_kpa: float = 101.325) -> np.ndarray:
    """Pressure-amplitude decay rate of air a (Np/m; the amplitude falls as exp(-a s)),
    ISO 9613-1.  The paper's cases use 20 C, 70 % and 1 atm (Tables 2-3)."""
    lib = _load()
    return np.array([lib.orc_air_absorption_np(float(f), float(temperature_c),
                                               float(humidity_pct), float(pressure_kpa))
                     for f in np.atleast_1d(freqs)])


def delany_bazley(freq: float, sigma_kpa: float) -> complex:
    """Normalised surface impedance Z / (rho c) of a porous surface of effective flow
    resistivity sigma (kPa s m^-2), Delany and Bazley's model, exp(-i omega t)."""
    z = np.zeros(2)
    _load().orc_delany_bazley_z(C.c_double(freq), C.c_double(sigma_kpa), _p(z))
    return complex(z[0], z[1])


def plane_wave_reflection(Z: complex, cos_theta: float) -> complex:
    """(Z cos theta - 1) / (Z cos theta + 1): plane wave on a locally reacting surface."""
    z = np.array([complex(Z).real, complex(Z).imag])
    r = np.zeros(2)
    _load().orc_plane_wave_reflection_r(_p(z), C.c_double(cos_theta), _p(r))
    return complex(r[0], r[1])


def incidence_cos(scene, tr: "Trace") -> np.ndarray:
    """Per segment: cosine of the incidence angle at the reflection that starts it (1 for
    each ray's first segment)."""
    sc, keep = _scene_struct(scene)
    t = np.ascontiguousarray(tr.t, np.float64)
    dep = np.ascontiguousarray(tr.depth, np.int32)
    hit = np.ascontiguousarray(tr.hit, np.int32)
    out = np.zeros(tr.n_seg)
    _load().orc_incidence_cos(C.byref(sc), C.c_int64(tr.n_seg), _p(t), _p(dep), _p(hit), _p(out))
    return out


def path_factor(scene, tr: "Trace", sigma, freqs) -> np.ndarray:
    """Complex (F, S): per frequency and segment, the product of the plane-wave reflection
    factors of the porous surfaces (sigma[m] > 0, Delany-Bazley) met before the segment."""
    cosi = incidence_cos(scene, tr)
    sg = np.ascontiguousarray(sigma, np.float64)
    fr = np.ascontiguousarray(freqs, np.float64)
    dep = np.ascontiguousarray(tr.depth, np.int32)
    bm = np.ascontiguousarray(tr.bmat, np.int32)
    out = np.zeros((fr.shape[0], tr.n_seg, 2))
    _load().orc_path_factor(C.c_int64(tr.n_seg), _p(dep), _p(bm), _p(cosi), _p(sg), _p(fr),
                            C.c_int(fr.shape[0]), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def _losses(tr, freqs, absorption, sigma, scene):
    seg_factor = None
    if sigma is not None:
        assert scene is not None, "porous surfaces need the scene (normals at the reflections)"
        seg_factor = path_factor(scene, tr, sigma, freqs)
    return absorption, seg_factor


def default_weight(n_rays: int) -> np.ndarray:
    return np.full(n_rays, 4.0 * np.pi / n_rays)


def _weights(tr: Trace, weight):
    if weight is not None:
        return np.ascontiguousarray(weight, np.float64)
    return default_weight(tr.n_rays) if tr.w is None else np.ascontiguousarray(tr.w, np.float64)


def gbs_sum(tr: Trace, receivers: np.ndarray, freqs, b, c: float, gamma, weight=None,
            window: int = 1, cutoff: float = 16.0, b_mask=None, absorption=None, sigma=None,
            scene=None) -> np.ndarray:
    """Complex pressure p[f, r] (complex128).  absorption: per-frequency amplitude decay of
    air (Np/m); sigma: per-material flow resistivity (kPa s m^-2, <= 0 hard), which needs
    the scene the trace came from."""
    lib = _load()
    recv = np.ascontiguousarray(np.asarray(receivers, np.float32).astype(np.float64))
    nr = recv.shape[0]
    gam = np.ascontiguousarray(gamma, np.float64)
    w = _weights(tr, weight)
    segs, k1 = _segs_struct(tr)
    args, k2 = _args_struct(c, freqs, b, cutoff, window, b_mask,
                            *_losses(tr, freqs, absorption, sigma, scene))
    out = np.zeros((len(freqs), nr, 2), np.float64)
    lib.orc_sum(C.byref(segs), C.byref(args), _p(recv), C.c_int64(nr), _p(gam), _p(w), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def gbs_adjoint(tr: Trace, receivers, freqs, b, c, gamma, g, weight=None, window: int = 1,
                cutoff: float = 16.0, b_mask=None, absorption=None, sigma=None, scene=None):
    """Gradients (d gamma[M], d weight[N], d b[F]) of a real loss with dL/dp = g (F, Nr)."""
    lib = _load()
    recv = np.ascontiguousarray(np.asarray(receivers, np.float32).astype(np.float64))
    nr = recv.shape[0]
    gam = np.ascontiguousarray(gamma, np.float64)
    w = _weights(tr, weight)
    gg = np.ascontiguousarray(np.stack([np.real(g), np.imag(g)], -1), np.float64)
    segs, k1 = _segs_struct(tr)
    args, k2 = _args_struct(c, freqs, b, cutoff, window, b_mask,
                            *_losses(tr, freqs, absorption, sigma, scene))
    dg = np.zeros(gam.shape[0]); dw = np.zeros(tr.n_rays); db = np.zeros(len(freqs))
    lib.orc_sum_adjoint(C.byref(segs), C.byref(args), _p(recv), C.c_int64(nr), _p(gam),
                        C.c_int(gam.shape[0]), _p(w), C.c_int64(tr.n_rays), _p(gg), _p(dg),
                        _p(dw), _p(db))
    return dg, dw, db


def synthesize(p, freqs, amp, t0: float, dt: float, n_t: int) -> np.ndarray:
    """Time signals of a superposition of time-harmonic fields (exp(-i omega t) convention):
    h[n, r] = Re sum_f amp_f p[f, r] exp(-i 2 pi freq_f (t0 + n dt)), in FP64; with
    amp_f = S(freq_f) df this is the Fourier synthesis of a source spectrum S."""
    p = np.asarray(p, np.complex128)
    t = t0 + dt * np.arange(int(n_t), dtype=np.float64)
    ph = np.exp(-2j * np.pi * np.outer(t, np.asarray(freqs, np.float64)))      # (n_t, F)
    return np.real((ph * np.asarray(amp, np.complex128)[None, :]) @ p)


def count_kept(tr: Trace, receivers, freqs, b, c, window=1, cutoff=16.0) -> int:
    lib = _load()
    recv = np.ascontiguousarray(np.asarray(receivers, np.float32).astype(np.float64))
    segs, k1 = _segs_struct(tr)
    args, k2 = _args_struct(c, freqs, b, cutoff, window, None)
    return int(lib.orc_count_kept(C.byref(segs), C.byref(args), _p(recv), C.c_int64(recv.shape[0])))


def solve(workload, source_index: int = 0, receivers=None, weight=None, gamma=None):
    """Trace one source of a workload and sum at its receivers (or a given subset)."""
    src = workload.sources[source_index]
    tr = trace(workload.scene, src)
    recv = workload.receivers if receivers is None else receivers
    gam = workload.scene.gamma if gamma is None else gamma
    return tr, gbs_sum(tr, recv, workload.freqs, workload.beam_b[source_index],
                       workload.scene.c, gam, weight, workload.window, workload.cutoff)
