"""ctypes binding of libgbt (include/gbt.h) plus a thin torch front end.

The ``gbt_*`` functions below mirror the C ABI one to one: they marshal
arguments, call the library and raise ``GBTError`` on a non-zero status.
Every step of the computation runs in the library's CUDA kernels; torch only
provides device memory and the current stream.  Importing this module never
touches the GPU; the first call loads ``libgbt.so`` and fails loudly if it has
not been built (``python -m paper_2501_13382_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbt.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "gbt.h")

MAX_FREQ = 16
WINDOW_SEGMENT, WINDOW_LINE = 0, 1
BATCH_AUTO, BATCH_FUSED, BATCH_CONCURRENT = 0, 1, 2
PRECISION_F32, PRECISION_F64 = 0, 1
FAN_FIBONACCI, FAN_EXPLICIT, FAN_LATLONG = 0, 1, 2
ACCEL_AUTO, ACCEL_BVH, ACCEL_LINEAR = 0, 1, 2

STATUS_NAMES = {0: "GBT_OK", 1: "GBT_ERR_INVALID_ARG", 2: "GBT_ERR_OOM", 3: "GBT_ERR_CUDA",
                4: "GBT_ERR_TIMEOUT", 5: "GBT_ERR_DEVICE_STATUS", 6: "GBT_ERR_UNSUPPORTED"}


class GBTError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gbt_allocator(C.Structure):
    _fields_ = [("alloc", C.c_void_p), ("free", C.c_void_p), ("ctx", C.c_void_p)]


class gbt_scene_desc(C.Structure):
    _fields_ = [("c", C.c_double), ("ground_enabled", C.c_int32), ("ground_material", C.c_int32),
                ("ground_z", C.c_double), ("n_tri", C.c_int64), ("tri_xyz", C.c_void_p),
                ("tri_material", C.c_void_p), ("tri_face", C.c_void_p),
                ("n_materials", C.c_int32), ("accel", C.c_int32)]


class gbt_source_desc(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("n_rays", C.c_int64), ("ray_begin", C.c_int64),
                ("ray_count", C.c_int64), ("fan", C.c_int32), ("max_reflections", C.c_int32),
                ("dirs", C.c_void_p), ("max_path", C.c_double), ("n_theta", C.c_int64),
                ("theta_deg", C.c_double * 2), ("phi_deg", C.c_double * 2)]


class gbt_segments(C.Structure):
    _fields_ = [("n_segments", C.c_int64), ("ray_off", C.c_void_p), ("seg_o", C.c_void_p),
                ("seg_t", C.c_void_p), ("seg_L", C.c_void_p), ("seg_s0", C.c_void_p),
                ("seg_bmat", C.c_void_p), ("seg_hit", C.c_void_p)]


class gbt_trace_info(C.Structure):
    _fields_ = [("n_fan", C.c_int64), ("ray_begin", C.c_int64), ("n_rays", C.c_int64),
                ("seg_capacity", C.c_int64), ("n_segments", C.c_int64),
                ("ray_off", C.c_void_p), ("seg_o", C.c_void_p), ("seg_t", C.c_void_p),
                ("seg_L", C.c_void_p), ("seg_s0", C.c_void_p), ("seg_ray", C.c_void_p),
                ("seg_depth", C.c_void_p), ("seg_bmat", C.c_void_p), ("seg_hit", C.c_void_p)]


class gbt_sum_args(C.Structure):
    _fields_ = [("recv", C.c_void_p), ("n_recv", C.c_int64), ("recv_order", C.c_void_p),
                ("n_freq", C.c_int32), ("window", C.c_int32),
                ("freq_hz", C.c_double * MAX_FREQ), ("beam_b", C.c_double * MAX_FREQ),
                ("gamma", C.c_void_p), ("ray_weight", C.c_void_p), ("out", C.c_void_p),
                ("cutoff", C.c_double), ("precision", C.c_int32), ("accumulate", C.c_int32),
                ("seg_split", C.c_int32), ("tile_cull", C.c_int32),
                ("max_device_bytes", C.c_int64), ("absorption", C.c_double * MAX_FREQ),
                ("flow_resistivity", C.c_void_p)]


class gbt_sum_stats(C.Structure):
    _fields_ = [("n_segments", C.c_int64), ("pairs", C.c_int64), ("pairs_prefiltered", C.c_int64),
                ("triples_kept", C.c_int64), ("pairs_tested", C.c_int64)]


class gbt_batch_desc(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("traces", C.c_void_p), ("args", C.c_void_p),
                ("use_graph", C.c_int32), ("autotune", C.c_int32), ("form", C.c_int32)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "gbt_version": (C.c_int32, []),
    "gbt_last_error": (C.c_char_p, []),
    "gbt_set_allocator": (C.c_int, [C.c_void_p]),
    "gbt_scene_create": (C.c_int, [C.POINTER(gbt_scene_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "gbt_scene_destroy": (C.c_int, [C.c_void_p]),
    "gbt_trace": (C.c_int, [C.c_void_p, C.POINTER(gbt_source_desc), C.c_void_p,
                            C.POINTER(C.c_void_p)]),
    "gbt_trace_info_get": (C.c_int, [C.c_void_p, C.POINTER(gbt_trace_info)]),
    "gbt_trace_import": (C.c_int, [C.c_void_p, C.POINTER(gbt_source_desc), C.POINTER(gbt_segments),
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    "gbt_trace_destroy": (C.c_int, [C.c_void_p]),
    "gbt_sum": (C.c_int, [C.c_void_p, C.POINTER(gbt_sum_args), C.c_void_p]),
    "gbt_synthesize": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.c_double, C.c_double, C.c_int64, C.c_void_p, C.c_int32,
                                 C.c_void_p]),
    "gbt_recv_order": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "gbt_air_absorption": (C.c_int, [C.c_int32, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                     C.c_void_p]),
    "gbt_recv_order_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "gbt_sum_backward": (C.c_int, [C.c_void_p, C.POINTER(gbt_sum_args), C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "gbt_solve": (C.c_int, [C.c_void_p, C.POINTER(gbt_source_desc), C.POINTER(gbt_sum_args),
                            C.c_void_p]),
    "gbt_batch_create": (C.c_int, [C.POINTER(gbt_batch_desc), C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "gbt_batch_submit": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gbt_batch_destroy": (C.c_int, [C.c_void_p]),
    "gbt_sync": (C.c_int, [C.c_void_p]),
    "gbt_selftest_timeout": (C.c_int, [C.c_int64, C.c_void_p]),
    "gbt_timing_enable": (C.c_int, [C.c_int32]),
    "gbt_list_capacity_set": (C.c_int, [C.c_int64]),
    "gbt_timing_read": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int32]),
    "gbt_launches_read": (C.c_int, [C.POINTER(C.c_int64), C.c_int32]),
    "gbt_sum_stats_get": (C.c_int, [C.c_void_p, C.POINTER(gbt_sum_args), C.POINTER(gbt_sum_stats),
                                    C.c_void_p]),
}


def load(path: Optional[str] = None):
    """Load libgbt.so (once).  Raises if the library has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libgbt.so not found at {p}: build it with "
                                   "`python -m paper_2501_13382_gb300.build` (no CPU fallback)")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def declared_functions(header: str = HEADER_PATH) -> list:
    """Names of the functions include/gbt.h declares."""
    import re
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gbt_[a-z_0-9]+)\s*\(",
                                 txt, flags=re.M)))


def _check(status: int, where: str):
    if status != 0:
        msg = load().gbt_last_error().decode(errors="replace")
        raise GBTError(status, where, msg)


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


# ------------------------------------------------------------ raw C calls --

def gbt_version() -> int:
    return int(load().gbt_version())


def gbt_scene_create(desc: gbt_scene_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().gbt_scene_create(C.byref(desc), C.c_void_p(stream), C.byref(h)), "gbt_scene_create")
    return h.value


def gbt_scene_destroy(h: int):
    _check(load().gbt_scene_destroy(C.c_void_p(h)), "gbt_scene_destroy")


def gbt_trace(scene: int, src: gbt_source_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().gbt_trace(C.c_void_p(scene), C.byref(src), C.c_void_p(stream), C.byref(h)),
           "gbt_trace")
    return h.value


def gbt_trace_import(scene: int, src: gbt_source_desc, segs: gbt_segments, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().gbt_trace_import(C.c_void_p(scene), C.byref(src), C.byref(segs),
                                   C.c_void_p(stream), C.byref(h)), "gbt_trace_import")
    return h.value


def gbt_trace_info_get(trace: int) -> gbt_trace_info:
    info = gbt_trace_info()
    _check(load().gbt_trace_info_get(C.c_void_p(trace), C.byref(info)), "gbt_trace_info_get")
    return info


def gbt_trace_destroy(trace: int):
    _check(load().gbt_trace_destroy(C.c_void_p(trace)), "gbt_trace_destroy")


def gbt_sum(trace: int, args: gbt_sum_args, stream: int = 0):
    _check(load().gbt_sum(C.c_void_p(trace), C.byref(args), C.c_void_p(stream)), "gbt_sum")


def gbt_air_absorption(freqs, temperature_c: float = 20.0, humidity_pct: float = 70.0,
                       pressure_kpa: float = 101.325) -> np.ndarray:
    """Amplitude decay rate of air (Np/m) per frequency, ISO 9613-1 (host computation)."""
    fr = np.ascontiguousarray(np.atleast_1d(np.asarray(freqs, np.float64)))
    out = np.zeros_like(fr)
    _check(load().gbt_air_absorption(int(fr.shape[0]), fr.ctypes.data, float(temperature_c),
                                     float(humidity_pct), float(pressure_kpa), out.ctypes.data),
           "gbt_air_absorption")
    return out


air_absorption = gbt_air_absorption


def gbt_recv_order(recv_ptr: int, n: int, order_ptr: int, stream: int = 0):
    _check(load().gbt_recv_order(C.c_void_p(recv_ptr), C.c_int64(n), C.c_void_p(order_ptr),
                                 C.c_void_p(stream)), "gbt_recv_order")


def gbt_recv_order_noalloc(recv_ptr: int, n: int, order_ptr: int, stream: int = 0):
    """gbt_recv_order without any device allocation (fixed scratch inside the library;
    n <= 1,048,576; calls that overlap on the GPU race on that scratch)."""
    _check(load().gbt_recv_order_noalloc(C.c_void_p(recv_ptr), C.c_int64(n), C.c_void_p(order_ptr),
                                         C.c_void_p(stream)), "gbt_recv_order_noalloc")


def gbt_sum_backward(trace: int, args: gbt_sum_args, grad_out: int, grad_gamma: int,
                     grad_w: int, grad_b: int, stream: int = 0):
    _check(load().gbt_sum_backward(C.c_void_p(trace), C.byref(args), C.c_void_p(grad_out),
                                   C.c_void_p(grad_gamma), C.c_void_p(grad_w), C.c_void_p(grad_b),
                                   C.c_void_p(stream)), "gbt_sum_backward")


def gbt_solve(scene: int, src: gbt_source_desc, args: gbt_sum_args, stream: int = 0):
    _check(load().gbt_solve(C.c_void_p(scene), C.byref(src), C.byref(args), C.c_void_p(stream)),
           "gbt_solve")


def gbt_batch_create(desc: gbt_batch_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().gbt_batch_create(C.byref(desc), C.c_void_p(stream), C.byref(h)),
           "gbt_batch_create")
    return h.value


def gbt_batch_submit(batch: int, stream: int = 0):
    _check(load().gbt_batch_submit(C.c_void_p(batch), C.c_void_p(stream)), "gbt_batch_submit")


def gbt_batch_destroy(batch: int):
    _check(load().gbt_batch_destroy(C.c_void_p(batch)), "gbt_batch_destroy")


def gbt_sync(stream: int = 0):
    _check(load().gbt_sync(C.c_void_p(stream)), "gbt_sync")


def gbt_selftest_timeout(spins: int, stream: int = 0):
    _check(load().gbt_selftest_timeout(C.c_int64(spins), C.c_void_p(stream)), "gbt_selftest_timeout")


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_allocator_keepalive = []


def gbt_set_allocator(alloc=None, free=None):
    """Install Python callables alloc(bytes, stream) -> int and free(ptr, stream) as the
    library's device allocator (None restores the default stream-ordered pool)."""
    if alloc is None:
        _check(load().gbt_set_allocator(None), "gbt_set_allocator")
        _allocator_keepalive.clear()
        return
    a = ALLOC_FN(lambda n, stream, ctx: alloc(int(n), stream or 0) or None)
    f = FREE_FN(lambda ptr, stream, ctx: free(int(ptr or 0), stream or 0))
    desc = gbt_allocator(C.cast(a, C.c_void_p).value, C.cast(f, C.c_void_p).value, None)
    _allocator_keepalive[:] = [a, f, desc]
    _check(load().gbt_set_allocator(C.byref(desc)), "gbt_set_allocator")


def use_torch_allocator():
    """Route the library's device memory through torch's caching allocator."""
    import torch

    def alloc(n, stream):
        return torch.cuda.caching_allocator_alloc(n, torch.cuda.current_device(), stream or None)

    def free(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)
    gbt_set_allocator(alloc, free)


def gbt_list_capacity_set(entries: int):
    """Bound on the tile lists' entries for the sums planned afterwards (0: the default);
    tiles whose lists do not fit test every segment, with the same field."""
    _check(load().gbt_list_capacity_set(C.c_int64(int(entries))), "gbt_list_capacity_set")


def gbt_timing_enable(enable: bool):
    _check(load().gbt_timing_enable(C.c_int32(1 if enable else 0)), "gbt_timing_enable")


def gbt_timing_read(reset: bool = True):
    n = C.c_int64()
    ms = C.c_double()
    _check(load().gbt_timing_read(C.byref(n), C.byref(ms), C.c_int32(1 if reset else 0)),
           "gbt_timing_read")
    return int(n.value), float(ms.value)


def gbt_launches_read(reset: bool = True) -> int:
    """Kernels the library has launched (since the last reset)."""
    n = C.c_int64(0)
    _check(load().gbt_launches_read(C.byref(n), C.c_int32(1 if reset else 0)), "gbt_launches_read")
    return int(n.value)


def gbt_sum_stats_get(trace: int, args: gbt_sum_args, stream: int = 0) -> gbt_sum_stats:
    st = gbt_sum_stats()
    _check(load().gbt_sum_stats_get(C.c_void_p(trace), C.byref(args), C.byref(st),
                                    C.c_void_p(stream)), "gbt_sum_stats_get")
    return st


# ------------------------------------------------------------ torch layer --

class Scene:
    """Device-resident scene built from ``inputs.Scene``."""

    def __init__(self, scene, accel: int = ACCEL_AUTO):
        self.src = scene
        tri = np.ascontiguousarray(scene.tri_xyz.reshape(-1, 9), np.float64)
        mat = np.ascontiguousarray(scene.tri_material, np.int32)
        face = np.ascontiguousarray(scene.tri_face, np.int32)
        d = gbt_scene_desc(float(scene.c), int(scene.ground), int(scene.ground_material),
                           float(scene.ground_z), int(tri.shape[0]),
                           tri.ctypes.data if tri.size else 0,
                           mat.ctypes.data if mat.size else 0,
                           face.ctypes.data if face.size else 0, int(scene.n_materials),
                           int(accel))
        self.handle = gbt_scene_create(d, _stream_ptr())
        self.c = float(scene.c)
        self.n_materials = int(scene.n_materials)

    def close(self):
        if getattr(self, "handle", None):
            gbt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def source_desc(source, ray_begin: int = 0, ray_count: int = 0, dirs=None) -> gbt_source_desc:
    s = gbt_source_desc()
    s.pos[:] = [float(v) for v in source.pos]
    s.n_rays = int(source.n_rays)
    s.ray_begin = int(ray_begin)
    s.ray_count = int(ray_count)
    s.fan = FAN_EXPLICIT if dirs is not None else int(getattr(source, "fan", FAN_FIBONACCI))
    s.max_reflections = int(source.max_reflections)
    s.dirs = _ptr(dirs)
    s.max_path = float(source.max_path)
    if s.fan == FAN_LATLONG:
        s.n_theta = int(source.n_theta)
        s.theta_deg[:] = [float(v) for v in source.theta_deg]
        s.phi_deg[:] = [float(v) for v in source.phi_deg]
    return s


class _CudaView:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2, "strides": None}


class Trace:
    """Traced fan (CSR of segments) living on the device."""

    def __init__(self, scene: Scene, source, ray_begin: int = 0, ray_count: int = 0, dirs=None,
                 segments: dict | None = None):
        """Traces `source` through `scene`, or, with `segments` (device tensors in the layout
        of `segments()`: ray_off, o, t, L, s0, bmat, optional hit), wraps a segment list
        computed elsewhere (gbt_trace_import)."""
        self.scene = scene
        self.source = source
        self._dirs = dirs
        self.ray_begin, self.ray_count = int(ray_begin), int(ray_count)
        desc = source_desc(source, ray_begin, ray_count, dirs)
        if segments is None:
            self.handle = gbt_trace(scene.handle, desc, _stream_ptr())
        else:
            sg = {k: v.contiguous() for k, v in segments.items() if k != "n_segments"}
            s = gbt_segments(int(sg["L"].shape[0]), _ptr(sg["ray_off"]), _ptr(sg["o"]),
                             _ptr(sg["t"]), _ptr(sg["L"]), _ptr(sg["s0"]), _ptr(sg["bmat"]),
                             _ptr(sg.get("hit")))
            self.handle = gbt_trace_import(scene.handle, desc, s, _stream_ptr())
        self.n_fan = int(source.n_rays)

    def save(self, path: str):
        """Writes the segment list and the source parameters to an .npz file (synchronises),
        so that sums can be rerun later without tracing (`Trace.load`)."""
        sg = {k: v.cpu().numpy() for k, v in self.segments().items() if k != "n_segments"}
        s = self.source
        np.savez(path, pos=np.asarray(s.pos, np.float64), n_rays=s.n_rays,
                 max_reflections=s.max_reflections, max_path=s.max_path,
                 fan=int(getattr(s, "fan", FAN_FIBONACCI)), n_theta=int(getattr(s, "n_theta", 0)),
                 theta_deg=np.asarray(getattr(s, "theta_deg", (0.0, 180.0)), np.float64),
                 phi_deg=np.asarray(getattr(s, "phi_deg", (0.0, 360.0)), np.float64),
                 ray_begin=self.ray_begin, ray_count=self.ray_count, **sg)

    @classmethod
    def load(cls, scene: Scene, path: str) -> "Trace":
        """A trace handle over a segment list written by `save` (gbt_trace_import)."""
        import torch
        from types import SimpleNamespace
        z = np.load(path)
        fan = int(z["fan"])
        src = SimpleNamespace(pos=z["pos"], n_rays=int(z["n_rays"]),
                              max_reflections=int(z["max_reflections"]),
                              max_path=float(z["max_path"]),
                              fan=FAN_FIBONACCI if fan == FAN_EXPLICIT else fan,
                              n_theta=int(z["n_theta"]), theta_deg=tuple(z["theta_deg"]),
                              phi_deg=tuple(z["phi_deg"]))
        seg = {k: torch.as_tensor(z[k], device="cuda")
               for k in ("ray_off", "o", "t", "L", "s0", "bmat", "hit")}
        return cls(scene, src, int(z["ray_begin"]), int(z["ray_count"]), segments=seg)

    def info(self) -> gbt_trace_info:
        return gbt_trace_info_get(self.handle)

    def segments(self) -> dict:
        """Copies of the CSR arrays as torch tensors (synchronises)."""
        import torch
        i = self.info()
        n = int(i.n_segments)
        nr = int(i.n_rays)

        def view(ptr, shape, typ):
            if int(np.prod(shape)) == 0:
                return torch.zeros(shape, dtype={"<f8": torch.float64, "<i4": torch.int32}[typ],
                                   device="cuda")
            return torch.as_tensor(_CudaView(ptr, shape, typ), device="cuda").clone()

        return {"n_segments": n, "ray_off": view(i.ray_off, (nr + 1,), "<i4"),
                "o": view(i.seg_o, (n, 3), "<f8"), "t": view(i.seg_t, (n, 3), "<f8"),
                "L": view(i.seg_L, (n,), "<f8"), "s0": view(i.seg_s0, (n,), "<f8"),
                "ray": view(i.seg_ray, (n,), "<i4"), "depth": view(i.seg_depth, (n,), "<i4"),
                "bmat": view(i.seg_bmat, (n,), "<i4"), "hit": view(i.seg_hit, (n,), "<i4")}

    def close(self):
        if getattr(self, "handle", None):
            gbt_trace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def recv_order(recv) -> "torch.Tensor":
    import torch
    n = int(recv.shape[0])
    order = torch.empty(n, dtype=torch.int32, device=recv.device)
    gbt_recv_order(_ptr(recv), n, _ptr(order), _stream_ptr())
    return order


def sum_args(recv, freqs: Sequence[float], beam_b: Sequence[float], gamma, out,
             ray_weight=None, order=None, window: int = WINDOW_LINE, cutoff: float = 16.0,
             precision: int = PRECISION_F32, accumulate: bool = False, seg_split: int = 0,
             max_device_bytes: int = 0, tile_cull: bool = False, absorption=None,
             flow_resistivity=None) -> gbt_sum_args:
    a = gbt_sum_args()
    a.recv = _ptr(recv)
    a.n_recv = int(recv.shape[0]) if recv is not None else 0
    a.recv_order = _ptr(order)
    a.n_freq = len(freqs)
    a.window = int(window)
    for f, (fr, b) in enumerate(zip(freqs, beam_b)):
        a.freq_hz[f] = float(fr)
        a.beam_b[f] = float(b)
    a.gamma = _ptr(gamma)
    a.ray_weight = _ptr(ray_weight)
    a.out = _ptr(out)
    a.cutoff = float(cutoff)
    a.precision = int(precision)
    a.accumulate = 1 if accumulate else 0
    a.seg_split = int(seg_split)
    a.tile_cull = 1 if tile_cull else 0
    a.max_device_bytes = int(max_device_bytes)
    if absorption is not None:
        ab = [float(v) for v in np.atleast_1d(absorption)]
        _require(len(ab) == len(freqs), "one absorption rate per frequency")
        for f, v in enumerate(ab):
            a.absorption[f] = v
    a.flow_resistivity = _ptr(flow_resistivity)
    return a


def _require(cond: bool, msg: str):
    if not cond:
        raise ValueError(msg)


def _check_sigma(flow_resistivity, n_materials: int):
    import torch
    if flow_resistivity is None:
        return
    _require(flow_resistivity.is_cuda and flow_resistivity.dtype == torch.float32
             and flow_resistivity.is_contiguous() and flow_resistivity.numel() == n_materials,
             f"flow_resistivity must be a contiguous float32 CUDA tensor of {n_materials} values")


def _check_tensors(recv, gamma, ray_weight, order, n_materials: int | None = None,
                   n_fan: int | None = None):
    """The library reads these device arrays by index (gamma per material, ray_weight per
    ray of the fan, order per receiver) and cannot see their sizes: check them here."""
    import torch
    _require(recv.is_cuda and recv.dtype == torch.float32 and recv.is_contiguous()
             and recv.dim() == 2 and recv.shape[1] == 3,
             "recv must be a contiguous float32 CUDA tensor of shape (n_recv, 3)")
    _require(gamma.is_cuda and gamma.dtype == torch.float32 and gamma.is_contiguous(),
             "gamma must be a contiguous float32 CUDA tensor")
    if n_materials is not None:
        _require(gamma.numel() == n_materials, f"gamma must hold {n_materials} coefficients")
    if ray_weight is not None:
        _require(ray_weight.is_cuda and ray_weight.dtype == torch.float32
                 and ray_weight.is_contiguous(), "ray_weight must be a contiguous float32 CUDA tensor")
        if n_fan is not None:
            _require(ray_weight.numel() == n_fan, f"ray_weight must hold {n_fan} weights")
    if order is not None:
        _require(order.is_cuda and order.dtype == torch.int32 and order.is_contiguous()
                 and order.numel() == recv.shape[0],
                 "order must be a contiguous int32 CUDA tensor with one entry per receiver")


def _check_out(out, nf: int, nr: int):
    import torch
    _require(out.is_cuda and out.dtype == torch.complex64 and out.is_contiguous(),
             "out must be a contiguous complex64 CUDA tensor")
    _require(tuple(out.shape) == (nf, nr), f"out must have shape ({nf}, {nr})")


def gbs_sum(trace: Trace, recv, freqs, beam_b, gamma, ray_weight=None, order=None,
            window: int = WINDOW_LINE, cutoff: float = 16.0, precision: int = PRECISION_F32,
            out=None, accumulate: bool = False, seg_split: int = 0, tile_cull: bool = False,
            absorption=None, flow_resistivity=None):
    """Complex pressure p[f, r] (torch complex64 on the device).  absorption: per-frequency
    amplitude decay rate of air (Np/m, see air_absorption); flow_resistivity: float32 CUDA
    tensor of per-material flow resistivities (kPa s m^-2, <= 0 hard).  Asynchronous:
    problems a kernel detects (a bounded wait that ran out) surface at gbt_sync."""
    import torch
    _check_tensors(recv, gamma, ray_weight, order, trace.scene.n_materials, trace.n_fan)
    _check_sigma(flow_resistivity, trace.scene.n_materials)
    nr = int(recv.shape[0])
    if out is None:
        out = torch.empty((len(freqs), nr), dtype=torch.complex64, device=recv.device)
    _check_out(out, len(freqs), nr)
    a = sum_args(recv, freqs, beam_b, gamma, out, ray_weight, order, window, cutoff, precision,
                 accumulate, seg_split, tile_cull=tile_cull, absorption=absorption,
                 flow_resistivity=flow_resistivity)
    gbt_sum(trace.handle, a, _stream_ptr())
    return out


def sum_stats(trace: Trace, recv, freqs, beam_b, gamma, ray_weight=None, order=None,
              window: int = WINDOW_LINE, cutoff: float = 16.0, tile_cull: bool = False) -> dict:
    _check_tensors(recv, gamma, ray_weight, order, trace.scene.n_materials, trace.n_fan)
    a = sum_args(recv, freqs, beam_b, gamma, None, ray_weight, order, window, cutoff,
                 tile_cull=tile_cull)
    st = gbt_sum_stats_get(trace.handle, a, _stream_ptr())
    return {"n_segments": st.n_segments, "pairs": st.pairs,
            "pairs_prefiltered": st.pairs_prefiltered, "triples_kept": st.triples_kept,
            "pairs_tested": st.pairs_tested}


def gbs_solve(scene: Scene, source, recv, freqs, beam_b, gamma, ray_weight=None, order=None,
              window: int = WINDOW_LINE, cutoff: float = 16.0, max_device_bytes: int = 0,
              out=None, accumulate: bool = False, tile_cull: bool = False, absorption=None,
              flow_resistivity=None):
    """Trace + sum of one source, chunked over rays under a device-byte budget."""
    import torch
    _check_tensors(recv, gamma, ray_weight, order, scene.n_materials, int(source.n_rays))
    _check_sigma(flow_resistivity, scene.n_materials)
    nr = int(recv.shape[0])
    if out is None:
        out = torch.empty((len(freqs), nr), dtype=torch.complex64, device=recv.device)
    _check_out(out, len(freqs), nr)
    a = sum_args(recv, freqs, beam_b, gamma, out, ray_weight, order, window, cutoff,
                 PRECISION_F32, accumulate, 0, max_device_bytes, tile_cull=tile_cull,
                 absorption=absorption, flow_resistivity=flow_resistivity)
    gbt_solve(scene.handle, source_desc(source), a, _stream_ptr())
    return out


class Batch:
    """Many (trace, receivers, frequencies) instances solved in one persistent launch.

    ``instances`` is a list of dicts with keys trace, recv, freqs, beam_b, gamma and
    optionally ray_weight, order, out (complex64 [F, Nr]); all share window and cutoff.
    ``submit()`` queues the whole batch (a CUDA graph replay after the first call when
    use_graph is set); results land in each instance's ``out``."""

    def __init__(self, instances, window: int = WINDOW_SEGMENT, cutoff: float = 16.0,
                 use_graph: bool = True, autotune: bool = False, tile_cull: bool = False,
                 form: int = BATCH_AUTO):
        import torch
        self.instances = []
        args = []
        for inst in instances:
            recv = inst["recv"]
            _check_tensors(recv, inst["gamma"], inst.get("ray_weight"), inst.get("order"),
                           inst["trace"].scene.n_materials, inst["trace"].n_fan)
            out = inst.get("out")
            if out is None:
                out = torch.empty((len(inst["freqs"]), recv.shape[0]), dtype=torch.complex64,
                                  device=recv.device)
            d = dict(inst, out=out)
            self.instances.append(d)
            _check_sigma(inst.get("flow_resistivity"), inst["trace"].scene.n_materials)
            args.append(sum_args(recv, inst["freqs"], inst["beam_b"], inst["gamma"], out,
                                 inst.get("ray_weight"), inst.get("order"), window, cutoff,
                                 tile_cull=tile_cull, absorption=inst.get("absorption"),
                                 flow_resistivity=inst.get("flow_resistivity")))
        n = len(args)
        self._args = (gbt_sum_args * n)(*args)
        self._traces = (C.c_void_p * n)(*[d["trace"].handle for d in self.instances])
        desc = gbt_batch_desc(n, C.cast(self._traces, C.c_void_p).value,
                              C.cast(self._args, C.c_void_p).value, 1 if use_graph else 0,
                              1 if autotune else 0, int(form))
        self.handle = gbt_batch_create(desc, _stream_ptr())

    @property
    def outputs(self):
        return [d["out"] for d in self.instances]

    def submit(self):
        gbt_batch_submit(self.handle, _stream_ptr())

    def close(self):
        if getattr(self, "handle", None):
            gbt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def synthesize(p, freqs, amp, t0: float, dt: float, n_t: int, out=None, accumulate: bool = False):
    """Time signals h[n, r] = Re sum_f amp_f p[f, r] exp(-i 2 pi freq_f (t0 + n dt)) from
    per-frequency fields p (complex64 [F, Nr] on the device, as gbs_sum returns them);
    float32 [n_t, Nr] (gbt_synthesize)."""
    import torch
    nf = len(freqs)
    _require(p.is_cuda and p.dtype == torch.complex64 and p.is_contiguous()
             and p.dim() == 2 and p.shape[0] == nf,
             f"p must be a contiguous complex64 CUDA tensor of shape ({nf}, n_recv)")
    _require(len(amp) == nf, "one amplitude per frequency")
    nr = int(p.shape[1])
    if out is None:
        out = torch.empty((int(n_t), nr), dtype=torch.float32, device=p.device)
    _require(out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
             and tuple(out.shape) == (int(n_t), nr), f"out must be float32 of shape ({n_t}, {nr})")
    fr = (C.c_double * nf)(*[float(f) for f in freqs])
    am = (C.c_double * (2 * nf))(*[v for a in amp for v in (complex(a).real, complex(a).imag)])
    _check(load().gbt_synthesize(_ptr(p), nf, nr, fr, am, float(t0), float(dt), int(n_t),
                                 _ptr(out), 1 if accumulate else 0, _stream_ptr()), "gbt_synthesize")
    return out


def gbs_sum_backward(trace: Trace, recv, freqs, beam_b, gamma, grad_out, ray_weight=None,
                     order=None, window: int = WINDOW_LINE, cutoff: float = 16.0,
                     need_weight: bool = True, need_b: bool = True, tile_cull: bool = False,
                     absorption=None, flow_resistivity=None):
    """(d gamma, d ray_weight, d b) of a real loss with dL/dp = grad_out (complex64 [F, Nr])."""
    import torch
    _check_tensors(recv, gamma, ray_weight, order, trace.scene.n_materials, trace.n_fan)
    _check_sigma(flow_resistivity, trace.scene.n_materials)
    go = grad_out.contiguous()
    _require(go.dtype == torch.complex64 and go.is_cuda
             and tuple(go.shape) == (len(freqs), int(recv.shape[0])),
             f"grad_out must be a complex64 CUDA tensor of shape ({len(freqs)}, {int(recv.shape[0])})")
    dg = torch.empty_like(gamma)
    dw = torch.empty(trace.n_fan, dtype=torch.float32, device=recv.device) if need_weight else None
    db = torch.empty(len(freqs), dtype=torch.float64, device=recv.device) if need_b else None
    a = sum_args(recv, freqs, beam_b, gamma, None, ray_weight, order, window, cutoff,
                 tile_cull=tile_cull, absorption=absorption, flow_resistivity=flow_resistivity)
    a.out = 0
    gbt_sum_backward(trace.handle, a, _ptr(go), _ptr(dg), _ptr(dw), _ptr(db), _stream_ptr())
    return dg, dw, db
