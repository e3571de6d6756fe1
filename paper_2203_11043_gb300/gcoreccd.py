"""ctypes binding of libgcoreccd (include/gcoreccd.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; the whole transport step runs in the library's CUDA
kernels.  If the shared library has not been built this module raises
(there is no CPU fallback).  Host arrays are numpy; device buffers are any
object with ``data_ptr()`` (a torch CUDA tensor) or a raw integer address.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GC_ABI_VERSION = 2
GC_OK, GC_INCOMPLETE = 0, 1
GC_ERR_PARAM, GC_ERR_ALLOC, GC_ERR_CUDA, GC_ERR_STATE = -1, -2, -3, -4
GC_ERR_DEVICE_TIMEOUT, GC_ERR_NO_DEVICE, GC_ERR_DEVICE_CHECK = -5, -6, -7
GC_FP64, GC_FP32, GC_FP32_KAHAN, GC_FP16X2 = 0, 1, 2, 3

# Every symbol include/gcoreccd.h declares.
EXPORTS = ("gc_default_params", "gc_create", "gc_load_carriers", "gc_run", "gc_collect",
           "gc_image", "gc_positions", "gc_get_stats", "gc_coulomb_field",
           "gc_coulomb_field_noalloc", "gc_save_state", "gc_restore_state", "gc_destroy",
           "gc_status_string", "gc_last_cuda_error", "gc_device_info", "gc_selftest_barrier_timeout",
           "gc_debug_inject")


class GcParams(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("thickness_um", ctypes.c_double),
        ("z_well_um", ctypes.c_double),
        ("a1_V_cm_um", ctypes.c_double),
        ("a2_V_cm", ctypes.c_double),
        ("T_K", ctypes.c_double),
        ("eps_si_rel", ctypes.c_double),
        ("softening_um", ctypes.c_double),
        ("dt_s", ctypes.c_double),
        ("max_steps", ctypes.c_int64),
        ("coulomb", ctypes.c_int32),
        ("diffusion", ctypes.c_int32),
        ("reflect_back", ctypes.c_int32),
        ("img_w", ctypes.c_int32),
        ("img_h", ctypes.c_int32),
        ("pixel_um", ctypes.c_double),
        ("graph_steps", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("newton", ctypes.c_int32),
        ("jchunk", ctypes.c_int32),
        ("pair_R", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("stored_charge", ctypes.c_int32),
        ("tile_frames", ctypes.c_int32),
        ("stored_z_um", ctypes.c_double),
        ("fuse_small", ctypes.c_int32),
        ("resident_ctas", ctypes.c_int32),
    ]


class GcStats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("n_active", ctypes.c_int64),
        ("n_collected", ctypes.c_int64),
        ("pair_interactions", ctypes.c_double),
        ("carrier_steps", ctypes.c_double),
        ("pair_variant", ctypes.c_int32),
        ("pair_blocks", ctypes.c_int32),
        ("jchunk", ctypes.c_int32),
        ("launches_per_step", ctypes.c_int32),
        ("pair_kernel_ms", ctypes.c_double),
        ("pair_kernel_launches", ctypes.c_int64),
        ("integrate_kernel_ms", ctypes.c_double),
        ("compact_kernel_ms", ctypes.c_double),
        ("timed_steps", ctypes.c_int64),
        ("device_loop", ctypes.c_int32),
        ("fused_path", ctypes.c_int32),
        ("tune_ms", ctypes.c_double),
        ("tune_candidates", ctypes.c_int32),
        ("tune_cached", ctypes.c_int32),
        ("pair_kernel_variant", ctypes.c_int32),
        ("small_n", ctypes.c_int32),
    ]


class GcState(ctypes.Structure):
    _fields_ = [
        ("xyz", ctypes.c_void_p),
        ("collect_step", ctypes.c_void_p),
        ("image", ctypes.c_void_p),
        ("off_image", ctypes.c_void_p),
        ("step", ctypes.c_int64),
        ("pair_interactions", ctypes.c_double),
        ("carrier_steps", ctypes.c_double),
    ]


class GcError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {gc_status_string(status)}"
        if status in (GC_ERR_CUDA, GC_ERR_NO_DEVICE, GC_ERR_ALLOC):
            msg += f" [{gc_last_cuda_error()}]"
        super().__init__(msg)
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The release library, or with GCORECCD_DEBUG=1 in the environment the
    GC_DEBUG build (bounds-checked kernels, fault planting)."""
    return _build.LIB_DEBUG if os.environ.get("GCORECCD_DEBUG") == "1" else _build.LIB


def load():
    """Load libgcoreccd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libgcoreccd.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.gc_default_params.restype = None
        L.gc_default_params.argtypes = [ctypes.POINTER(GcParams)]
        L.gc_create.restype = I32
        L.gc_create.argtypes = [ctypes.POINTER(GcParams), P, ctypes.POINTER(P)]
        L.gc_load_carriers.restype = I32
        L.gc_load_carriers.argtypes = [P, P, I64, P, I64, P, P]
        L.gc_run.restype = I32
        L.gc_run.argtypes = [P, I64, ctypes.POINTER(I64)]
        L.gc_collect.restype = I32
        L.gc_collect.argtypes = [P, P, P, P, P, P]
        L.gc_image.restype = I32
        L.gc_image.argtypes = [P, P, ctypes.c_int]
        L.gc_positions.restype = I32
        L.gc_positions.argtypes = [P, P]
        L.gc_get_stats.restype = I32
        L.gc_get_stats.argtypes = [P, ctypes.POINTER(GcStats)]
        L.gc_coulomb_field.restype = I32
        L.gc_coulomb_field.argtypes = [P, I64, ctypes.c_double, ctypes.c_double, I32, P, P]
        L.gc_coulomb_field_noalloc.restype = I32
        L.gc_coulomb_field_noalloc.argtypes = [P, I64, ctypes.c_double, ctypes.c_double, I32, P, P]
        L.gc_save_state.restype = I32
        L.gc_save_state.argtypes = [P, ctypes.POINTER(GcState)]
        L.gc_restore_state.restype = I32
        L.gc_restore_state.argtypes = [P, ctypes.POINTER(GcState)]
        L.gc_destroy.restype = None
        L.gc_destroy.argtypes = [P]
        L.gc_status_string.restype = ctypes.c_char_p
        L.gc_status_string.argtypes = [I32]
        L.gc_last_cuda_error.restype = ctypes.c_char_p
        L.gc_last_cuda_error.argtypes = []
        L.gc_device_info.restype = I32
        L.gc_device_info.argtypes = [ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]
        L.gc_selftest_barrier_timeout.restype = I32
        L.gc_selftest_barrier_timeout.argtypes = [ctypes.c_double]
        L.gc_debug_inject.restype = I32
        L.gc_debug_inject.argtypes = [P, I32]
        _lib = L
        return L


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(int(t.data_ptr()))


def _check(status: int, where: str) -> int:
    if status < 0:
        raise GcError(status, where)
    return status


def gc_status_string(status: int) -> str:
    return load().gc_status_string(int(status)).decode()


def gc_last_cuda_error() -> str:
    return load().gc_last_cuda_error().decode()


def gc_default_params(**overrides) -> GcParams:
    p = GcParams()
    load().gc_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(f"gc_params has no field {k}")
        setattr(p, k, v)
    return p


def gc_debug_inject(sim, what: int) -> None:
    _check(load().gc_debug_inject(sim, int(what)), "gc_debug_inject")


def gc_selftest_barrier_timeout(limit_s: float) -> int:
    """Status of the bounded-wait self-test (GC_ERR_DEVICE_TIMEOUT expected);
    returned, not raised."""
    return int(load().gc_selftest_barrier_timeout(float(limit_s)))


def gc_device_info():
    sm, ma, mi = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().gc_device_info(ctypes.byref(sm), ctypes.byref(ma), ctypes.byref(mi)), "gc_device_info")
    return sm.value, ma.value, mi.value


def gc_create(params: GcParams, stream=None) -> ctypes.c_void_p:
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    h = ctypes.c_void_p()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().gc_create(ctypes.byref(params), s, ctypes.byref(h)), "gc_create")
    return h


def gc_load_carriers(sim, xyz, event_offsets=None, seeds=None, img_origin=None) -> None:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    n = xyz.shape[0]
    offs = None if event_offsets is None else np.ascontiguousarray(event_offsets, dtype=np.int64)
    n_ev = 1 if offs is None else len(offs) - 1
    sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
    org = None if img_origin is None else np.ascontiguousarray(img_origin, dtype=np.float64)
    if sd is not None and len(sd) != n_ev:
        raise ValueError("seeds must have one entry per event")
    if org is not None and org.size != 2 * n_ev:
        raise ValueError("img_origin must be [n_events, 2]")
    _check(load().gc_load_carriers(sim, _np_ptr(xyz), n, _np_ptr(offs), n_ev, _np_ptr(sd),
                                   _np_ptr(org)), "gc_load_carriers")


def gc_run(sim, steps: int = -1):
    """Returns (status, steps_done); status is GC_OK or GC_INCOMPLETE."""
    done = ctypes.c_int64()
    st = _check(load().gc_run(sim, int(steps), ctypes.byref(done)), "gc_run")
    return st, done.value


def gc_collect(sim, n: int, n_events: int) -> dict:
    final_xy = np.zeros((n, 2))
    cs = np.zeros(n, dtype=np.int32)
    col = np.zeros(n_events, dtype=np.int64)
    off = np.zeros(n_events, dtype=np.int64)
    act = np.zeros(n_events, dtype=np.int64)
    _check(load().gc_collect(sim, _np_ptr(final_xy), _np_ptr(cs), _np_ptr(col), _np_ptr(off),
                             _np_ptr(act)), "gc_collect")
    return dict(final_xy=final_xy, collect_step=cs, n_collected=col, n_offimage=off, n_active=act)


def gc_image(sim, n_events: int, img_h: int, img_w: int, out=None):
    """Host copy (numpy) by default; `out` may be a device tensor of uint32/int32."""
    if out is not None:
        _check(load().gc_image(sim, _dev_ptr(out), 1), "gc_image")
        return out
    img = np.zeros((n_events, img_h, img_w), dtype=np.uint32)
    _check(load().gc_image(sim, _np_ptr(img), 0), "gc_image")
    return img


def gc_positions(sim, n: int) -> np.ndarray:
    xyz = np.zeros((n, 3))
    _check(load().gc_positions(sim, _np_ptr(xyz)), "gc_positions")
    return xyz


def gc_get_stats(sim) -> dict:
    st = GcStats()
    _check(load().gc_get_stats(sim, ctypes.byref(st)), "gc_get_stats")
    return {k: getattr(st, k) for k, _ in GcStats._fields_}


def gc_coulomb_field(xyz_dev, n: int, softening_um: float, eps_si_rel: float, precision: int,
                     E_dev, stream=None) -> None:
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().gc_coulomb_field(_dev_ptr(xyz_dev), int(n), float(softening_um), float(eps_si_rel),
                                   int(precision), _dev_ptr(E_dev), s), "gc_coulomb_field")


GC_NOALLOC_MAX_CARRIERS = 32768


def gc_coulomb_field_noalloc(xyz_dev, n: int, softening_um: float, eps_si_rel: float, precision: int,
                             E_dev, stream=None) -> None:
    """gc_coulomb_field without any device allocation (n <= GC_NOALLOC_MAX_CARRIERS);
    for callers that may not allocate.  Calls must not overlap on the GPU."""
    s = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().gc_coulomb_field_noalloc(_dev_ptr(xyz_dev), int(n), float(softening_um),
                                           float(eps_si_rel), int(precision), _dev_ptr(E_dev), s),
           "gc_coulomb_field_noalloc")


def gc_save_state(sim, n: int, n_events: int, img_h: int, img_w: int) -> dict:
    """Checkpoint as numpy arrays plus the step and the counters."""
    arrs = dict(xyz=np.zeros((n, 3)), collect_step=np.zeros(n, dtype=np.int32),
                image=np.zeros((n_events, img_h, img_w), dtype=np.uint32),
                off_image=np.zeros(n_events, dtype=np.int64))
    st = GcState(*(arrs[k].ctypes.data for k in ("xyz", "collect_step", "image", "off_image")), 0, 0.0, 0.0)
    _check(load().gc_save_state(sim, ctypes.byref(st)), "gc_save_state")
    arrs.update(step=st.step, pair_interactions=st.pair_interactions, carrier_steps=st.carrier_steps)
    return arrs


def gc_restore_state(sim, state: dict) -> None:
    a = {k: np.ascontiguousarray(state[k], dtype=t) for k, t in
         (("xyz", np.float64), ("collect_step", np.int32), ("image", np.uint32), ("off_image", np.int64))}
    st = GcState(*(a[k].ctypes.data for k in ("xyz", "collect_step", "image", "off_image")),
                 int(state["step"]), float(state["pair_interactions"]), float(state["carrier_steps"]))
    _check(load().gc_restore_state(sim, ctypes.byref(st)), "gc_restore_state")


def gc_destroy(sim) -> None:
    if sim:
        load().gc_destroy(sim)


class Simulation:
    """Owning wrapper around a gc_sim handle (same calls, fewer arguments)."""

    def __init__(self, params: GcParams, xyz, event_offsets=None, seeds=None, img_origin=None,
                 stream=None):
        self.params = params
        self.handle = gc_create(params, stream)
        try:
            xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
            self.n = xyz.shape[0]
            self.n_events = 1 if event_offsets is None else len(event_offsets) - 1
            gc_load_carriers(self.handle, xyz, event_offsets, seeds, img_origin)
        except Exception:
            gc_destroy(self.handle)
            self.handle = None
            raise

    def run(self, steps: int = -1):
        return gc_run(self.handle, steps)

    def collect(self) -> dict:
        return gc_collect(self.handle, self.n, self.n_events)

    def image(self, out=None):
        return gc_image(self.handle, self.n_events, self.params.img_h, self.params.img_w, out)

    def positions(self) -> np.ndarray:
        return gc_positions(self.handle, self.n)

    def stats(self) -> dict:
        return gc_get_stats(self.handle)

    def save_state(self) -> dict:
        return gc_save_state(self.handle, self.n, self.n_events, self.params.img_h, self.params.img_w)

    def restore_state(self, state: dict) -> None:
        gc_restore_state(self.handle, state)

    def close(self):
        if self.handle:
            gc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
