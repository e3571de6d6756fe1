"""FP64 CPU oracle of the G-CoReCCD transport step (arXiv 2203.11043).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library ``paper_2203_11043_gb300``, and neither imports the other.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over field points);
this module only compiles it (gcc) and marshals numpy arrays into it.

Pins (tests/test_oracle_pins.py): Eq. 2 against hand-evaluated mobility values
and its closed-form limits; Eq. 6 against the gradient of the softened
potential, its pairwise antisymmetry and the 2- and 3-body closed forms;
Philox-4x32-10 against published known-answer vectors; Box-Muller against the
normal distribution; the whole Coulomb-off step against the analytic drift
time and lateral spread; the 2-body run against an independent ODE solution.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, OpenMP if available)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("thickness_um", ctypes.c_double),
        ("z_well_um", ctypes.c_double),
        ("a1", ctypes.c_double),
        ("a2", ctypes.c_double),
        ("T", ctypes.c_double),
        ("eps_si_rel", ctypes.c_double),
        ("softening_um", ctypes.c_double),
        ("dt_s", ctypes.c_double),
        ("max_steps", ctypes.c_int64),
        ("coulomb", ctypes.c_int32),
        ("diffusion", ctypes.c_int32),
        ("reflect_back", ctypes.c_int32),
        ("pixel_um", ctypes.c_double),
        ("img_w", ctypes.c_int32),
        ("img_h", ctypes.c_int32),
        ("stored_charge", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("stored_z_um", ctypes.c_double),
    ]


class OrcState(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("n_events", ctypes.c_int64),
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("ev_off", ctypes.c_void_p),
        ("seeds", ctypes.c_void_p),
        ("img_origin", ctypes.c_void_p),
        ("collect_step", ctypes.c_void_p),
        ("image", ctypes.c_void_p),
        ("off_image", ctypes.c_void_p),
        ("step", ctypes.c_int64),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # A test may point this at a deliberately broken copy of the
            # oracle to check that the pins catch the mistake.
            path = os.environ.get("GCORECCD_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.orc_mobility.restype = ctypes.c_double
            L.orc_mobility.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_coulomb_K.restype = ctypes.c_double
            L.orc_coulomb_K.argtypes = [ctypes.c_double]
            L.orc_thermal_voltage.restype = ctypes.c_double
            L.orc_thermal_voltage.argtypes = [ctypes.c_double]
            L.orc_philox4x32_10.restype = None
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_diffusion_normals.restype = None
            L.orc_diffusion_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint64, P]
            L.orc_coulomb_field.restype = None
            L.orc_coulomb_field.argtypes = [P, P, P, P, ctypes.c_int64, P, ctypes.c_int64,
                                            ctypes.c_double, ctypes.c_double, P]
            L.orc_init.restype = ctypes.c_int
            L.orc_init.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcState)]
            L.orc_run.restype = ctypes.c_int64
            L.orc_run.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcState),
                                  ctypes.c_int64]
            L.orc_step_targets.restype = None
            L.orc_step_targets.argtypes = [ctypes.POINTER(OrcParams), P, P, P, P,
                                           ctypes.c_int64, P, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.c_uint64, P]
            L.orc_stored_field.restype = None
            L.orc_stored_field.argtypes = [ctypes.POINTER(OrcParams), P, P, P, ctypes.c_int64, P]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_num_threads.argtypes = []
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- default parameters (the CCD of the X-ray and muon workloads) ----------
DEFAULTS = dict(thickness_um=675.0, z_well_um=0.0, a1=2.0, a2=1500.0, T=140.0,
                eps_si_rel=11.7, softening_um=0.01, dt_s=1e-11, max_steps=100000,
                coulomb=1, diffusion=1, reflect_back=1, pixel_um=15.0,
                img_w=32, img_h=32, stored_charge=0, pad=0, stored_z_um=0.0)


def make_params(**kw) -> OrcParams:
    d = dict(DEFAULTS)
    d.update(kw)
    return OrcParams(**d)


def mobility(E_abs: float, T: float) -> float:
    """Eq. 2."""
    return lib().orc_mobility(float(E_abs), float(T))


def coulomb_K(eps_rel: float = 11.7) -> float:
    """Eq. 6 constant in V/cm * um^2."""
    return lib().orc_coulomb_K(float(eps_rel))


def thermal_voltage(T: float) -> float:
    return lib().orc_thermal_voltage(float(T))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def diffusion_normals(seed: int, ids, step: int) -> np.ndarray:
    """[len(ids), 3] normals of the given carriers at one step."""
    ids = np.atleast_1d(np.asarray(ids, dtype=np.int64))
    out = np.zeros((len(ids), 3))
    buf = np.zeros(3)
    L = lib()
    for k, i in enumerate(ids):
        L.orc_diffusion_normals(int(seed), int(i), int(step), _ptr(buf))
        out[k] = buf
    return out


def coulomb_field(xyz: np.ndarray, softening_um: float = 0.01, eps_rel: float = 11.7,
                  src=None, targets=None) -> np.ndarray:
    """Eq. 6 field in V/cm at `targets` (default: all) from `src` (default: all)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    x = np.ascontiguousarray(xyz[:, 0])
    y = np.ascontiguousarray(xyz[:, 1])
    z = np.ascontiguousarray(xyz[:, 2])
    src = np.arange(n, dtype=np.int64) if src is None else np.ascontiguousarray(src, np.int64)
    tg = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    E = np.zeros((len(tg), 3))
    lib().orc_coulomb_field(_ptr(x), _ptr(y), _ptr(z), _ptr(src), len(src), _ptr(tg), len(tg),
                            float(softening_um), coulomb_K(eps_rel), _ptr(E))
    return E


class Simulation:
    """Oracle simulation of one or more independent events.

    xyz: [n, 3] initial positions (um); ev_off: [E+1] event offsets (default one
    event); seeds: [E]; img_origin: [E, 2] lower-left image corners (um).
    """

    def __init__(self, params: OrcParams, xyz, ev_off=None, seeds=None, img_origin=None):
        xyz = np.asarray(xyz, dtype=np.float64)
        self.p = params
        self.n = xyz.shape[0]
        self.x = np.ascontiguousarray(xyz[:, 0]).copy()
        self.y = np.ascontiguousarray(xyz[:, 1]).copy()
        self.z = np.ascontiguousarray(xyz[:, 2]).copy()
        self.ev_off = (np.array([0, self.n], dtype=np.int64) if ev_off is None
                       else np.ascontiguousarray(ev_off, dtype=np.int64))
        E = len(self.ev_off) - 1
        self.n_events = E
        self.seeds = (np.ones(E, dtype=np.uint64) if seeds is None
                      else np.ascontiguousarray(seeds, dtype=np.uint64))
        if img_origin is None:
            img_origin = np.zeros((E, 2))
        self.img_origin = np.ascontiguousarray(img_origin, dtype=np.float64).reshape(E, 2)
        self.collect_step = np.full(self.n, -1, dtype=np.int32)
        self.image = np.zeros((E, params.img_h, params.img_w), dtype=np.uint32)
        self.off_image = np.zeros(E, dtype=np.int64)
        self.st = OrcState(self.n, E, _ptr(self.x).value, _ptr(self.y).value,
                           _ptr(self.z).value, _ptr(self.ev_off).value,
                           _ptr(self.seeds).value, _ptr(self.img_origin).value,
                           _ptr(self.collect_step).value, _ptr(self.image).value,
                           _ptr(self.off_image).value, 0)
        rc = lib().orc_init(ctypes.byref(self.p), ctypes.byref(self.st))
        if rc != 0:
            raise ValueError("oracle: invalid parameters")

    @property
    def step(self) -> int:
        return int(self.st.step)

    def run(self, steps: int = 1 << 62) -> int:
        r = lib().orc_run(ctypes.byref(self.p), ctypes.byref(self.st), int(steps))
        if r < 0:
            raise ValueError("oracle: invalid arguments")
        return int(r)

    def positions(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)

    def n_active(self) -> np.ndarray:
        act = self.collect_step < 0
        return np.array([int(act[self.ev_off[e]:self.ev_off[e + 1]].sum())
                         for e in range(self.n_events)], dtype=np.int64)


def step_targets(params: OrcParams, xyz, src, targets, seed: int, step: int) -> np.ndarray:
    """New positions of carriers `targets` after step `step`, with the field from `src`."""
    xyz = np.asarray(xyz, dtype=np.float64)
    x = np.ascontiguousarray(xyz[:, 0])
    y = np.ascontiguousarray(xyz[:, 1])
    z = np.ascontiguousarray(xyz[:, 2])
    src = np.ascontiguousarray(src, dtype=np.int64)
    tg = np.ascontiguousarray(targets, dtype=np.int64)
    out = np.zeros((len(tg), 3))
    lib().orc_step_targets(ctypes.byref(params), _ptr(x), _ptr(y), _ptr(z), _ptr(src),
                           len(src), _ptr(tg), len(tg), int(seed), int(step), _ptr(out))
    return out


def stored_field(params: OrcParams, image, origin, xyz) -> np.ndarray:
    """Field in V/cm at points xyz [m, 3] from the charge stored in one event's image."""
    img = np.ascontiguousarray(image, dtype=np.uint32)
    org = np.ascontiguousarray(origin, dtype=np.float64).reshape(2)
    pts = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    E = np.zeros((len(pts), 3))
    lib().orc_stored_field(ctypes.byref(params), _ptr(img), _ptr(org), _ptr(pts), len(pts), _ptr(E))
    return E


def num_threads() -> int:
    return int(lib().orc_num_threads())
