"""Seeded synthetic event generators (initial hole positions only).

These stand in for the paper's inputs: X-ray charge clouds (Sec. 5.1: a 3-D
Gaussian of N = E / w holes) and a muon track crossing the CCD (Sec. 5.2: the
paper's track comes from GEANT4, which is not available, so a straight line of
uniformly placed holes with Gaussian transverse jitter stands in for it).

This module holds none of the transport arithmetic; it only draws initial
positions with numpy's PCG64 generator and is shared by the tests, the smoke
check and the benchmark.  Positions are in um with z = 0 at the collection
surface and z = thickness at the back (Sec. 2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

THICKNESS_UM = 675.0
PIXEL_UM = 15.0
PAIR_ENERGY_EV = 3.75  # energy per electron-hole pair used by the workloads


@dataclasses.dataclass
class Workload:
    """Initial positions of one or more events plus their bookkeeping."""
    name: str
    xyz: np.ndarray          # [n, 3] float64, um
    ev_off: np.ndarray       # [E+1] int64
    seeds: np.ndarray        # [E] uint64 (diffusion-stream keys)
    img_origin: np.ndarray   # [E, 2] float64, lower-left image corner, um
    img_w: int
    img_h: int

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_events(self) -> int:
        return int(len(self.ev_off) - 1)


def centred_origin(cx: float, cy: float, w: int, h: int, pixel_um: float = PIXEL_UM):
    """Lower-left corner of a w x h image centred on (cx, cy)."""
    return (cx - 0.5 * w * pixel_um, cy - 0.5 * h * pixel_um)


def gaussian_cloud(n: int, sigma_um: float, centre, rng: np.random.Generator) -> np.ndarray:
    """Isotropic 3-D Gaussian cloud of n holes around `centre`."""
    return np.asarray(centre, dtype=np.float64)[None, :] + sigma_um * rng.standard_normal((n, 3))


def single_cloud(n: int = 256, sigma_um: float = 0.5, z0_um: float = 300.0, seed: int = 1,
                 img: int = 32, name: str = "cloud") -> Workload:
    """One X-ray-like cloud centred at (0, 0, z0)."""
    rng = np.random.default_rng(seed)
    xyz = gaussian_cloud(n, sigma_um, (0.0, 0.0, z0_um), rng)
    ox, oy = centred_origin(0.0, 0.0, img, img)
    return Workload(name, xyz, np.array([0, n], np.int64), np.array([seed], np.uint64),
                    np.array([[ox, oy]]), img, img)


def xray_5p9kev(seed: int = 1, img: int = 64) -> Workload:
    """5.9 keV X-ray: N = 1573 holes, sigma 0.3 um, depth uniform in [0, thickness)."""
    rng = np.random.default_rng(seed)
    z0 = rng.uniform(0.0, THICKNESS_UM)
    n = int(round(5900.0 / PAIR_ENERGY_EV))
    xyz = gaussian_cloud(n, 0.3, (0.0, 0.0, z0), rng)
    ox, oy = centred_origin(0.0, 0.0, img, img)
    return Workload("xray-5.9keV", xyz, np.array([0, n], np.int64), np.array([seed], np.uint64),
                    np.array([[ox, oy]]), img, img)


def xray_batch(n_events: int = 4096, e_min_kev: float = 1.0, e_max_kev: float = 18.0,
               sigma_um: float = 0.3, first_seed: int = 1, img: int = 64) -> Workload:
    """Independent X-ray events with energies uniform in [e_min, e_max] keV.

    Event k uses seed first_seed + k both for its own draws (energy, depth,
    cloud) and as its diffusion-stream key.
    """
    parts, sizes, seeds = [], [], []
    for k in range(n_events):
        seed = first_seed + k
        rng = np.random.default_rng(seed)
        energy_ev = 1000.0 * rng.uniform(e_min_kev, e_max_kev)
        z0 = rng.uniform(0.0, THICKNESS_UM)
        n = int(round(energy_ev / PAIR_ENERGY_EV))
        parts.append(gaussian_cloud(n, sigma_um, (0.0, 0.0, z0), rng))
        sizes.append(n)
        seeds.append(seed)
    ev_off = np.zeros(n_events + 1, np.int64)
    ev_off[1:] = np.cumsum(sizes)
    ox, oy = centred_origin(0.0, 0.0, img, img)
    origin = np.tile(np.array([[ox, oy]]), (n_events, 1))
    return Workload("xray-batch", np.concatenate(parts, axis=0), ev_off,
                    np.asarray(seeds, np.uint64), origin, img, img)


def _track(n: int, length_um: float, jitter_um: float, y_offset: float,
           rng: np.random.Generator) -> np.ndarray:
    """Straight track from the back surface (z = thickness) to the front
    (z = 0), centred on x = 0, with holes uniform along it and Gaussian jitter
    in the two directions orthogonal to it."""
    dz = THICKNESS_UM
    dx = math.sqrt(length_um ** 2 - dz ** 2)
    u = np.array([dx, 0.0, -dz]) / length_um          # along the track
    v = np.array([0.0, 1.0, 0.0])                     # orthogonal, in y
    w = np.cross(u, v)                                # orthogonal, in the x-z plane
    start = np.array([-0.5 * dx, y_offset, THICKNESS_UM])
    t = rng.uniform(0.0, length_um, size=n)
    jv = jitter_um * rng.standard_normal(n)
    jw = jitter_um * rng.standard_normal(n)
    return start[None, :] + t[:, None] * u[None, :] + jv[:, None] * v[None, :] + jw[:, None] * w[None, :]


def muon_track(n: int = 200_000, length_um: float = 2500.0, jitter_um: float = 0.5,
               seed: int = 1, img: int = 512) -> Workload:
    """One muon-like straight track of n holes across the full thickness."""
    rng = np.random.default_rng(seed)
    xyz = _track(n, length_um, jitter_um, 0.0, rng)
    ox, oy = centred_origin(0.0, 0.0, img, img)
    return Workload("muon", xyz, np.array([0, n], np.int64), np.array([seed], np.uint64),
                    np.array([[ox, oy]]), img, img)


def track_bundle(n_tracks: int = 16, per_track: int = 65536, spacing_um: float = 30.0,
                 length_um: float = 2500.0, jitter_um: float = 0.5, seed: int = 1,
                 img: int = 512) -> Workload:
    """n_tracks parallel muon-like tracks, spacing_um apart in y, as ONE event."""
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(n_tracks):
        y_off = (k - 0.5 * (n_tracks - 1)) * spacing_um
        parts.append(_track(per_track, length_um, jitter_um, y_off, rng))
    xyz = np.concatenate(parts, axis=0)
    n = xyz.shape[0]
    ox, oy = centred_origin(0.0, 0.0, img, img)
    return Workload("track-bundle", xyz, np.array([0, n], np.int64), np.array([seed], np.uint64),
                    np.array([[ox, oy]]), img, img)


def subsample(wl: Workload, n: int, seed: int = 7) -> Workload:
    """The first event of `wl` reduced to n randomly chosen holes (ids renumbered)."""
    rng = np.random.default_rng(seed)
    a, b = int(wl.ev_off[0]), int(wl.ev_off[1])
    pick = np.sort(rng.choice(np.arange(a, b), size=min(n, b - a), replace=False))
    xyz = wl.xyz[pick]
    return Workload(wl.name + f"-sub{len(pick)}", xyz, np.array([0, len(pick)], np.int64),
                    wl.seeds[:1].copy(), wl.img_origin[:1].copy(), wl.img_w, wl.img_h)
