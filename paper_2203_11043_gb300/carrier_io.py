"""Carrier positions from files (Sec. 3.2: positions may be loaded from an
external file, e.g. a simulated particle track).

Formats:
  * text / CSV: one carrier per line, ``x y z`` or ``x y z event`` (um;
    separators: whitespace or commas; ``#`` starts a comment).  Lines of one
    event must be contiguous; event labels are arbitrary integers.
  * ``.npy``: a float array of shape [n, 3] (one event) or [n, 4] (the last
    column is the event label, contiguous per event).

The reader only parses; it returns an ``inputs.Workload`` ready for
``gc_load_carriers`` (image origins centred on each event's x-y centroid,
seeds 1..E unless given).  ``save_carriers`` writes the text format.
"""
from __future__ import annotations

import os

import numpy as np

from .inputs import PIXEL_UM, Workload, centred_origin


def _parse_text(path: str) -> np.ndarray:
    rows = []
    with open(path) as f:
        for ln, line in enumerate(f, 1):
            line = line.split("#", 1)[0].replace(",", " ").strip()
            if not line:
                continue
            vals = line.split()
            if len(vals) not in (3, 4):
                raise ValueError(f"{path}:{ln}: expected 3 or 4 columns, got {len(vals)}")
            rows.append([float(v) for v in vals])
    if not rows:
        return np.zeros((0, 3))
    widths = {len(r) for r in rows}
    if len(widths) != 1:
        raise ValueError(f"{path}: mixed 3- and 4-column lines")
    return np.asarray(rows, dtype=np.float64)


def load_carriers(path: str, img: int = 64, pixel_um: float = PIXEL_UM, seeds=None,
                  name: str | None = None) -> Workload:
    """Read carriers from `path` into a Workload."""
    if path.endswith(".npy"):
        arr = np.asarray(np.load(path), dtype=np.float64)
        if arr.ndim != 2 or arr.shape[1] not in (3, 4):
            raise ValueError(f"{path}: expected an [n, 3] or [n, 4] array, got {arr.shape}")
    else:
        arr = _parse_text(path)
    if not np.all(np.isfinite(arr)):
        raise ValueError(f"{path}: non-finite values")
    xyz = np.ascontiguousarray(arr[:, :3])
    n = xyz.shape[0]
    if arr.shape[1] == 4 and n:
        labels = arr[:, 3]
        starts = np.concatenate([[0], np.nonzero(np.diff(labels))[0] + 1])
        if len(np.unique(labels)) != len(starts):
            raise ValueError(f"{path}: the lines of an event must be contiguous")
        ev_off = np.concatenate([starts, [n]]).astype(np.int64)
    else:
        ev_off = np.array([0, n], dtype=np.int64)
    E = len(ev_off) - 1
    if seeds is None:
        seeds = np.arange(1, E + 1, dtype=np.uint64)
    seeds = np.asarray(seeds, dtype=np.uint64)
    if len(seeds) != E:
        raise ValueError("one seed per event is needed")
    origin = np.zeros((E, 2))
    for e in range(E):
        a, b = ev_off[e], ev_off[e + 1]
        cx, cy = (xyz[a:b, 0].mean(), xyz[a:b, 1].mean()) if b > a else (0.0, 0.0)
        origin[e] = centred_origin(cx, cy, img, img, pixel_um)
    return Workload(name or os.path.basename(path), xyz, ev_off, seeds, origin, img, img)


def save_carriers(path: str, xyz, ev_off=None) -> None:
    """Write carriers as text, with an event column when there is more than one event."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    with open(path, "w") as f:
        f.write("# x_um y_um z_um" + (" event" if ev_off is not None and len(ev_off) > 2 else "") + "\n")
        if ev_off is None or len(ev_off) <= 2:
            for x, y, z in xyz:
                f.write(f"{x:.17g} {y:.17g} {z:.17g}\n")
        else:
            for e in range(len(ev_off) - 1):
                for x, y, z in xyz[ev_off[e]:ev_off[e + 1]]:
                    f.write(f"{x:.17g} {y:.17g} {z:.17g} {e}\n")
