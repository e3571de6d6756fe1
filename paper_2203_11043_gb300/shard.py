"""Sharding of batched events across ranks (one process per GPU).

Each X-ray interaction is simulated as an independent cloud (Sec. 5.1), and
an event's result does not depend on the other events loaded with it (its
diffusion stream is keyed by its own seed and the carrier's index within the
event).  A batch therefore splits across GPUs with no exchange during the
run: each rank loads only its events through the same C ABI, runs them to
completion, and the images, counts and per-carrier results are gathered once
at the end.

Events are dealt by longest-processing-time first on a cost proxy: the pair
work of a step, N_e^2, times the number of steps the event lives, which grows
with its depth (the drift time to the wells), so N_e^2 (z0 + 5 um).

This module moves host arrays only; it holds none of the transport
arithmetic.
"""
from __future__ import annotations

import heapq

import numpy as np

from .inputs import Workload


def event_costs(wl: Workload) -> np.ndarray:
    """Cost proxy per event: N_e^2 (mean initial depth + 5 um)."""
    sizes = np.diff(wl.ev_off).astype(np.float64)
    depth = np.zeros(wl.n_events)
    for e in range(wl.n_events):
        a, b = int(wl.ev_off[e]), int(wl.ev_off[e + 1])
        depth[e] = float(wl.xyz[a:b, 2].mean()) if b > a else 0.0
    return sizes * sizes * (np.maximum(depth, 0.0) + 5.0)


def lpt_partition(costs, world: int) -> list:
    """Events dealt to `world` ranks, largest cost first, each to the rank
    with the least cost so far (ties to the lower rank).  Returns, per rank,
    its event indices in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda e: (-costs[e], e))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for e in order:
        load, r = heapq.heappop(heap)
        parts[r].append(e)
        heapq.heappush(heap, (load + costs[e], r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def sub_workload(wl: Workload, events) -> Workload:
    """The events `events` of wl (in that order) as a workload of their own."""
    events = np.asarray(events, dtype=np.int64)
    parts = [wl.xyz[int(wl.ev_off[e]):int(wl.ev_off[e + 1])] for e in events]
    sizes = [len(p) for p in parts]
    ev_off = np.zeros(len(events) + 1, np.int64)
    ev_off[1:] = np.cumsum(sizes)
    xyz = np.concatenate(parts, axis=0) if parts else np.zeros((0, 3))
    return Workload(f"{wl.name}-shard", xyz, ev_off, wl.seeds[events].copy(), wl.img_origin[events].copy(),
                    wl.img_w, wl.img_h)


PER_EVENT = ("image", "n_offimage", "n_collected", "n_active")
PER_CARRIER = ("final_xy", "collect_step", "positions")


def assemble(wl: Workload, parts) -> dict:
    """Global results from per-rank results: `parts` is a list of
    (events, result) pairs, where result holds per-event arrays (first axis
    over that rank's events, in order) and optionally per-carrier arrays
    (first axis over that rank's carriers, event by event).  Returns the same
    keys in the global event and carrier order; every event must come from
    exactly one rank."""
    E = wl.n_events
    seen = np.zeros(E, dtype=np.int64)
    out = {}
    for events, res in parts:
        events = np.asarray(events, dtype=np.int64)
        seen[events] += 1
        sizes = wl.ev_off[events + 1] - wl.ev_off[events]
        local_off = np.zeros(len(events) + 1, np.int64)
        local_off[1:] = np.cumsum(sizes)
        for k, v in res.items():
            v = np.asarray(v)
            if k in PER_EVENT:
                if k not in out:
                    out[k] = np.zeros((E,) + v.shape[1:], dtype=v.dtype)
                out[k][events] = v
            elif k in PER_CARRIER:
                if k not in out:
                    out[k] = np.zeros((wl.n,) + v.shape[1:], dtype=v.dtype)
                for i, e in enumerate(events):
                    a, b = int(wl.ev_off[e]), int(wl.ev_off[e + 1])
                    out[k][a:b] = v[local_off[i]:local_off[i + 1]]
    if not np.all(seen == 1):
        raise ValueError("every event must be simulated by exactly one rank")
    return out


def gather(wl: Workload, events, result: dict, dst: int = 0):
    """Gather every rank's (events, result) to rank `dst` over the default
    torch.distributed process group and assemble them there (gloo or NCCL);
    returns the global results on `dst` and None elsewhere.  Called once,
    after the run: the run itself has no collective."""
    import torch.distributed as dist
    payload = (np.asarray(events, dtype=np.int64), {k: np.asarray(v) for k, v in result.items()})
    rank = dist.get_rank()
    got = [None] * dist.get_world_size() if rank == dst else None
    dist.gather_object(payload, got, dst=dst)
    return assemble(wl, got) if rank == dst else None
