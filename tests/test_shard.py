"""Sharding of batched events across ranks (host logic on CPU, gloo world
size 2) and its equivalence with an unsharded run on one GPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2203_11043_gb300 import inputs as I  # noqa: E402
from paper_2203_11043_gb300 import shard  # noqa: E402


def fake_result(wl, events):
    """Per-event and per-carrier arrays that encode the global ids, as a
    rank's simulation results would be laid out."""
    sub = shard.sub_workload(wl, events)
    ids = np.concatenate([np.arange(wl.ev_off[e], wl.ev_off[e + 1]) for e in events]) if len(events) else \
        np.zeros(0, np.int64)
    img = np.stack([np.full((wl.img_h, wl.img_w), e, np.uint32) for e in events]) if len(events) else \
        np.zeros((0, wl.img_h, wl.img_w), np.uint32)
    return {"image": img, "n_offimage": np.asarray(events, np.int64) * 3,
            "collect_step": ids.astype(np.int32), "final_xy": np.stack([ids, -ids], 1).astype(np.float64),
            "positions": sub.xyz}


def test_lpt_partition_covers_every_event_once_and_balances():
    costs = np.random.default_rng(1).uniform(1, 100, size=1000)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, world)
        allev = np.sort(np.concatenate(parts))
        assert np.array_equal(allev, np.arange(1000))
        loads = np.array([costs[p].sum() for p in parts])
        # LPT is within 4/3 of the optimum, and the optimum is at least the mean and the largest job
        assert loads.max() <= 4 / 3 * max(loads.sum() / world, costs.max()) + 1e-9


def test_event_costs_follow_size_and_depth():
    wl = I.xray_batch(n_events=16)
    c = shard.event_costs(wl)
    sizes = np.diff(wl.ev_off)
    e = np.argsort(sizes)
    depth = np.array([wl.xyz[wl.ev_off[k]:wl.ev_off[k + 1], 2].mean() for k in range(16)])
    np.testing.assert_allclose(c, sizes.astype(float) ** 2 * (depth + 5.0))


def test_assemble_restores_global_order():
    wl = I.xray_batch(n_events=12, img=8)
    parts = shard.lpt_partition(shard.event_costs(wl), 3)
    out = shard.assemble(wl, [(p, fake_result(wl, p)) for p in parts])
    ids = np.arange(wl.n)
    assert np.array_equal(out["collect_step"], ids)
    assert np.array_equal(out["final_xy"][:, 1], -ids)
    assert np.array_equal(out["positions"], wl.xyz)
    assert np.array_equal(out["n_offimage"], np.arange(12) * 3)
    assert np.array_equal(out["image"][:, 0, 0], np.arange(12))
    with pytest.raises(ValueError):  # an event given to two ranks
        shard.assemble(wl, [(parts[0], fake_result(wl, parts[0])), (parts[0], fake_result(wl, parts[0]))])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2203_11043_gb300 import inputs as I2
    from paper_2203_11043_gb300 import shard as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = I2.xray_batch(n_events=10, img=8)
    parts = S.lpt_partition(S.event_costs(wl), world)
    mine = parts[rank]
    sub = S.sub_workload(wl, mine)
    assert np.array_equal(sub.seeds, wl.seeds[mine])
    res = fake_result(wl, mine)
    out = S.gather(wl, mine, res)
    if rank == 0:
        q.put((rank, out["collect_step"].tolist(), out["image"][:, 0, 0].tolist(), [len(p) for p in parts]))
    else:
        q.put((rank, out, None, None))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_over_gloo_world_size_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = I.xray_batch(n_events=10, img=8)
    r0, r1 = got
    assert r0[1] == list(range(wl.n)) and r0[2] == list(range(10)) and sum(r0[3]) == 10
    assert r1[1] is None


@pytest.mark.gpu
def test_sharded_run_equals_unsharded_on_one_gpu():
    """The batch run as one simulation and as two shards (run one after the
    other on the same GPU, as two ranks would) gives the same bits once the
    shards are assembled: an event's result does not depend on its batch
    (pair shape pinned)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11043_gb300 import build
    build.build()
    import paper_2203_11043_gb300 as gc
    gc.load()
    wl = I.xray_batch(n_events=48)

    def run(w):
        p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=w.img_w, img_h=w.img_h, autotune=0,
                                 pair_R=4, jchunk=2048)
        with gc.Simulation(p, w.xyz, w.ev_off, w.seeds, w.img_origin) as sim:
            st, _ = sim.run(-1)
            assert st == gc.GC_OK
            r = sim.collect()
            return {"image": sim.image(), "n_offimage": r["n_offimage"], "n_collected": r["n_collected"],
                    "collect_step": r["collect_step"], "final_xy": r["final_xy"], "positions": sim.positions()}

    whole = run(wl)
    parts = shard.lpt_partition(shard.event_costs(wl), 2)
    got = shard.assemble(wl, [(p, run(shard.sub_workload(wl, p))) for p in parts])
    for k in whole:
        assert np.array_equal(got[k], whole[k]), k
