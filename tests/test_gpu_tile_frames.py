"""Tile frames (gc_params.tile_frames = 1) on the GPU against the FP64 oracle.

With tile frames, events of >= 2048 holes are put in Morton order at load
and their FP32 shadow is taken relative to the FP64 origin of each 256-slot
tile; a pair item moves its i's and every staged j-tile into the frame of its
first i-tile with the same FP32 expression on both sides, so a hole's own
term stays exactly 0.  Checks:

  * one step, sampled holes against the oracle's step: within 1e-5 um for
    compact and extended events (event frame: within 1e-4 um), both errors
    printed;
  * resumed run == uninterrupted run, graph == eager (bit-identical);
  * a batch with one large event: events below 2048 holes are bit-identical
    to the same batch without tile frames (they keep the event frame), counts
    exact;
  * (test_gpu_workloads) FP32 + Kahan and FP16x2 with tile frames on a
    10,000-hole track: sigma_x, sigma_y within 0.5 % and image L1 <= 1 % of
    the FP64 form's.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_11043_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SMALL_EVENT = 2048  # events below this size run the 4-lane path in the event frame


@pytest.fixture(scope="module")
def gc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_11043_gb300 import build
    build.build()
    import paper_2203_11043_gb300 as g
    g.load()
    return g


def one_step_error(gc, wl, tile_frames, n_targets=48, img=512):
    p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=img, img_h=img, tile_frames=tile_frames)
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as sim:
        x0 = sim.positions()
        cs0 = sim.collect()["collect_step"]
        assert sim.run(1) == (gc.GC_OK, 1)
        x1 = sim.positions()
        st = sim.stats()
    active = np.nonzero(cs0 < 0)[0]
    rng = np.random.default_rng(2)
    tg = np.sort(rng.choice(active, size=min(n_targets, len(active)), replace=False))
    want = O.step_targets(O.make_params(img_w=img, img_h=img), x0, active, tg, int(wl.seeds[0]), 1)
    return np.abs(x1[tg] - want).max(), st


WORKLOADS = {
    "cloud10k": lambda: I.single_cloud(n=10_000, sigma_um=0.5, z0_um=300.0, seed=5, img=64),
    "bundle65k": lambda: I.subsample(I.track_bundle(), 65_536, seed=3),
    "muon20k": lambda: I.muon_track(n=20_000, seed=2),
    "bundle1M": lambda: I.track_bundle(),
}


@pytest.mark.parametrize("which", list(WORKLOADS))
def test_one_step_sampled_both_frames(gc, which):
    wl = WORKLOADS[which]()
    assert wl.n_events == 1 and wl.n >= SMALL_EVENT
    err_ev, st_ev = one_step_error(gc, wl, 0)
    err_tf, st_tf = one_step_error(gc, wl, 1)
    print(f"{which}: one step, FP32 + Kahan vs oracle: max |dr| event frame {err_ev:.2e} um, "
          f"tile frames {err_tf:.2e} um")
    # one more launch per step (the shadow kernel) with tile frames
    assert st_tf["launches_per_step"] == st_ev["launches_per_step"] + 1
    assert err_ev < 1e-4, err_ev
    assert err_tf < 1e-5, err_tf


def test_resume_equals_uninterrupted_with_tile_frames(gc):
    wl = I.single_cloud(n=9000, sigma_um=1.5, z0_um=30.0, seed=23, img=32)  # arrivals from ~step 80
    p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=32, img_h=32, graph_steps=8,
                             pair_R=4, tile_frames=1)
    k = 60
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as a:
        a.run(2 * k)
        want = (a.positions(), a.collect()["collect_step"], a.image(), a.stats())
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as b:
        b.run(k)
        state = b.save_state()
    assert np.sum(state["collect_step"] < 0) >= SMALL_EVENT  # the checkpoint is taken in tile frames
    assert np.any(want[1] > k)                         # and holes are collected after it
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as c:
        c.restore_state(state)
        c.run(k)
        got = (c.positions(), c.collect()["collect_step"], c.image(), c.stats())
    for g_, w_ in zip(got[:3], want[:3]):
        assert np.array_equal(g_, w_)
    assert got[3]["pair_interactions"] == want[3]["pair_interactions"]


def test_graph_equals_eager_with_tile_frames(gc):
    wl = I.single_cloud(n=8500, sigma_um=1.0, z0_um=15.0, seed=31, img=32)
    outs = []
    for gs in (0, 6):
        p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=32, img_h=32, graph_steps=gs,
                                 pair_R=4, tile_frames=1)
        with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as sim:
            st, done = sim.run(40)
            assert st == gc.GC_OK and done == 40
            outs.append((sim.positions(), sim.collect()["collect_step"], sim.image()))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_batch_with_one_large_event(gc):
    """Events below SMALL_EVENT keep the event frame and the 4-lane path:
    bit-identical with and without tile frames; counts exact everywhere."""
    big = I.single_cloud(n=9000, sigma_um=1.0, z0_um=6.0, seed=41, img=32)
    small = I.xray_batch(n_events=24)
    xyz = np.concatenate([small.xyz, big.xyz])
    ev_off = np.concatenate([small.ev_off, [small.n + big.n]]).astype(np.int64)
    seeds = np.concatenate([small.seeds, big.seeds]).astype(np.uint64)
    origin = np.concatenate([small.img_origin[:, :], big.img_origin[:, :]])
    img = small.img_w
    res = []
    for tf in (0, 1):
        p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=img, img_h=img, pair_R=4,
                                 jchunk=8192, tile_frames=tf, autotune=0)  # the same shape in both frames
        with gc.Simulation(p, xyz, ev_off, seeds, origin) as sim:
            st, steps = sim.run(-1)
            assert st == gc.GC_OK
            out = sim.collect()
            out.update(positions=sim.positions(), image=sim.image())
            res.append(out)
    sizes = np.diff(ev_off)
    for r in res:
        assert np.array_equal(r["n_collected"], sizes)
        assert np.array_equal(r["image"].reshape(len(sizes), -1).sum(1) + r["n_offimage"], sizes)
    a, b = small.n, xyz.shape[0]
    small_ev = [e for e in range(len(sizes) - 1) if sizes[e] < SMALL_EVENT]
    assert len(small_ev) >= 8
    for e in small_ev:
        s0, s1 = int(ev_off[e]), int(ev_off[e + 1])
        assert np.array_equal(res[0]["positions"][s0:s1], res[1]["positions"][s0:s1])
        assert np.array_equal(res[0]["collect_step"][s0:s1], res[1]["collect_step"][s0:s1])
        assert np.array_equal(res[0]["image"][e], res[1]["image"][e])
    # the large event: same statistics in both frames
    for c in (0, 1):
        assert res[1]["positions"][a:b, c].std() == pytest.approx(res[0]["positions"][a:b, c].std(),
                                                                  rel=5e-3)


def test_stored_charge_with_tile_frames_against_oracle(gc):
    """Stored-charge field (Sec. 1) and tile frames together on a 3000-hole
    cloud near the wells: counts exact, sigma_x, sigma_y within 0.5 % and
    image L1 <= 1 % of the FP64 oracle's."""
    wl = I.single_cloud(n=3000, sigma_um=1.0, z0_um=12.0, seed=51, img=32)
    kw = dict(stored_charge=1, stored_z_um=0.0)
    p = gc.gc_default_params(precision=gc.GC_FP32_KAHAN, img_w=32, img_h=32, tile_frames=1, **kw)
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as sim:
        st, _ = sim.run(-1)
        assert st == gc.GC_OK
        got = sim.collect()
        got.update(positions=sim.positions(), image=sim.image())
        assert sim.stats()["launches_per_step"] == 6  # pair, pixels, integrate, compact, finalize, shadow
    ref = O.Simulation(O.make_params(img_w=32, img_h=32, **kw), wl.xyz, wl.ev_off, wl.seeds, wl.img_origin)
    ref.run()
    assert got["n_collected"][0] == wl.n and np.all(ref.collect_step >= 0)
    for c in (0, 1):
        assert got["positions"][:, c].std() == pytest.approx(ref.positions()[:, c].std(), rel=5e-3)
    assert np.abs(got["image"].astype(np.int64) - ref.image.astype(np.int64)).sum() <= 0.01 * wl.n
