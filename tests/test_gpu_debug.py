"""The GC_DEBUG build (bounds-checked kernels) and the device-side checks.

  * On valid inputs the checks stay silent: every path (four-launch step,
    two-launch fused step, the persistent, cluster-resident and
    grid-resident single-event kernels, FP64 form) runs with the error word 0 and gives the release build's bits (the checks
    only guard accesses; the arithmetic is the same).
  * A planted fault -- event offsets that do not match the carriers, written
    on the host before upload (gc_debug_inject) -- is caught on the device
    before any kernel uses the offsets: gc_run returns GC_ERR_DEVICE_CHECK,
    nothing faults, and the device stays usable.
  * A planted missing peer -- one CTA of the grid-resident kernel withholds
    its first step's words -- makes every other CTA's bounded wait run out:
    gc_run returns GC_ERR_DEVICE_TIMEOUT within seconds, nothing faults or
    hangs, and the device stays usable.

The debug library runs in a child process (GCORECCD_DEBUG=1), since this
process has the release library loaded.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2203_11043_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, os.environ["ROOT"])
from paper_2203_11043_gb300 import build, inputs as I
build.build(debug=True)
import paper_2203_11043_gb300 as gc
assert gc.library_path().endswith("libgcoreccd_debug.so")
gc.load()
from tests.test_gpu_debug import cases
out = {}
for name, wl, kw in cases():
    p = gc.gc_default_params(img_w=wl.img_w, img_h=wl.img_h, autotune=0, pair_R=4, **kw)
    with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as sim:
        st, steps = sim.run(-1)
        out[name] = dict(status=st, steps=steps, path=sim.stats()["fused_path"])
        np.save(os.path.join(os.environ["OUT"], name + ".npy"), sim.positions())
# planted fault: offsets that do not match the carriers
wl = I.single_cloud(n=500, z0_um=30.0, img=16)
h = gc.gc_create(gc.gc_default_params(img_w=16, img_h=16))
try:
    gc.gc_debug_inject(h, 1)
    gc.gc_load_carriers(h, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin)
    try:
        gc.gc_run(h, -1)
        out["inject"] = "no error"
    except gc.GcError as e:
        out["inject"] = int(e.status)
finally:
    gc.gc_destroy(h)
# planted: one CTA of the grid-resident kernel withholds its first words
import time
wx = I.xray_5p9kev()
h = gc.gc_create(gc.gc_default_params(img_w=wx.img_w, img_h=wx.img_h, fuse_small=4))
try:
    gc.gc_load_carriers(h, wx.xyz, wx.ev_off, wx.seeds, wx.img_origin)
    gc.gc_debug_inject(h, 2)
    t0 = time.time()
    try:
        gc.gc_run(h, -1)
        out["withhold"] = "no error"
    except gc.GcError as e:
        out["withhold"] = int(e.status)
    out["withhold_s"] = time.time() - t0
finally:
    gc.gc_destroy(h)
# the device is usable afterwards
p = gc.gc_default_params(img_w=16, img_h=16)
with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as sim:
    out["after"] = int(sim.run(-1)[0])
print(json.dumps(out))
"""


def cases():
    """(name, workload, parameters) run in both builds: the cluster kernel,
    the persistent kernel and the grid-resident kernel (one small event), the
    two-launch fused step (a batch), the four-launch step throughout and with
    the hand-over (a larger event), and the FP64 form."""
    big = I.single_cloud(n=12000, sigma_um=0.6, z0_um=20.0, seed=44, img=32)
    batch = I.xray_batch(n_events=24)
    # the j-chunk is pinned: occupancy (and so the automatic j-chunk) differs between the builds
    return [("cluster_fp32", I.xray_5p9kev(), dict(precision=2, jchunk=512, fuse_small=5)),
            ("se_fp32", I.xray_5p9kev(), dict(precision=2, jchunk=512, fuse_small=3)),
            ("resident_fp32", I.xray_5p9kev(), dict(precision=2, fuse_small=4)),
            ("fused_batch", batch, dict(precision=2, jchunk=2048)),
            ("four_launch", big, dict(precision=2, fuse_small=0, jchunk=2048)),
            ("handover", big, dict(precision=2, jchunk=2048)),
            ("fp64_batch", batch, dict(precision=0, jchunk=512))]


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


def test_debug_build_checks_are_silent_then_catch_a_planted_fault(gc, tmp_path):
    env = dict(os.environ, GCORECCD_DEBUG="1", ROOT=ROOT, OUT=str(tmp_path))
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["inject"] == gc.GC_ERR_DEVICE_CHECK
    assert out["withhold"] == gc.GC_ERR_DEVICE_TIMEOUT and out["withhold_s"] < 30, out
    assert out["after"] == gc.GC_OK
    for name, wl, kw in cases():
        assert out[name]["status"] == gc.GC_OK, name
        p = gc.gc_default_params(img_w=wl.img_w, img_h=wl.img_h, autotune=0, pair_R=4, **kw)
        with gc.Simulation(p, wl.xyz, wl.ev_off, wl.seeds, wl.img_origin) as sim:
            st, steps = sim.run(-1)
            assert steps == out[name]["steps"] and sim.stats()["fused_path"] == out[name]["path"]
            assert np.array_equal(sim.positions(), np.load(tmp_path / (name + ".npy"))), name


def test_release_build_refuses_fault_planting(gc):
    h = gc.gc_create(gc.gc_default_params())
    try:
        with pytest.raises(gc.GcError) as err:
            gc.gc_debug_inject(h, 1)
        assert err.value.status == gc.GC_ERR_STATE
    finally:
        gc.gc_destroy(h)
