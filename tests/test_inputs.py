"""The seeded synthetic inputs follow the stated recipe (the stand-ins for the
paper's X-ray clouds, Sec. 5.1, and GEANT4 muon track, Sec. 5.2): sizes,
seeds, geometry and spreads, reproducibility from the seed, and the property
the sharding relies on -- an event of the batch is drawn from its own seed
only, so any sub-batch holds the same events bit for bit."""
import math

import numpy as np
import pytest

from paper_2203_11043_gb300 import inputs as I


def test_single_cloud_and_5p9kev_cloud():
    wl = I.single_cloud()
    assert wl.n == 256 and wl.n_events == 1 and list(wl.ev_off) == [0, 256] and wl.img_w == 32
    # centred on (0, 0, 300) with sigma 0.5 (sampling tolerance: 5 standard errors)
    assert np.all(np.abs(wl.xyz.mean(0) - [0.0, 0.0, 300.0]) < 5 * 0.5 / math.sqrt(256))
    assert np.all(np.abs(wl.xyz.std(0) / 0.5 - 1.0) < 5 / math.sqrt(2 * 256))
    # the image is centred on the cloud: 32 pixels of 15 um
    assert np.allclose(wl.img_origin[0], [-240.0, -240.0])
    assert np.array_equal(I.single_cloud().xyz, wl.xyz)
    assert not np.array_equal(I.single_cloud(seed=2).xyz, wl.xyz)
    x = I.xray_5p9kev()
    assert x.n == round(5900 / 3.75) == 1573 and x.img_w == 64
    z0 = x.xyz[:, 2].mean()
    assert 0.0 <= z0 <= 675.0
    assert np.all(np.abs(x.xyz.std(0) / 0.3 - 1.0) < 5 / math.sqrt(2 * 1573))


def test_xray_batch_sizes_seeds_and_independent_events():
    full = I.xray_batch()
    sizes = np.diff(full.ev_off)
    assert full.n_events == 4096 and full.n == sizes.sum()
    assert np.array_equal(full.seeds, np.arange(1, 4097, dtype=np.uint64))
    # N = lround(E / 3.75 eV), E ~ U(1, 18) keV
    assert sizes.min() >= round(1000 / 3.75) and sizes.max() <= round(18000 / 3.75)
    assert sizes.min() < 400 and sizes.max() > 4600  # the range is covered
    depth = np.array([full.xyz[a:b, 2].mean() for a, b in zip(full.ev_off[:-1], full.ev_off[1:])])
    assert depth.min() > -2.0 and depth.max() < 677.0
    # each event depends on its own seed only: the first 16 events as a batch of their own,
    # and events 100..115 drawn from seeds 101..116
    sub = I.xray_batch(n_events=16)
    assert np.array_equal(sub.xyz, full.xyz[:full.ev_off[16]])
    mid = I.xray_batch(n_events=16, first_seed=101)
    assert np.array_equal(mid.xyz, full.xyz[full.ev_off[100]:full.ev_off[116]])
    assert np.array_equal(np.diff(mid.ev_off), sizes[100:116])


def test_muon_track_geometry():
    wl = I.muon_track(n=50_000)
    xyz = wl.xyz
    dz, length = 675.0, 2500.0
    dx = math.sqrt(length ** 2 - dz ** 2)  # 2407.2 um along x
    u = np.array([dx, 0.0, -dz]) / length
    start = np.array([-0.5 * dx, 0.0, 675.0])
    t = (xyz - start) @ u  # position along the track
    assert t.min() > -3.0 and t.max() < length + 3.0
    # uniform along the track: mean and spread of U(0, L)
    assert abs(t.mean() / length - 0.5) < 0.01 and abs(t.std() / (length / math.sqrt(12)) - 1) < 0.02
    # 0.5 um jitter in the two orthogonal directions, none along the track
    r = xyz - start - t[:, None] * u
    assert abs(r[:, 1].std() / 0.5 - 1.0) < 0.02
    w = np.cross(u, [0.0, 1.0, 0.0])
    assert abs((r @ w).std() / 0.5 - 1.0) < 0.02
    assert np.abs(r @ u).max() < 1e-9


@pytest.mark.parametrize("n_tracks,per_track", [(16, 65536), (4, 1000)])
def test_track_bundle_is_one_event_of_parallel_tracks(n_tracks, per_track):
    wl = I.track_bundle(n_tracks=n_tracks, per_track=per_track)
    assert wl.n == n_tracks * per_track and wl.n_events == 1 and wl.img_w == 512
    y = wl.xyz[:, 1].reshape(n_tracks, per_track)
    centres = np.median(y, axis=1)
    assert np.allclose(np.diff(centres), 30.0, atol=0.05)
    assert abs(centres.mean()) < 0.05
