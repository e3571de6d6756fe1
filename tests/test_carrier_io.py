"""Carrier files (Sec. 3.2: positions loaded from an external file)."""
import numpy as np
import pytest

from paper_2203_11043_gb300 import carrier_io, inputs


def test_text_round_trip_keeps_events_and_positions(tmp_path):
    wl = inputs.xray_batch(n_events=5)
    path = tmp_path / "batch.txt"
    carrier_io.save_carriers(str(path), wl.xyz, wl.ev_off)
    got = carrier_io.load_carriers(str(path), img=64)
    assert np.array_equal(got.xyz, wl.xyz)  # %.17g round-trips FP64 exactly
    assert np.array_equal(got.ev_off, wl.ev_off)
    assert got.n_events == 5 and list(got.seeds) == [1, 2, 3, 4, 5]


def test_csv_and_comments_one_event(tmp_path):
    path = tmp_path / "track.csv"
    path.write_text("# a GEANT4-style dump\n1.0, 2.0, 300.0\n\n1.5,2.5,301.0  # trailing\n")
    wl = carrier_io.load_carriers(str(path), img=32)
    np.testing.assert_array_equal(wl.xyz, [[1.0, 2.0, 300.0], [1.5, 2.5, 301.0]])
    assert wl.n_events == 1
    np.testing.assert_allclose(wl.img_origin[0], [1.25 - 16 * 15.0, 2.25 - 16 * 15.0])


def test_npy_with_event_column(tmp_path):
    a = np.array([[0, 0, 5, 7], [1, 1, 6, 7], [2, 2, 7, 3]], dtype=float)
    path = tmp_path / "c.npy"
    np.save(path, a)
    wl = carrier_io.load_carriers(str(path))
    assert list(wl.ev_off) == [0, 2, 3]


@pytest.mark.parametrize("text,err", [
    ("1 2\n", "3 or 4 columns"),
    ("1 2 3\n1 2 3 4\n", "mixed"),
    ("1 2 3 0\n1 2 3 1\n1 2 3 0\n", "contiguous"),
    ("1 2 nan\n", "non-finite"),
])
def test_malformed_files_are_rejected(tmp_path, text, err):
    path = tmp_path / "bad.txt"
    path.write_text(text)
    with pytest.raises(ValueError, match=err):
        carrier_io.load_carriers(str(path))
