"""The element-wise parity bounds catch what a whole-stream norm hides (CPU only).

The GPU tests compare with `tests/parity.py`; here its three bounds are exercised on
an oracle waveform of the 20 MHz mixed-numerology subframe (eq:multi-symb windows) and
on its QAM grid, with planted errors on copied arrays.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests import parity


@pytest.fixture(scope="module")
def frame():
    geom = wl.config_mixed_20mhz()
    grid = wl.qam_grid(geom, 1, 5)[0].astype(np.complex128)
    return geom, grid, fo.tx_frame(geom, grid)


def test_windows_cover_the_frame(frame):
    geom, grid, w = frame
    ws = parity.wave_windows(geom)
    # 14 symbols of the 15 kHz group and 28 of the 30 kHz group
    assert len(ws) == 14 + 28
    covered = np.zeros(w.size, bool)
    for a, b in ws:
        covered[a:b] = True
    assert covered.all()
    gw = parity.grid_windows(geom)
    assert gw[-1][1] == grid.size and len(gw) == 42


def test_complex64_rounding_passes(frame):
    geom, grid, w = frame
    s = parity.check(w.astype(np.complex64), w, 1e-5, parity.wave_windows(geom))
    assert s["rel"] < 1e-7 and s["sample"] < 1e-6


def test_single_sample_error_fails_only_per_sample(frame):
    geom, grid, w = frame
    rms = np.sqrt(np.mean(np.abs(w) ** 2))
    bad = w.astype(np.complex64).astype(np.complex128)
    bad[17001] += 1e-4 * rms
    s = parity.parity_stats(bad, w, parity.wave_windows(geom))
    assert s["rel"] <= 1e-5 and s["window"] <= 1e-5          # both norms pass
    with pytest.raises(AssertionError, match="per sample"):
        parity.check(bad, w, 1e-5, parity.wave_windows(geom))


def test_error_inside_one_window_fails_the_window_bound(frame):
    geom, grid, w = frame
    rms = np.sqrt(np.mean(np.abs(w) ** 2))
    bad = w.copy()
    a, b = parity.wave_windows(geom)[6]
    mid = (a + b) // 2
    bad[mid - 500:mid + 500] += 2e-5 * rms                     # below the per-sample bound
    s = parity.parity_stats(bad, w, parity.wave_windows(geom))
    assert s["rel"] <= 1e-5 and s["sample"] <= parity.SAMPLE_FACTOR * 1e-5
    with pytest.raises(AssertionError, match="window RMS"):
        parity.check(bad, w, 1e-5, parity.wave_windows(geom))


def test_one_bad_grid_row_fails(frame):
    geom, grid, w = frame
    rx = fo.rx_frame(geom, w)
    bad = rx.copy()
    a, b = parity.grid_windows(geom)[20]
    bad[a:b] *= 1 + 3e-5                                        # one symbol scaled
    s = parity.parity_stats(bad, rx, parity.grid_windows(geom))
    assert s["rel"] <= 1e-5
    with pytest.raises(AssertionError, match="window RMS"):
        parity.check(bad, rx, 1e-5, parity.grid_windows(geom))


def test_continuous_windows_hop_by_ns():
    geom = wl.config_single_5mhz()
    ws = parity.wave_windows(geom)
    g = geom.groups[0]
    d = fo.Dims(g, geom.subbands[0])
    assert all(b2[0] - b1[0] == d.N_S for b1, b2 in zip(ws, ws[1:]))
    assert ws[0] == (0, d.N) and ws[-1][1] == fo.frame_len(geom)
