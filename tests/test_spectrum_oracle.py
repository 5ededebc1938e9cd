"""Spectral containment on the oracle (CPU), with the PSD estimator bench.py reports.

The paper's wide-band scenario (10 MHz, 52 PRB, 15 kHz) states that the out-of-band PSD
of continuous FC processing is about 5 dB below that of discontinuous (symbol-
synchronized) processing, with the paper's own transition weights. With this
repository's raised-cosine weights the oracle gives 4 dB on the mean out-of-band level;
the test asks for 2-8 dB, and for both FC forms to sit far below unfiltered CP-OFDM (FC
with I = 1 and all-ones weights, the delayed identity)."""
import numpy as np

import bench
import workloads as wl
from oracle import fc_oracle as fo

CH = 5000.0 / 15.0          # 10 MHz channel edge, in 15 kHz subcarrier spacings


def oob(geom, streams=16):
    q = wl.qam_grid(geom, streams, 77)
    w = np.stack([fo.tx_frame(geom, q[s]) for s in range(streams)])
    return bench.psd_out_of_band(w, 1024, 624, CH)


def test_estimator_on_white_noise_is_flat():
    rng = np.random.default_rng(5)
    w = rng.standard_normal((8, 16384)) + 1j * rng.standard_normal((8, 16384))
    r = bench.psd_out_of_band(w, 1024, 624, CH)
    assert all(abs(v) < 1.0 for v in r.values()), r


def test_continuous_below_symsync_below_plain():
    cont = oob(wl.config_nr10mhz_52prb(wl.CONTINUOUS))
    sync = oob(wl.config_nr10mhz_52prb(wl.SYMBOL_SYNC))
    plain = oob(bench.plain_cp_ofdm_nr10mhz())
    assert plain["oob_mean_db"] > -45.0, plain                    # sinc sidelobes of plain CP-OFDM
    assert sync["oob_mean_db"] < plain["oob_mean_db"] - 50.0, (sync, plain)
    gap = sync["oob_mean_db"] - cont["oob_mean_db"]
    assert 2.0 <= gap <= 8.0, (cont, sync)
    for k in ("edge_plus_180khz_db", "edge_plus_500khz_db", "edge_plus_1000khz_db"):
        assert cont[k] < sync[k] < plain[k], (k, cont, sync, plain)
