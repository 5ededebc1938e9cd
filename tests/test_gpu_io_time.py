"""GPU parity of the time-domain I/O (FC_FLAG_IO_TIME: the FC part alone) against the
oracle's time-domain entry points, on arbitrary (non-OFDM) complex inputs, with the
element-wise bounds of `tests/parity.py` (every FC block or symbol window of the
waveform and every recovered symbol body, and every sample)."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests import parity

pytestmark = pytest.mark.gpu
TOL = 1e-5
IO_TIME = 8


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import build
    build.build()
    return torch


def c64(a):
    return np.asarray(a).astype(np.complex64)


def check(torch, geom, S, seed, tol=TOL):
    from paper_2008_00672_gb300 import Plan
    plan = Plan(geom)
    n_tx, n_rx = (sum(x) for x in fo.time_lengths(geom))
    assert (plan.tx_in_len, plan.rx_out_len) == (n_tx, n_rx)
    rng = np.random.default_rng(seed)
    t_in = c64(rng.standard_normal((S, n_tx)) + 1j * rng.standard_normal((S, n_tx)))
    w = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(torch.from_numpy(t_in).cuda(), w)
    x = c64(rng.standard_normal((S, plan.wave_len)) + 1j * rng.standard_normal((S, plan.wave_len)))
    t_out = torch.empty((S, n_rx), dtype=torch.complex64, device="cuda")
    plan.rx_analyze(torch.from_numpy(x).cuda(), t_out)
    torch.cuda.synchronize()
    w, t_out = w.cpu().numpy(), t_out.cpu().numpy()
    ww, bw = parity.wave_windows(geom), parity.body_windows(geom)
    for s in range(S):
        parity.check(w[s], fo.tx_frame(geom, t_in[s].astype(np.complex128), io_time=True), tol, ww, ("tx", s))
        parity.check(t_out[s], fo.rx_frame(geom, x[s].astype(np.complex128), io_time=True), tol, bw, ("rx", s))
    plan.close()


def two_subbands(mode, stx, srx):
    g = wl.Group(64, 32, (16, 8, 8, 12) if mode == fo.SYMBOL_SYNC else (8, 8, 8, 8))
    subs = (wl.Subband(32, 32, 18, 7, 0, wl.rc_transition_weights(32, 18, 3)),
            wl.Subband(32, 32, 10, -12, 0, wl.rc_transition_weights(32, 10, 3)))
    return wl.Geometry(mode, stx, srx, (g,), subs, flags=IO_TIME)


@pytest.mark.parametrize("mode,stx,srx", [(fo.SYMBOL_SYNC, fo.OLA, fo.OLS), (fo.SYMBOL_SYNC, fo.OLS, fo.OLA),
                                          (fo.CONTINUOUS, fo.OLA, fo.OLA), (fo.CONTINUOUS, fo.OLS, fo.OLS)])
def test_time_io_small(torch_cuda, mode, stx, srx):
    check(torch_cuda, two_subbands(mode, stx, srx), 3, 7)


def test_time_io_nr20mhz_mixed_numerology(torch_cuda):
    check(torch_cuda, dataclasses.replace(wl.config_mixed_20mhz(), flags=IO_TIME), 2, 8)


def test_time_io_tensor_path(torch_cuda):
    """FC_FLAG_TENSOR_DFT with time I/O: the block passes on the tensor cores, the OFDM
    passes replaced by copies."""
    check(torch_cuda, dataclasses.replace(wl.config_100mhz(1), flags=IO_TIME | 4), 1, 9, tol=3e-5)
