"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Both sides get the same seeded inputs, rounded once to complex64 (the ABI's
type), so the comparison measures the FP32 computation only. The bar is the
RMS-normalised error ||gpu - oracle|| / ||oracle|| <= 1e-5, per stream, on the
TX waveform and on the RX QAM estimates, and beside it the same bound on every
symbol window (sigma_n .. sigma_n + 3N/2, or one FC block at hop N_S) of the
waveform and every symbol row of the grid, and 5e-5 of the signal RMS on every
single sample (`tests/parity.py`).
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests import parity

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import build
    build.build()
    return torch


def c64(a):
    return np.asarray(a).astype(np.complex64)


def rel(a, b):
    b = np.asarray(b)
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def gpu_tx_rx(torch, geom, grid, wave_rx, shape=None):
    from paper_2008_00672_gb300 import Plan
    plan = Plan(geom)
    for direction, (chunks, generic) in (shape or {}).items():   # a launch shape the autotuner can pick
        plan.set_choice(grid.shape[0], direction, chunks, generic)
    g = torch.from_numpy(c64(grid)).cuda()
    w = torch.empty((grid.shape[0], plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(g, w)
    wr = torch.from_numpy(c64(wave_rx)).cuda()
    est = torch.empty_like(g)
    plan.rx_analyze(wr, est)
    torch.cuda.synchronize()
    out = w.cpu().numpy(), est.cpu().numpy()
    plan.close()
    return out


def check_geometry(torch, geom, n_streams, seed, snr_db=30.0, streams_to_check=None, shape=None):
    grid = c64(wl.qam_grid(geom, n_streams, seed)).astype(np.complex128)
    idx = list(range(n_streams)) if streams_to_check is None else streams_to_check
    ref_tx = {s: fo.tx_frame(geom, grid[s]) for s in idx}
    # RX input: the oracle waveform plus AWGN, rounded to complex64 (same for both sides)
    flen = fo.frame_len(geom)
    wave_rx = np.zeros((n_streams, flen), dtype=np.complex128)
    for s in idx:
        wave_rx[s] = wl.awgn(ref_tx[s], snr_db, seed + 7919 * (s + 1))
    wave_rx = c64(wave_rx).astype(np.complex128)
    w, e = gpu_tx_rx(torch, geom, grid, wave_rx, shape)
    # FC_FLAG_REDUCED_RX: compare with the oracle's own eq:reduc form
    reduced = bool(geom.flags & 2) and geom.mode == wl.SYMBOL_SYNC and geom.scheme_rx == fo.OLS
    ww, gw = parity.wave_windows(geom), parity.grid_windows(geom)
    for s in idx:
        parity.check(w[s], ref_tx[s], TOL, ww, ("tx", s))
        parity.check(e[s], fo.rx_frame(geom, wave_rx[s], simplified=reduced), TOL, gw, ("rx", s))
    return w, e


def geom1(mode, stx, srx, N, N_O, L, Lo, act, c, n_cp, D=None, lead=-1):
    D = wl.rc_transition_weights(L, act if Lo == L else min(act, L - 8), 3) if D is None else D
    g = wl.Group(N, N_O, tuple(n_cp), lead)
    s = wl.Subband(L, Lo, act, c, 0, D)
    return wl.Geometry(mode, stx, srx, (g,), (s,))


# ---------------------------------------------------------------------------
# small geometries spanning the schemes, radices and edge cases
# ---------------------------------------------------------------------------

SYNC_SMALL = [
    # N, L, c, n_cp  (OLA/OLS TX x OLA/OLS RX)
    (32, 16, 3, (6, 4, 4, 5)),
    (64, 16, -5, (16, 0, 3, 16, 9)),             # L_CP = N_CP/4 floors, CP = N/4 and 0
    (48, 24, 7, (12, 9, 9)),                      # radix 3
    (128, 64, 60, (10, 9, 9, 9, 9, 9, 9)),        # subband wraps past the Nyquist bin
]


@pytest.mark.parametrize("stx", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("srx", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("case", SYNC_SMALL)
def test_sync_small(torch_cuda, stx, srx, case):
    N, L, c, n_cp = case
    geom = geom1(fo.SYMBOL_SYNC, stx, srx, N, N // 2, L, L, L - 8, c, n_cp)
    check_geometry(torch_cuda, geom, 3, 11)


CONT_SMALL = [
    # N, N_O, L, L_OFDM, act, c, n_cp, lead
    (64, 32, 48, 48, 36, -7, (8, 4, 4, 8), -1),          # I = 4/3, radix 3
    (64, 16, 32, 32, 24, 9, (6, 2, 2, 2), -1),            # lambda = 0.25
    (64, 32, 64, 64, 40, 0, (16, 8, 8), -1),              # I = 1
    (128, 64, 64, 32, 20, -20, (8, 4, 4, 4, 8), -1),      # L_OFDM < L
    (64, 32, 32, 32, 20, 5, (4, 2, 2, 2), 32),            # longer lead pad
    (64, 24, 32, 32, 20, -6, (8, 4, 4, 8), -1),           # lambda = 0.375
    (64, 48, 32, 32, 20, 3, (8, 4, 4, 8), -1),            # lambda = 0.75
]


@pytest.mark.parametrize("stx", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("srx", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("case", CONT_SMALL)
def test_continuous_small(torch_cuda, stx, srx, case):
    N, N_O, L, Lo, act, c, n_cp, lead = case
    D = wl.rc_transition_weights(L, min(act * L // Lo, L - 8), 3)
    geom = geom1(fo.CONTINUOUS, stx, srx, N, N_O, L, Lo, act, c, n_cp, D=D, lead=lead)
    check_geometry(torch_cuda, geom, 2, 13)


def test_sync_two_subbands_one_group_overlapping_transitions(torch_cuda):
    """Two subbands of different L share the long IDFT; their transition bins overlap and add."""
    g = wl.Group(128, 64, (12, 8, 8, 8))
    s1 = wl.Subband(64, 64, 36, -24, 0, wl.rc_transition_weights(64, 36, 6))
    s2 = wl.Subband(32, 32, 16, 20, 0, wl.rc_transition_weights(32, 16, 4))
    geom = wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (g,), (s1, s2))
    check_geometry(torch_cuda, geom, 2, 17)


def test_continuous_two_subbands_one_group(torch_cuda):
    g = wl.Group(128, 64, (16, 8, 8, 8))
    s1 = wl.Subband(64, 64, 40, -30, 0, wl.rc_transition_weights(64, 40, 6))
    s2 = wl.Subband(32, 32, 16, 40, 0, wl.rc_transition_weights(32, 16, 4))
    geom = wl.Geometry(fo.CONTINUOUS, fo.OLS, fo.OLA, (g,), (s1, s2))
    check_geometry(torch_cuda, geom, 2, 19)


def test_sync_three_groups_subband_order(torch_cuda):
    """Groups given out of order, subbands listed against the group order."""
    ga = wl.Group(64, 32, (12, 8, 8))
    gb = wl.Group(32, 16, (6, 4, 4, 4, 4, 4))
    gc = wl.Group(128, 64, (20, 16))
    sb = wl.Subband(16, 16, 10, 5, 1, wl.rc_transition_weights(16, 10, 2))
    sa = wl.Subband(32, 32, 20, -12, 0, wl.rc_transition_weights(32, 20, 3))
    sc = wl.Subband(64, 64, 30, 33, 2, wl.rc_transition_weights(64, 30, 4))
    geom = wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (ga, gb, gc), (sb, sc, sa))
    check_geometry(torch_cuda, geom, 3, 23)


def test_single_symbol_and_full_band(torch_cuda):
    geom = geom1(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, 32, 16, 32, 32, 32, 0, (8,), D=np.ones(32))
    check_geometry(torch_cuda, geom, 1, 29)


# ---------------------------------------------------------------------------
# the named 5G NR workloads
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [fo.CONTINUOUS, fo.SYMBOL_SYNC])
def test_nr10mhz_52prb(torch_cuda, mode):
    """The wide-band scenario of the paper's EVM figures (10 MHz, N = 1024, 52 PRB,
    L = 768), continuous and symbol-synchronized, on the generic kernels."""
    check_geometry(torch_cuda, wl.config_nr10mhz_52prb(mode), 3, 17)


def test_nr5mhz_single_subband_ols(torch_cuda):
    check_geometry(torch_cuda, wl.config_single_5mhz(), 3, wl.default_seed(1))


@pytest.mark.parametrize("flags", [0, 1, 2])
def test_nr20mhz_mixed_numerology_symbol_sync(torch_cuda, flags):
    """flags=0: warp-specialised kernels; flags=1: generic shared-memory kernels;
    flags=2: warp kernels with the eq:reduc RX for the L = 1024 subband."""
    geom = dataclasses.replace(wl.config_mixed_20mhz(), flags=flags)
    check_geometry(torch_cuda, geom, 2, wl.default_seed(2))


WARP_CASES = [
    # (N, L, act, c, n_cp, stx, srx)
    (2048, 1024, 612, -300, (160, 144, 144), fo.OLA, fo.OLS),
    (2048, 1024, 600, 700, (144, 0, 512, 16), fo.OLS, fo.OLA),     # band wraps past N/2; CP 0 and N/4
    (2048, 1024, 1000, -1, (8, 9, 7), fo.OLA, fo.OLA),             # odd starts: float2 reductions
    (1024, 512, 288, 159, (88, 72, 72, 72), fo.OLA, fo.OLS),
    (1024, 512, 500, -400, (0, 256, 30, 72, 72), fo.OLS, fo.OLS),   # two TX pairs and a single
    (1024, 512, 400, 3, (40,), fo.OLA, fo.OLA),                       # one symbol: no TX pair
    (2048, 1024, 500, 100, (144,), fo.OLS, fo.OLS),                   # one symbol: only the initialising TX launch
]


@pytest.mark.parametrize("case", WARP_CASES)
def test_warp_path_single_group(torch_cuda, case):
    N, L, act, c, n_cp, stx, srx = case
    D = wl.rc_transition_weights(L, act, min(8, (L - act) // 2))
    geom = geom1(fo.SYMBOL_SYNC, stx, srx, N, N // 2, L, L, act, c, n_cp, D=D)
    check_geometry(torch_cuda, geom, 3, 31)


@pytest.mark.parametrize("case", [c for c in WARP_CASES if c[6] == fo.OLS])
def test_reduced_rx_single_group(torch_cuda, case):
    """eq:reduc RX (FC_FLAG_REDUCED_RX) against the oracle's eq:reduc form; for L = 512
    the flag is ignored and the direct kernel runs (same result up to rounding)."""
    N, L, act, c, n_cp, stx, srx = case
    D = wl.rc_transition_weights(L, act, min(8, (L - act) // 2))
    geom = dataclasses.replace(geom1(fo.SYMBOL_SYNC, stx, srx, N, N // 2, L, L, act, c, n_cp, D=D), flags=2)
    check_geometry(torch_cuda, geom, 3, 41)


@pytest.mark.parametrize("flags", [0, 2])
def test_warp_path_two_groups_odd_offsets(torch_cuda, flags):
    """Two numerology groups whose alignment puts group B at an odd sample offset."""
    ga = wl.Group(2048, 1024, (161, 144, 144))
    gb = wl.Group(1024, 512, (88, 72, 72, 72, 72, 72))
    sa = wl.Subband(1024, 1024, 600, -310, 0, wl.rc_transition_weights(1024, 600, 8))
    sb = wl.Subband(512, 512, 280, 160, 1, wl.rc_transition_weights(512, 280, 8))
    geom = wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (ga, gb), (sa, sb), flags=flags)
    check_geometry(torch_cuda, geom, 2, 37)


@pytest.mark.parametrize("N,L,cps", [(2048, 1024, ((160, 144, 144, 144), (150, 144, 144, 154))),
                                      (1024, 512, ((72, 72, 88), (80, 72, 80)))])
def test_warp_path_two_groups_same_numerology(torch_cuda, N, L, cps):
    """Two groups of one numerology (one subband each, both halves of the band): with two
    N = 2048 groups no launch initialises the waveform (a memset zeroes it); with two
    N = 1024 groups both groups' symbol pairs share one launch."""
    act = 12 * (L // 48)
    ga, gb = wl.Group(N, N // 2, cps[0]), wl.Group(N, N // 2, cps[1])
    sa = wl.Subband(L, L, act, -N // 4, 0, wl.rc_transition_weights(L, act, 8))
    sb = wl.Subband(L, L, act, N // 4 + 1, 1, wl.rc_transition_weights(L, act, 8))
    geom = wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (ga, gb), (sa, sb))
    check_geometry(torch_cuda, geom, 2, 43)


def test_nr100mhz_two_slots(torch_cuda):
    check_geometry(torch_cuda, wl.config_100mhz(2), 1, wl.default_seed(3))


# ---------------------------------------------------------------------------
# batching: a stream's result does not depend on the batch it runs in
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,flags", [("mixed20", 0), ("mixed20", 1), ("single5", 0)])
def test_batch_invariance(torch_cuda, name, flags):
    """A stream alone (many chunks per stream) and inside a large batch (one chunk
    per stream) gives the same output: bit-identical where each output sample is
    written once (RX, generic TX), within 1e-6 where the warp-specialised TX adds
    overlapping blocks with floating-point reductions in arbitrary order."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan
    geom = dataclasses.replace(wl.NAMED[name](), flags=flags)
    plan = Plan(geom)
    big = 333
    grid = c64(wl.qam_grid(geom, 4, 5)).astype(np.complex64)
    gbig = np.tile(grid, (big // 4 + 1, 1))[:big]
    g1 = torch.from_numpy(grid[2:3].copy()).cuda()
    gb = torch.from_numpy(gbig).cuda()
    w1 = torch.empty((1, plan.wave_len), dtype=torch.complex64, device="cuda")
    wb = torch.empty((big, plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(g1, w1)
    plan.tx_synthesize(gb, wb)
    e1 = torch.empty_like(g1)
    eb = torch.empty_like(gb)
    plan.rx_analyze(w1, e1)
    plan.rx_analyze(wb, eb)
    torch.cuda.synchronize()
    warp_tx = geom.mode == wl.SYMBOL_SYNC and flags == 0
    for k in range(2, big, 4):
        if warp_tx:
            assert rel(wb[k].cpu().numpy(), w1[0].cpu().numpy()) <= 1e-6
            assert rel(eb[k].cpu().numpy(), e1[0].cpu().numpy()) <= 1e-6
        else:
            assert torch.equal(wb[k], w1[0])
            assert torch.equal(eb[k], e1[0])
    # RX alone on an identical input is deterministic on every path
    eb2 = torch.empty_like(gb)
    wsame = w1.repeat(big, 1).contiguous()
    plan.rx_analyze(wsame, eb2)
    torch.cuda.synchronize()
    for k in range(0, big, 37):
        assert torch.equal(eb2[k], eb2[0])


# ---------------------------------------------------------------------------
# full benchmark size: sampled streams against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [None, {0: (1, 0), 1: (4, 0)}, {0: (2, 0), 1: (2, 0)}],
                         ids=["built-in", "tx1-rx4", "tx2-rx2"])
def test_bench_size_sampled_streams(torch_cuda, shape):
    """The benchmark's batch of 1 ms subframes (2048 streams) in the launch shapes its
    set-up autotuning picks (chunks per stream for TX / RX; measured: TX 1, RX 4):
    three sampled streams, including the last, against the oracle."""
    geom = wl.config_mixed_20mhz()
    check_geometry(torch_cuda, geom, 2048, wl.default_seed(2), streams_to_check=[0, 1025, 2047], shape=shape)


# ---------------------------------------------------------------------------
# ABI argument handling on a device
# ---------------------------------------------------------------------------

def test_warp_path_unaligned_output_falls_back(torch_cuda):
    """An 8-byte (not 16-byte) aligned waveform buffer takes the generic TX kernel
    and still matches the oracle."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan
    geom = wl.config_mixed_20mhz()
    plan = Plan(geom)
    grid = c64(wl.qam_grid(geom, 1, 41))
    g = torch.from_numpy(grid).cuda()
    raw = torch.empty(plan.wave_len + 1, dtype=torch.complex64, device="cuda")
    w = raw[1:]
    assert w.data_ptr() % 16 == 8
    plan.tx_synthesize(g, w.view(1, -1))
    torch.cuda.synchronize()
    parity.check(w.cpu().numpy(), fo.tx_frame(geom, grid[0].astype(np.complex128)), TOL,
                 parity.wave_windows(geom))


def test_abi_errors_and_noop(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import fc
    geom = wl.config_single_5mhz()
    p = fc.Plan(geom)
    # zero streams: no-op, even with NULL buffers
    fc.fc_tx_synthesize(p.handle, 0, None, None)
    g = torch.zeros((1, p.grid_len), dtype=torch.complex64, device="cuda")
    w = torch.zeros((1, p.wave_len), dtype=torch.complex64, device="cuda")
    with pytest.raises(fc.FcError) as ei:     # workspace missing (continuous mode needs one)
        fc.fc_tx_synthesize(p.handle, 1, g.data_ptr(), w.data_ptr(), 0, 0)
    assert ei.value.status == fc.FC_ERR_INVALID
    with pytest.raises(fc.FcError):
        fc.fc_rx_analyze(p.handle, -1, w.data_ptr(), g.data_ptr())
    with pytest.raises(fc.FcError):
        fc.fc_tx_synthesize(p.handle, 1, None, w.data_ptr())
    p.close()


# ---------------------------------------------------------------------------
# the one-warp-per-pair continuous kernels (L = 384, N = 512, overlap-save side)
# ---------------------------------------------------------------------------

W384_CASES = [
    # n_cp (multiples of 4: L_CP = 3 N_CP / 4), c, active, TX, RX, lead pad (high rate)
    ((40, 36, 36, 36, 36, 36, 36), 0, 288, fo.OLS, fo.OLS, -1),
    ((40, 36, 36), -100, 200, fo.OLS, fo.OLA, -1),        # warp TX, generic RX
    ((36, 36, 40, 36, 36), 150, 300, fo.OLA, fo.OLS, -1),  # generic TX, warp RX
    ((40,), 7, 100, fo.OLS, fo.OLS, 384),                  # one symbol, longer lead pad
    ((0, 4, 8, 12), 255, 360, fo.OLS, fo.OLS, -1),         # band edge at the Nyquist bin
]


@pytest.mark.parametrize("case", W384_CASES)
def test_warp_continuous_384_512(torch_cuda, case):
    n_cp, c, act, stx, srx, lead = case
    D = wl.rc_transition_weights(384, act, min(8, (384 - act) // 2))
    geom = geom1(fo.CONTINUOUS, stx, srx, 512, 256, 384, 384, act, c, n_cp, D=D, lead=lead)
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Plan
    plan = Plan(geom)
    for d, side in ((FC_TX, stx), (FC_RX, srx)):
        assert plan.choice(3, d)[1] == (0 if side == fo.OLS else 1), (d, plan.choice(3, d))
    plan.close()
    check_geometry(torch_cuda, geom, 3, 43)


def test_nr5mhz_bench_size_sampled(torch_cuda):
    """The 5 MHz slot workload at the bench's launch (2^16 slots, one per stream) on the
    warp continuous kernels: three sampled streams, the last included, TX against the
    oracle and RX (on the TX output) against the oracle."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan
    geom = wl.config_single_5mhz()
    S = 1 << 16
    plan = Plan(geom)
    base = c64(wl.qam_grid(geom, 64, wl.default_seed(1)))
    grid = torch.from_numpy(base).cuda().repeat(S // 64, 1).contiguous()
    wave = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    est = torch.empty_like(grid)
    ws = plan.workspace(S)
    plan.tx_synthesize(grid, wave, ws)
    plan.rx_analyze(wave, est, ws)
    torch.cuda.synchronize()
    for s in (0, S // 2 + 5, S - 1):
        g = base[s % 64].astype(np.complex128)
        w = wave[s].cpu().numpy()
        parity.check(w, fo.tx_frame(geom, g), TOL, parity.wave_windows(geom), ("tx", s))
        parity.check(est[s].cpu().numpy(), fo.rx_frame(geom, w.astype(np.complex128)), TOL,
                     parity.grid_windows(geom), ("rx", s))
    plan.close()
