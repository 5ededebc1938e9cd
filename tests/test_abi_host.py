"""CPU-side checks of the C-ABI library: it loads, exports every function the
header declares, and its host-only geometry validation agrees with the oracle's
frame arithmetic and rejects what the paper's equations do not define."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fcofdm.h")


@pytest.fixture(scope="module")
def fc():
    from paper_2008_00672_gb300 import build
    build.build()
    from paper_2008_00672_gb300 import fc as fcmod
    fcmod.load_library()
    return fcmod


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(fc_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["fc_plan_create", "fc_tx_synthesize", "fc_rx_analyze", "fc_plan_destroy", "fc_query",
              "fc_geometry_check", "fc_status_string", "fc_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(fc):
    lib = fc.load_library()
    for n in declared_functions():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", fc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_status_strings(fc):
    for code in range(6):
        assert fc.fc_status_string(code).startswith("FC_")


def _sizes_match(fc, geom):
    s = fc.fc_geometry_check(geom)
    assert s.wave_len == fo.frame_len(geom)
    assert s.grid_len == geom.grid_len()
    return s


@pytest.mark.parametrize("name", ["single5", "mixed20"])
def test_sizes_match_oracle_named(fc, name):
    geom = wl.NAMED[name]()
    s = _sizes_match(fc, geom)
    assert s.nominal_len == geom.nominal_samples()
    if geom.mode == wl.SYMBOL_SYNC:
        assert s.workspace_per_stream == 0


def test_sizes_match_oracle_100mhz(fc):
    geom = wl.config_100mhz(10)
    s = _sizes_match(fc, geom)
    assert s.nominal_len == 614400
    assert s.workspace_per_stream > 0


def test_nominal_samples_printed_configs(fc):
    """One slot at 7.68 Msps = 7680 samples; 1 ms at 30.72 Msps = 30720."""
    assert fc.fc_geometry_check(wl.config_single_5mhz()).nominal_len == 7680
    assert fc.fc_geometry_check(wl.config_mixed_20mhz()).nominal_len == 30720


def _g(mode, N, N_O, L, Lo, act, c, ncp, lead=-1, stx=0, srx=1):
    g = wl.Group(N, N_O, tuple(ncp), lead)
    s = wl.Subband(L, Lo, act, c, 0, np.ones(L))
    return wl.Geometry(mode, stx, srx, (g,), (s,))


@pytest.mark.parametrize("geom,code", [
    (_g(1, 32, 8, 16, 16, 8, 0, (2,)), 1),            # symbol-sync needs lambda = 0.5
    (_g(1, 32, 16, 16, 16, 8, 0, (9,)), 1),           # N_CP > N/4
    (_g(1, 32, 16, 18, 18, 8, 0, (2,)), 1),           # 4 does not divide L
    (_g(1, 32, 16, 16, 32, 8, 0, (2,)), 1),           # L_OFDM != L in symbol-sync mode
    (_g(0, 32, 16, 16, 16, 8, 0, (3,)), 1),           # fractional low-rate CP in continuous mode
    (_g(0, 32, 10, 24, 24, 8, 0, (0,)), 1),           # L_O = N_O L/N not an integer
    (_g(0, 32, 16, 16, 16, 20, 0, (4,)), 1),          # L_act > L_OFDM
    (_g(0, 32, 16, 16, 16, 8, 0, (4,), lead=4), 1),   # lead pad shorter than L_L
    (_g(0, 8192, 4096, 8192, 8192, 8, 0, (0,)), 2),   # beyond the largest built transform
    (_g(0, 40, 20, 40, 40, 8, 0, (0,)), 2),           # 5 is not a built radix
])
def test_invalid_geometry_rejected(fc, geom, code):
    with pytest.raises(fc.FcError) as ei:
        fc.fc_geometry_check(geom)
    assert ei.value.status == code


def _ns(mode=0, stx=0, srx=1, groups=((32, 16, -1, (4,)),), subs=((16, 16, 8, 0, 0),)):
    """A geometry as plain attributes (no workload-side validation), for the ABI checks."""
    from types import SimpleNamespace as NS
    gs = tuple(NS(n_long=N, n_overlap=NO, lead_pad=lead, n_cp=tuple(cp)) for N, NO, lead, cp in groups)
    ss = tuple(NS(l_short=L, l_ofdm=Lo, n_active=act, centre_bin=c, group=g, weights=np.ones(L))
               for L, Lo, act, c, g in subs)
    return NS(mode=mode, scheme_tx=stx, scheme_rx=srx, groups=gs, subbands=ss, flags=0)


@pytest.mark.parametrize("geom,code,why", [
    (_ns(mode=7), 1, "unknown mode"),
    (_ns(stx=5), 1, "unknown OLA/OLS scheme"),
    (_ns(groups=((32, 32, -1, (4,)),)), 1, "need 0 <= N_O < N"),
    (_ns(groups=((32, 16, -1, ()),)), 1, "need n_symbols >= 1"),
    (_ns(groups=((32, 16, -1, (4, -4)),)), 1, "negative N_CP"),
    (_ns(groups=((40, 20, -1, (0,)),), subs=((20, 20, 8, 0, 0),)), 2, "N must be 2^a 3^b"),
    (_ns(subs=((16, 16, 8, 0, 3),)), 1, "subband group out of range"),
    (_ns(subs=((64, 64, 8, 0, 0),)), 1, "need 1 <= L <= N"),
    (_ns(subs=((16, 16, 0, 0, 0),)), 1, "need 1 <= L_act <= L_OFDM"),
    (_ns(groups=((32, 16, -1, (0,)),), subs=((24, 16, 8, 0, 0),)), 1, "N_OFDM = L_OFDM N / L is not an integer"),
    (_ns(groups=((32, 16, -1, (4,)), (32, 16, -1, (4,))),), 1, "a group has no subband"),
    (_ns(subs=((16, 16, 8, -4, 0), (16, 8, 4, 6, 0))), 1, "equal high-rate durations"),
])
def test_invalid_geometry_rejected_more(fc, geom, code, why):
    """Each host-side check of fc_geometry_check, reached by a geometry that breaks only it."""
    with pytest.raises(fc.FcError) as ei:
        fc.fc_geometry_check(geom)
    assert ei.value.status == code and why in str(ei.value), str(ei.value)


def test_oracle_rejects_the_same_invalid_geometry():
    """The oracle refuses the geometries the paper leaves undefined, as the library does."""
    for geom in [_g(1, 32, 8, 16, 16, 8, 0, (2,)), _g(1, 32, 16, 16, 16, 8, 0, (9,)),
                 _g(0, 32, 16, 16, 16, 8, 0, (3,))]:
        with pytest.raises(ValueError):
            fo.tx_frame(geom, np.zeros(geom.grid_len(), complex))


def _stream_cases():
    from tests.test_stream_semantics import STREAMABLE, small_sync
    named = [(n, wl.NAMED[n]()) for n in ("single5", "mixed20")]
    return named + list(STREAMABLE), small_sync(5, (16, 8, 8, 9))


def test_stream_sizes_match_the_slot_identities(fc):
    """slot_len / stream_delay from the planner agree with the slot duration and the
    one-slot frame of the oracle for every geometry whose stream identities hold."""
    from tests.test_stream_semantics import slot_len
    good, bad = _stream_cases()
    for name, geom in good:
        s = fc.fc_geometry_check(geom)
        assert s.slot_len == slot_len(geom), name
        assert s.stream_delay == fo.frame_len(geom) - slot_len(geom), name
    assert fc.fc_geometry_check(bad).slot_len == 0      # c_m T / N not an integer


def test_stream_sizes_refuse_unequal_group_slots(fc):
    """Two groups whose CP lists last different times cannot share a stream slot."""
    ga = wl.Group(64, 32, (16, 16, 16, 16))
    gb = wl.Group(32, 16, (8,) * 6)
    sa = wl.Subband(32, 32, 20, 6, 0, wl.rc_transition_weights(32, 20, 3))
    sb = wl.Subband(16, 16, 10, -4, 1, wl.rc_transition_weights(16, 10, 2))
    geom = wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (ga, gb), (sa, sb))
    assert fc.fc_geometry_check(geom).slot_len == 0


def test_uneven_carriers_plan_on_the_host(fc):
    """Every carrier of the uneven multi-carrier workload is a valid geometry with the
    oracle's frame and grid sizes, and the draw covers every bandwidth and SCS."""
    carriers = wl.config_uneven_carriers()
    assert len(carriers) == 64
    seen_bw, seen_scs = set(), set()
    for c in carriers:
        s = fc.fc_geometry_check(c)
        assert s.wave_len == fo.frame_len(c) and s.grid_len == c.grid_len(), c.name
        _, bw, scs, _ = c.name.split("_")
        seen_bw.add(bw)
        seen_scs.add(scs)
        n = c.groups[0].n_long
        assert n & (n - 1) == 0 and 128 <= n <= 4096
    assert seen_bw == {"5MHz", "10MHz", "20MHz", "50MHz", "100MHz"}
    assert seen_scs == {"15kHz", "30kHz", "60kHz"}


def test_tensor_flag_plans_its_workspace(fc):
    """FC_FLAG_TENSOR_DFT on the 100 MHz carrier: R rows of 4096 bins more workspace
    and three TX / RX kernels; other geometries ignore the flag."""
    import dataclasses
    geom = wl.config_100mhz(2)
    a = fc.fc_geometry_check(geom)
    b = fc.fc_geometry_check(dataclasses.replace(geom, flags=4))
    d = fo.Dims(geom.groups[0], geom.subbands[0])
    n_low = sum(fo.low_rate_cp(d, fo.CONTINUOUS)) + d.B * d.L_ofdm
    R = fo.continuous_block_count(n_low, fo.lead_pad_low(geom.groups[0], d), d)
    assert b.workspace_per_stream - a.workspace_per_stream == R * 4096 * 8
    assert (b.tx_kernels, b.rx_kernels) == (3, 3)
    m = wl.config_mixed_20mhz()
    assert fc.fc_geometry_check(dataclasses.replace(m, flags=4)).workspace_per_stream == 0


def test_time_io_sizes(fc):
    """Time-domain I/O lengths follow the oracle's layout; the active I/O lengths switch
    from the grid to them only with FC_FLAG_IO_TIME."""
    import dataclasses
    for name in ("single5", "mixed20"):
        geom = wl.NAMED[name]()
        s = fc.fc_geometry_check(geom)
        tx, rx = fo.time_lengths(geom)
        assert (s.time_tx_len, s.time_rx_len) == (sum(tx), sum(rx))
        assert (s.tx_in_len, s.rx_out_len) == (s.grid_len, s.grid_len)
        t = fc.fc_geometry_check(dataclasses.replace(geom, flags=8))
        assert (t.tx_in_len, t.rx_out_len) == (sum(tx), sum(rx))


def test_bf16_io_sizes(fc):
    """FC_FLAG_IO_BF16 halves the bytes of a sample and nothing else: the lengths stay,
    the workspace stays FP32, and the tensor-core passes (which accumulate into the
    output) give way to the generic kernels. A symbol-sync plan of the one-warp kernels
    adds its TX blocks into a complex64 frame in the workspace (one frame a stream) and
    rounds it into the BF16 output in a second launch; its RX widens the BF16 waveform
    into that frame first."""
    import dataclasses
    for geom in (wl.config_single_5mhz(), wl.config_mixed_20mhz(), wl.config_100mhz(2)):
        a = fc.fc_geometry_check(geom)
        b = fc.fc_geometry_check(dataclasses.replace(geom, flags=16))
        assert (a.sample_bytes, b.sample_bytes) == (8, 4)
        for f in ("grid_len", "wave_len", "slot_len", "stream_delay", "tx_in_len", "rx_out_len"):
            assert getattr(a, f) == getattr(b, f), f
        if geom.mode == fo.SYMBOL_SYNC:
            assert a.workspace_per_stream == 0
            assert b.workspace_per_stream == 8 * (b.wave_len + b.wave_len % 2)
            # one launch per numerology group's job shape (two here; TX: the N = 2048
            # jobs in two, the even symbols' initialising the waveform), + the BF16 pass
            assert (a.tx_kernels, a.rx_kernels) == (3, 2)
            assert (b.tx_kernels, b.rx_kernels) == (4, 3)
        else:
            assert b.workspace_per_stream == a.workspace_per_stream
    g = wl.config_100mhz(2)
    t = fc.fc_geometry_check(dataclasses.replace(g, flags=4 | 16))
    assert (t.tx_kernels, t.rx_kernels) == (2, 2)
    assert t.workspace_per_stream == fc.fc_geometry_check(g).workspace_per_stream
    it = fc.fc_geometry_check(dataclasses.replace(wl.config_single_5mhz(), flags=8 | 16))
    assert it.sample_bytes == 4 and it.tx_in_len == it.time_tx_len


def test_warp_launch_counts(fc):
    """Symbol-sync plans of the one-warp kernels launch one kernel per numerology job shape
    and direction; TX adds one where the plan's only N = 2048 group's even symbols
    initialise the waveform (two N = 2048 groups: a memset instead); complex-BF16 I/O
    adds its rounding / widening pass. Plans outside the one-warp shapes: one launch."""
    import dataclasses

    def sync(groups, subs):
        return wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, tuple(groups), tuple(subs))

    A = lambda cps: wl.Group(2048, 1024, cps)                      # noqa: E731
    B = lambda cps: wl.Group(1024, 512, cps)                       # noqa: E731
    sa = lambda c, g: wl.Subband(1024, 1024, 480, c, g, wl.rc_transition_weights(1024, 480, 8))   # noqa: E731
    sb = lambda c, g: wl.Subband(512, 512, 240, c, g, wl.rc_transition_weights(512, 240, 8))      # noqa: E731
    cases = [
        (sync([A((144, 144, 144))], [sa(0, 0)]), (2, 1)),          # init + odd symbols
        (sync([A((144,))], [sa(0, 0)]), (1, 1)),                   # one symbol: the init launch alone
        (sync([B((72, 72, 72))], [sb(0, 0)]), (1, 1)),             # memset + pairs
        (sync([A((160, 144, 144, 144)), A((150, 144, 144, 154))], [sa(-512, 0), sa(513, 1)]), (1, 1)),
        (wl.config_mixed_20mhz(), (3, 2)),
    ]
    for geom, (tx, rx) in cases:
        z = fc.fc_geometry_check(geom)
        assert (z.tx_kernels, z.rx_kernels) == (tx, rx), (geom.name, z.tx_kernels, z.rx_kernels)
        b = fc.fc_geometry_check(dataclasses.replace(geom, flags=16))
        assert (b.tx_kernels, b.rx_kernels) == (tx + 1, rx + 1)
    g = fc.fc_geometry_check(dataclasses.replace(wl.config_mixed_20mhz(), flags=1))   # generic kernels
    assert (g.tx_kernels, g.rx_kernels) == (1, 1)


def test_no_gpu_fails_loudly(fc):
    """There is no CPU path: without a usable GPU, creating a plan or a server returns
    FC_ERR_CUDA (and the binding raises) instead of computing anything on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for make in (lambda: fc.fc_plan_create(wl.config_single_5mhz()), lambda: fc.fc_server_create(0, 1, 0)):
        with pytest.raises(fc.FcError) as ei:
            make()
        assert ei.value.status == fc.FC_ERR_CUDA
