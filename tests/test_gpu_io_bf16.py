"""GPU parity of complex-BF16 I/O (FC_FLAG_IO_BF16) against the FP64 oracle fed the same
BF16 inputs.

A BF16 output sample is the exact result rounded once to BF16: every real component g
is the BF16 rounding of some value within the FP32 path's error budget
eps = 1e-5 rms(y) of the oracle's FP64 value y (y lies within eps of the interval of
reals that round to g), and at least 95 % of the components equal the oracle's own
rounding bf16_round(y) bit for bit (rounding toward zero would miss about half). The
others sit within eps of a rounding boundary or of zero, where the BF16 spacing is
finest: about 0.1 % of them at 1024 points, 2 % for the 4096-point carrier. The same
holds for the slots of
the stream calls, whose TX tail and RX look-behind stay FP32 (one rounding per slot
sample); batches (graph and persistent queues, BF16 and complex64 items side by side),
host pipelines and the server return the frame calls' bytes exactly, except where the
one-warp symbol-sync TX adds overlapping blocks with FP32 reductions in arbitrary
order: two runs then differ in the last FP32 bit of some sums, and a BF16 output by
one BF16 step where such a sum sits at a rounding boundary (a few in 10^5).
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests.test_stream_semantics import k_slots, stack_grids

pytestmark = pytest.mark.gpu
TOL = 1e-5
BF16 = 16
IO_TIME = 8


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import build
    build.build()
    return torch


def to_bf16(torch, x):
    """Complex input samples -> bfloat16 (re, im) host tensor (the input quantisation)."""
    c = torch.from_numpy(np.ascontiguousarray(np.asarray(x).astype(np.complex64)))
    return torch.view_as_real(c).to(torch.bfloat16).contiguous()


def to_c128(t):
    """bfloat16 (re, im) tensor -> complex128 numpy array (exact)."""
    import torch
    a = t.detach().cpu().to(torch.float64).numpy()
    return a[..., 0] + 1j * a[..., 1]


def rounding_interval(g):
    """[lo, hi]: the reals that round to the BF16 values g (ties aside)."""
    a = np.abs(g)
    _, ex = np.frexp(a)                                   # a = f 2^ex, 1/2 <= f < 1
    e = np.maximum(ex - 1, -126)
    up = np.ldexp(1.0, e - 7)                             # spacing above a
    down = np.where((a == np.ldexp(1.0, ex - 1)) & (ex - 1 > -126), up / 2, up)   # below a power of two
    lo_mag, hi_mag = a - down / 2, a + up / 2
    tiny = 2.0**-134
    lo = np.where(g > 0, lo_mag, np.where(g < 0, -hi_mag, -tiny))
    hi = np.where(g > 0, hi_mag, np.where(g < 0, -lo_mag, tiny))
    return lo, hi


def check_rounded(g, y, what):
    """g: one stream's BF16 result (complex128), y: the oracle's FP64 result. Every
    component of g must be the BF16 rounding of some value within the FP32 budget
    eps = 1e-5 rms(y) of y, i.e. y lies within eps of g's rounding interval."""
    g, y = np.asarray(g), np.asarray(y)
    assert g.shape == y.shape, what
    eps = TOL * float(np.sqrt(np.mean(np.abs(y) ** 2)))
    agree = 0
    for gp, yp in ((g.real, y.real), (g.imag, y.imag)):
        lo, hi = rounding_interval(gp)
        out = np.maximum(lo - yp, yp - hi)
        assert np.all(out <= eps), (what, float(out.max() / eps), int(np.argmax(out)))
        agree += int(np.count_nonzero(gp == fo.bf16_round(yp)))
    frac = agree / (2 * g.size)
    assert frac >= 0.95, (what, frac)
    return frac


def assert_bf16_match(a, b, what="", max_frac=1e-3):
    """Two BF16 results of the same call: equal, but for at most max_frac of the
    components, which differ by one BF16 step (FP32 sums of the one-warp TX reduced in
    another order, rounded on either side of a boundary)."""
    import torch
    ia, ib = a.detach().cpu().view(torch.int16), b.detach().cpu().view(torch.int16)
    diff = ia != ib
    n = int(diff.sum())
    if n == 0:
        return
    fa = a.detach().cpu().float()[diff].double().numpy()
    fb = b.detach().cpu().float()[diff].double().numpy()
    step = np.ldexp(1.0, np.frexp(np.maximum(np.abs(fa), np.abs(fb)))[1] - 8)   # BF16 spacing there
    assert np.all(np.abs(fa - fb) <= step), (what, "more than one BF16 step")
    assert n <= max_frac * diff.numel(), (what, n, diff.numel())


def tx_rx_case(torch, geom, S, seed, io_time=False):
    """Frame TX and RX of a BF16 plan against the oracle on BF16-quantised inputs."""
    from paper_2008_00672_gb300 import Plan
    plan = Plan(geom)
    assert plan.io_bf16 and plan.sample_bytes == 4
    rng = np.random.default_rng(seed)
    if io_time:
        n_in = plan.tx_in_len
        src = (rng.standard_normal((S, n_in)) + 1j * rng.standard_normal((S, n_in))) * 0.5
    else:
        src = wl.qam_grid(geom, S, seed)
    g_in = to_bf16(torch, src)
    w = torch.empty((S, plan.wave_len, 2), dtype=torch.bfloat16, device="cuda")
    plan.tx_synthesize(g_in.cuda(), w)
    src_q = to_c128(g_in)
    refs = [fo.tx_frame(geom, src_q[s], io_time=io_time) for s in range(S)]
    x = np.stack([wl.awgn(refs[s], 30.0, seed + 11 * s) for s in range(S)])
    x_in = to_bf16(torch, x)
    est = torch.empty((S, plan.rx_out_len, 2), dtype=torch.bfloat16, device="cuda")
    plan.rx_analyze(x_in.cuda(), est)
    torch.cuda.synchronize()
    w_np, est_np, x_q = to_c128(w), to_c128(est), to_c128(x_in)
    for s in range(S):
        check_rounded(w_np[s], refs[s], (geom.name, "tx", s))
        check_rounded(est_np[s], fo.rx_frame(geom, x_q[s], io_time=io_time), (geom.name, "rx", s))
    plan.close()


def two_subbands(mode, stx, srx, flags=BF16):
    g = wl.Group(64, 32, (16, 8, 8, 12) if mode == fo.SYMBOL_SYNC else (8, 8, 8, 8))
    subs = (wl.Subband(32, 32, 18, 7, 0, wl.rc_transition_weights(32, 18, 3)),
            wl.Subband(32, 32, 10, -12, 0, wl.rc_transition_weights(32, 10, 3)))
    return wl.Geometry(mode, stx, srx, (g,), subs, flags=flags, name=f"two_subbands_{mode}{stx}{srx}")


MODES = [(fo.SYMBOL_SYNC, fo.OLA, fo.OLS), (fo.SYMBOL_SYNC, fo.OLS, fo.OLA),
         (fo.CONTINUOUS, fo.OLA, fo.OLA), (fo.CONTINUOUS, fo.OLS, fo.OLS)]


@pytest.mark.parametrize("mode,stx,srx", MODES)
def test_bf16_small(torch_cuda, mode, stx, srx):
    tx_rx_case(torch_cuda, two_subbands(mode, stx, srx), 3, 21)


@pytest.mark.parametrize("mode,stx,srx", MODES[::3])
def test_bf16_time_io(torch_cuda, mode, stx, srx):
    tx_rx_case(torch_cuda, two_subbands(mode, stx, srx, BF16 | IO_TIME), 2, 22, io_time=True)


def test_bf16_nr5mhz_continuous(torch_cuda):
    tx_rx_case(torch_cuda, dataclasses.replace(wl.config_single_5mhz(), flags=BF16), 3, 23)


def test_bf16_nr20mhz_mixed_numerology(torch_cuda):
    """The one-warp-per-symbol kernels with BF16 I/O (TX into a complex64 frame in the
    workspace, then one rounding pass; RX from the waveform widened into that frame)."""
    geom = dataclasses.replace(wl.config_mixed_20mhz(), flags=BF16)
    from paper_2008_00672_gb300 import Plan
    p = Plan(geom)
    # one launch per numerology group's job shape (TX: the N = 2048 jobs in two), + the
    # rounding (TX) / widening (RX) pass
    assert (p.tx_kernels, p.rx_kernels) == (4, 3) and p.workspace_per_stream >= 8 * p.wave_len
    p.close()
    tx_rx_case(torch_cuda, geom, 2, 24)


WARP_BF16 = [
    # (N, L, act, c, n_cp, stx, srx, flags)
    (2048, 1024, 600, 700, (144, 0, 512, 16), fo.OLS, fo.OLA, BF16),   # band past N/2, CP 0 and N/4, OLA RX
    (2048, 1024, 1000, -1, (8, 9, 7), fo.OLA, fo.OLS, BF16 | 2),       # odd starts; eq:reduc flag: direct form
    (1024, 512, 500, -400, (0, 256, 30, 72, 72), fo.OLS, fo.OLA, BF16),
]


@pytest.mark.parametrize("case", WARP_BF16)
def test_bf16_warp_path_single_group(torch_cuda, case):
    N, L, act, c, n_cp, stx, srx, flags = case
    g = wl.Group(N, N // 2, n_cp)
    sb = wl.Subband(L, L, act, c, 0, wl.rc_transition_weights(L, act, min(8, (L - act) // 2)))
    geom = wl.Geometry(fo.SYMBOL_SYNC, stx, srx, (g,), (sb,), flags=flags, name=f"warp_bf16_{N}_{stx}{srx}")
    tx_rx_case(torch_cuda, geom, 3, 27)


def test_bf16_warp_path_two_groups_odd_offsets(torch_cuda):
    ga = wl.Group(2048, 1024, (161, 144, 144))
    gb = wl.Group(1024, 512, (88, 72, 72, 72, 72, 72))
    sa = wl.Subband(1024, 1024, 600, -310, 0, wl.rc_transition_weights(1024, 600, 8))
    sb = wl.Subband(512, 512, 280, 160, 1, wl.rc_transition_weights(512, 280, 8))
    geom = wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (ga, gb), (sa, sb), flags=BF16, name="warp_bf16_two_groups")
    tx_rx_case(torch_cuda, geom, 2, 28)


def test_bf16_uneven_carriers(torch_cuda):
    for geom in wl.config_uneven_carriers(seed=1402, n_carriers=5, n_slots=1):
        tx_rx_case(torch_cuda, dataclasses.replace(geom, flags=BF16), 1, 25)


def test_bf16_tensor_flag_takes_the_generic_path(torch_cuda):
    """FC_FLAG_TENSOR_DFT with BF16 I/O on the 100 MHz carrier: the FP32 kernels run
    (two per direction) and the result is the oracle's, rounded."""
    from paper_2008_00672_gb300 import Plan
    geom = dataclasses.replace(wl.config_100mhz(1), flags=BF16 | 4)
    p = Plan(geom)
    assert (p.tx_kernels, p.rx_kernels) == (2, 2)
    p.close()
    tx_rx_case(torch_cuda, geom, 1, 26)


def test_bf16_streams_round_once(torch_cuda):
    """K stream calls of a BF16 plan give the K-slot frame of the repeated geometry,
    rounded once per sample (the carried tail is added in FP32)."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan, State
    for base in (wl.config_mixed_20mhz(), wl.config_single_5mhz()):
        geom = dataclasses.replace(base, flags=BF16)
        K, S = 2, 2
        plan = Plan(geom)
        T, D = plan.slot_len, plan.stream_delay
        st = State(plan, S)
        grids_in = [to_bf16(torch, wl.qam_grid(geom, S, 31 + k)) for k in range(K)]
        grids = [to_c128(g) for g in grids_in]
        outs = []
        for k in range(K + 1):
            gin = grids_in[k] if k < K else torch.zeros_like(grids_in[0])
            o = torch.empty((S, T, 2), dtype=torch.bfloat16, device="cuda")
            st.tx(gin.cuda(), o)
            outs.append(to_c128(o))
        tx_stream = np.concatenate(outs, axis=1)
        big = k_slots(geom, K)
        refs = []
        for s in range(S):
            ref = fo.tx_frame(big, stack_grids(geom, [grids[k][s] for k in range(K)]))
            refs.append(ref)
            check_rounded(tx_stream[s, :K * T + D], ref, (geom.name, "stream tx", s))
        # RX: BF16 slots of the noisy K-slot frame after a priming call
        x = np.stack([wl.awgn(refs[s], 30.0, 41 + s) for s in range(S)])
        x_in = to_bf16(torch, x)
        x_q = to_c128(x_in)
        prime = torch.zeros((S, T, 2), dtype=torch.bfloat16)
        if D:
            prime[:, T - D:] = x_in[:, :D]
        est = torch.empty((S, plan.grid_len, 2), dtype=torch.bfloat16, device="cuda")
        st.rx(prime.cuda(), est)
        got = []
        for k in range(K):
            st.rx(x_in[:, D + k * T:D + (k + 1) * T].contiguous().cuda(), est)
            got.append(to_c128(est))
        for s in range(S):
            ref = fo.split_grid(big, fo.rx_frame(big, x_q[s]))
            for k in range(K):
                parts = fo.split_grid(geom, got[k][s])
                for m in range(len(geom.subbands)):
                    B = geom.groups[geom.subbands[m].group].n_symbols
                    check_rounded(parts[m], ref[m][k * B:(k + 1) * B], (geom.name, "stream rx", s, k, m))
        st.close()
        plan.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_bf16_batch_equals_frame_calls(torch_cuda, persistent):
    """BF16 and complex64 items in one batch (graph replay; persistent: per-type queues)
    give exactly the bytes of their own frame calls."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Batch, Plan
    carriers = wl.config_uneven_carriers(seed=1403, n_carriers=6, n_slots=1)
    cs = []
    for i, g in enumerate(carriers):
        bf = i % 2 == 0
        geom = dataclasses.replace(g, flags=BF16 if bf else 0)
        plan = Plan(geom)
        S = 2
        q = wl.qam_grid(geom, S, 50 + i)
        if bf:
            grid = to_bf16(torch, q).cuda()
            wave = torch.zeros((S, plan.wave_len, 2), dtype=torch.bfloat16, device="cuda")
            est = torch.zeros((S, plan.grid_len, 2), dtype=torch.bfloat16, device="cuda")
        else:
            grid = torch.from_numpy(q.astype(np.complex64)).cuda()
            wave = torch.zeros((S, plan.wave_len), dtype=torch.complex64, device="cuda")
            est = torch.zeros((S, plan.grid_len), dtype=torch.complex64, device="cuda")
        rx_in = torch.empty_like(wave)
        plan.tx_synthesize(grid, rx_in)
        cs.append((plan, grid, wave, rx_in, est))
    items = [(c[0], FC_TX, c[1], c[2]) for c in cs] + [(c[0], FC_RX, c[3], c[4]) for c in cs]
    b = Batch(items, n_lanes=3, use_graph=True, persistent=persistent)
    for _ in range(2):
        b.launch()
    torch.cuda.synchronize()
    for plan, grid, wave, rx_in, est in cs:
        w1, e1 = torch.empty_like(wave), torch.empty_like(est)
        plan.tx_synthesize(grid, w1)
        plan.rx_analyze(rx_in, e1)
        torch.cuda.synchronize()
        assert torch.equal(w1.view(torch.int16) if w1.dtype == torch.bfloat16 else w1,
                           wave.view(torch.int16) if wave.dtype == torch.bfloat16 else wave)
        assert torch.equal(e1.view(torch.int16) if e1.dtype == torch.bfloat16 else e1,
                           est.view(torch.int16) if est.dtype == torch.bfloat16 else est)
    b.close()
    for c in cs:
        c[0].close()


def test_bf16_host_pipeline_equals_device_calls(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import Pipeline, Plan
    geom = dataclasses.replace(wl.config_mixed_20mhz(), flags=BF16)
    plan = Plan(geom)
    S = 5
    h_grid = to_bf16(torch, wl.qam_grid(geom, S, 61)).pin_memory()
    h_wave = torch.empty((S, plan.wave_len, 2), dtype=torch.bfloat16).pin_memory()
    h_est = torch.empty((S, plan.grid_len, 2), dtype=torch.bfloat16).pin_memory()
    pipe = Pipeline(plan, chunk_streams=2, depth=2)
    pipe.tx(h_grid, h_wave)
    torch.cuda.synchronize()
    pipe.rx(h_wave, h_est)
    torch.cuda.synchronize()
    d_wave = torch.empty((S, plan.wave_len, 2), dtype=torch.bfloat16, device="cuda")
    d_est = torch.empty((S, plan.grid_len, 2), dtype=torch.bfloat16, device="cuda")
    plan.tx_synthesize(h_grid.cuda(), d_wave)
    plan.rx_analyze(d_wave, d_est)
    torch.cuda.synchronize()
    assert plan.tx_kernels == 4                       # the one-warp TX (three launches), rounding pass
    assert_bf16_match(h_wave, d_wave, "pipeline tx")
    # RX writes every output once: the same bytes (its input is the pipeline's waveform)
    plan.rx_analyze(h_wave.cuda(), d_est)
    torch.cuda.synchronize()
    assert torch.equal(h_est.view(torch.int16), d_est.cpu().view(torch.int16))
    pipe.close()
    plan.close()


def test_bf16_served_slots_equal_stream_calls(torch_cuda):
    """A BF16 carrier and a complex64 carrier served together: every BF16 result equals
    that carrier's own stream calls byte for byte."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Plan, Server, State
    g_bf = dataclasses.replace(wl.config_single_5mhz(), flags=BF16)
    g_c = wl.config_mixed_20mhz()
    srv = Server(n_lanes=2)
    a, c = srv.add_carrier(g_bf), srv.add_carrier(g_c)
    za, zc = srv.sizes[a], srv.sizes[c]
    assert (za.sample_bytes, zc.sample_bytes) == (4, 8)
    rng = np.random.default_rng(71)
    reqs, ours = [], []
    t = 0.0
    for k in range(6):
        d = FC_TX if k % 3 != 2 else FC_RX
        if d == FC_TX:
            h_in = to_bf16(torch, wl.qam_grid(g_bf, 1, 80 + k)[0]).pin_memory()
            h_out = torch.empty((za.slot_len, 2), dtype=torch.bfloat16).pin_memory()
        else:
            x = (rng.standard_normal(za.slot_len) + 1j * rng.standard_normal(za.slot_len)) * 0.05
            h_in = to_bf16(torch, x).pin_memory()
            h_out = torch.empty((za.grid_len, 2), dtype=torch.bfloat16).pin_memory()
        reqs.append((t, a, d, h_in, h_out))
        ours.append((d, h_in, h_out))
        q = torch.from_numpy(wl.qam_grid(g_c, 1, 90 + k)[0].astype(np.complex64)).pin_memory()
        reqs.append((t, c, FC_TX, q, torch.empty(zc.slot_len, dtype=torch.complex64).pin_memory()))
        t += 2e-4
    srv.run(reqs)
    srv.close()
    plan = Plan(g_bf)
    st = State(plan, 1)
    for d, h_in, h_out in ours:
        dev_in = h_in.cuda().unsqueeze(0)
        if d == FC_TX:
            o = torch.empty((1, za.slot_len, 2), dtype=torch.bfloat16, device="cuda")
            st.tx(dev_in, o)
        else:
            o = torch.empty((1, za.grid_len, 2), dtype=torch.bfloat16, device="cuda")
            st.rx(dev_in, o)
        torch.cuda.synchronize()
        assert torch.equal(o[0].cpu().view(torch.int16), h_out.view(torch.int16))
    st.close()
    plan.close()


def test_bf16_alignment_and_dtype_checks(torch_cuda):
    """BF16 buffers need 4-byte alignment (checked before any launch); the binding
    refuses complex64 tensors for a BF16 plan."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan, fc
    geom = dataclasses.replace(wl.config_single_5mhz(), flags=BF16)
    plan = Plan(geom)
    g = torch.zeros(plan.grid_len * 2 + 8, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(plan.wave_len * 2 + 8, dtype=torch.bfloat16, device="cuda")
    ws = plan.workspace(1)
    wsp, wsb = (ws.data_ptr(), ws.numel()) if ws is not None else (0, 0)
    fc.fc_tx_synthesize(plan.handle, 1, g.data_ptr() + 4, w.data_ptr() + 4, wsp, wsb)     # 4-byte aligned: fine
    with pytest.raises(fc.FcError) as e:
        fc.fc_tx_synthesize(plan.handle, 1, g.data_ptr() + 2, w.data_ptr(), wsp, wsb)
    assert e.value.status == fc.FC_ERR_INVALID
    torch.cuda.synchronize()
    with pytest.raises(ValueError):
        plan.tx_synthesize(torch.zeros((1, plan.grid_len), dtype=torch.complex64, device="cuda"),
                           torch.zeros((1, plan.wave_len), dtype=torch.complex64, device="cuda"))
    plan.close()
