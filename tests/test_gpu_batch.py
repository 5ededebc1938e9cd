"""GPU: batch executor (uneven carriers side by side, CUDA graph replay) and the
autotuner. Every batched result must equal the item's own call (same kernels, so up
to the order of floating-point reductions) and the FP64 oracle (<= 1e-5 per stream and
per symbol window or grid row, 5e-5 of the signal RMS per sample: `tests/parity.py`)."""
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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def c64(a):
    return np.asarray(a).astype(np.complex64)


def setup(torch, carriers, n_streams, seed):
    from paper_2008_00672_gb300 import Plan
    out = []
    for i, geom in enumerate(carriers):
        plan = Plan(geom)
        grid = c64(wl.qam_grid(geom, n_streams, seed + 31 * i))
        out.append(dict(geom=geom, plan=plan, grid_np=grid.astype(np.complex128),
                        grid=torch.from_numpy(grid).cuda(),
                        wave=torch.zeros((n_streams, plan.wave_len), dtype=torch.complex64, device="cuda"),
                        rx_in=None, est=torch.zeros((n_streams, plan.grid_len), dtype=torch.complex64,
                                                    device="cuda")))
    return out


@pytest.mark.parametrize("use_graph,persistent", [(True, False), (False, False), (True, True), (False, True)])
def test_batch_uneven_carriers_match_oracle(torch_cuda, use_graph, persistent):
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Batch
    carriers = wl.config_uneven_carriers(seed=1400, n_carriers=8, n_slots=1)
    S = 2
    cs = setup(torch, carriers, S, 500)
    # RX inputs: the oracle waveform of each carrier plus 30 dB AWGN
    for j, c in enumerate(cs):
        ref = [fo.tx_frame(c["geom"], c["grid_np"][s]) for s in range(S)]
        c["ref_tx"] = ref
        x = np.stack([c64(wl.awgn(ref[s], 30.0, 77 + 13 * j + s)).astype(np.complex128) for s in range(S)])
        c["rx_np"] = x
        c["rx_in"] = torch.from_numpy(c64(x)).cuda()
    items = [(c["plan"], FC_TX, c["grid"], c["wave"]) for c in cs] + \
            [(c["plan"], FC_RX, c["rx_in"], c["est"]) for c in cs]
    b = Batch(items, n_lanes=4, use_graph=use_graph, persistent=persistent)
    for _ in range(2):                       # second launch replays the graph
        for c in cs:
            c["wave"].zero_()
            c["est"].zero_()
        b.launch()
        torch.cuda.synchronize()
        for c in cs:
            w, e = c["wave"].cpu().numpy(), c["est"].cpu().numpy()
            ww, gw = parity.wave_windows(c["geom"]), parity.grid_windows(c["geom"])
            for s in range(S):
                parity.check(w[s], c["ref_tx"][s], TOL, ww, (c["geom"].name, "tx", s))
                parity.check(e[s], fo.rx_frame(c["geom"], c["rx_np"][s]), TOL, gw, (c["geom"].name, "rx", s))
    # new inputs in the same buffers: the replayed graph reads them
    for i, c in enumerate(cs):
        g2 = c64(wl.qam_grid(c["geom"], S, 900 + i))
        c["grid"].copy_(torch.from_numpy(g2))
        c["ref_tx"] = [fo.tx_frame(c["geom"], g2[s].astype(np.complex128)) for s in range(S)]
    b.launch()
    torch.cuda.synchronize()
    for c in cs:
        w = c["wave"].cpu().numpy()
        for s in range(S):
            parity.check(w[s], c["ref_tx"][s], TOL, parity.wave_windows(c["geom"]), (c["geom"].name, s))
    b.close()
    for c in cs:
        c["plan"].close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_warp_carriers_match_oracle(torch_cuda, use_graph):
    """One-warp carriers in a batch, captured into a CUDA graph (their calls are chains of
    programmatic dependent launches: the symbol-sync TX initialising launch, the
    per-shape launches, the continuous kernels' second launch) or run on lanes."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Batch
    carriers = [wl.config_mixed_20mhz(), wl.config_single_5mhz(), wl.config_mixed_20mhz()]
    S = 2
    cs = setup(torch, carriers, S, 700)
    for j, c in enumerate(cs):
        ref = [fo.tx_frame(c["geom"], c["grid_np"][s]) for s in range(S)]
        c["ref_tx"] = ref
        x = np.stack([c64(wl.awgn(ref[s], 30.0, 91 + 13 * j + s)).astype(np.complex128) for s in range(S)])
        c["rx_np"] = x
        c["rx_in"] = torch.from_numpy(c64(x)).cuda()
    items = [(c["plan"], FC_TX, c["grid"], c["wave"]) for c in cs] + \
            [(c["plan"], FC_RX, c["rx_in"], c["est"]) for c in cs]
    b = Batch(items, n_lanes=3, use_graph=use_graph)
    for _ in range(2):                       # the second launch replays the graph
        for c in cs:
            c["wave"].fill_(1.0)             # the TX calls initialise their waveforms themselves
            c["est"].zero_()
        b.launch()
        torch.cuda.synchronize()
        for c in cs:
            w, e = c["wave"].cpu().numpy(), c["est"].cpu().numpy()
            ww, gw = parity.wave_windows(c["geom"]), parity.grid_windows(c["geom"])
            for s in range(S):
                parity.check(w[s], c["ref_tx"][s], TOL, ww, (c["geom"].name, "tx", s))
                parity.check(e[s], fo.rx_frame(c["geom"], c["rx_np"][s]), TOL, gw, (c["geom"].name, "rx", s))
    b.close()
    for c in cs:
        c["plan"].close()


def test_batch_equals_single_calls(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_TX, Batch
    carriers = wl.config_uneven_carriers(seed=1401, n_carriers=12, n_slots=1)
    cs = setup(torch, carriers, 3, 600)
    b = Batch([(c["plan"], FC_TX, c["grid"], c["wave"]) for c in cs], n_lanes=6, use_graph=True)
    b.launch()
    torch.cuda.synchronize()
    for c in cs:
        single = torch.empty_like(c["wave"])
        c["plan"].tx_synthesize(c["grid"], single)
        torch.cuda.synchronize()
        assert rel(c["wave"].cpu().numpy(), single.cpu().numpy()) < 1e-6, c["geom"].name
    b.close()


def test_autotune_keeps_results_and_records_a_choice(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Plan
    geom = wl.config_mixed_20mhz()
    plan = Plan(geom)
    S = 40
    grid = torch.from_numpy(c64(wl.qam_grid(geom, S, 3))).cuda()
    before = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(grid, before)
    plan.autotune(S, reps=3)
    for d in (FC_TX, FC_RX):
        k, generic = plan.choice(S, d)
        assert k in (1, 2, 4, 8, 16, 32, 64) and generic in (0, 1)
    after = torch.empty_like(before)
    plan.tx_synthesize(grid, after)
    torch.cuda.synchronize()
    ref = fo.tx_frame(geom, c64(wl.qam_grid(geom, S, 3))[S - 1].astype(np.complex128))
    parity.check(after[S - 1].cpu().numpy(), ref, TOL, parity.wave_windows(geom))
    assert rel(after.cpu().numpy(), before.cpu().numpy()) < 1e-6
    plan.close()


def test_set_choice_round_trip_and_validation(torch_cuda):
    from paper_2008_00672_gb300 import FC_RX, FC_TX, FcError, Plan
    plan = Plan(wl.config_mixed_20mhz())
    plan.set_choice(100, FC_RX, 4, 0)
    assert plan.choice(100, FC_RX) == (4, 0)
    plan.set_choice(100, FC_TX, 2, 1)
    assert plan.choice(100, FC_TX) == (2, 1)
    with pytest.raises(FcError):
        plan.set_choice(100, FC_TX, 3, 0)          # not a split the plan has
    plan.close()


@pytest.mark.parametrize("name", ["nr5_cont", "mixed20_generic"])
def test_cta_sizes_give_identical_results(torch_cuda, name):
    """The generic kernels come in 512-, 256- and 128-thread CTAs, picked per call by the
    number of CTAs it launches (and the persistent queues take the smallest that fits).
    Every element sees the same operations in the same order whatever the CTA size, so a
    stream's result is bit-identical: alone (one stream, 256-thread CTAs), among 1024
    streams (128-thread CTAs where the plan fits them) and in a persistent batch."""
    import dataclasses
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Batch, Plan
    geom = wl.config_single_5mhz() if name == "nr5_cont" else \
        dataclasses.replace(wl.config_mixed_20mhz(), flags=1)
    plan = Plan(geom)
    S = 1024
    base = c64(wl.qam_grid(geom, 4, 700))
    grid = torch.from_numpy(base).cuda().repeat(S // 4, 1).contiguous()
    wave = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    est = torch.empty_like(grid)
    plan.tx_synthesize(grid, wave)
    plan.rx_analyze(wave, est)
    w1 = torch.empty((1, plan.wave_len), dtype=torch.complex64, device="cuda")
    e1 = torch.empty((1, plan.grid_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(grid[:1], w1)
    plan.rx_analyze(wave[:1], e1)
    torch.cuda.synchronize()
    assert torch.equal(w1[0], wave[0]) and torch.equal(e1[0], est[0])
    if geom.mode == 1:                      # symbol-sync: the persistent queues
        wb = torch.empty((2, plan.wave_len), dtype=torch.complex64, device="cuda")
        eb = torch.empty((2, plan.grid_len), dtype=torch.complex64, device="cuda")
        b = Batch([(plan, FC_TX, grid[:2], wb), (plan, FC_RX, wave[:2], eb)], n_lanes=2, persistent=True)
        b.launch()
        torch.cuda.synchronize()
        assert torch.equal(wb, wave[:2]) and torch.equal(eb, est[:2])
        b.close()
    plan.close()


@pytest.mark.parametrize("persistent", [True, False])
def test_batch_autotune_keeps_results(torch_cuda, persistent):
    """fc_batch_autotune times the whole batch under each candidate chunk count and keeps
    the fastest; the replayed graph still matches the oracle."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_RX, FC_TX, Batch
    carriers = wl.config_uneven_carriers(seed=1402, n_carriers=8, n_slots=1)
    S = 2
    cs = setup(torch, carriers, S, 700)
    for j, c in enumerate(cs):
        c["ref_tx"] = [fo.tx_frame(c["geom"], c["grid_np"][s]) for s in range(S)]
        x = np.stack([c64(wl.awgn(c["ref_tx"][s], 30.0, 91 + 13 * j + s)).astype(np.complex128) for s in range(S)])
        c["rx_np"] = x
        c["rx_in"] = torch.from_numpy(c64(x)).cuda()
    items = [(c["plan"], FC_TX, c["grid"], c["wave"]) for c in cs] + \
            [(c["plan"], FC_RX, c["rx_in"], c["est"]) for c in cs]
    b = Batch(items, n_lanes=4, use_graph=True, persistent=persistent)
    b.launch()
    b.autotune(reps=2)
    for c in cs:
        c["wave"].zero_()
        c["est"].zero_()
    b.launch()
    torch.cuda.synchronize()
    for c in cs:
        w, e = c["wave"].cpu().numpy(), c["est"].cpu().numpy()
        ww, gw = parity.wave_windows(c["geom"]), parity.grid_windows(c["geom"])
        for s in range(S):
            parity.check(w[s], c["ref_tx"][s], TOL, ww, (c["geom"].name, "tx", s))
            parity.check(e[s], fo.rx_frame(c["geom"], c["rx_np"][s]), TOL, gw, (c["geom"].name, "rx", s))
    b.close()
    for c in cs:
        c["plan"].close()


def test_autotune_radix_schedules(torch_cuda):
    """On the generic kernels the autotuner also picks a radix schedule per transform size
    (written into the plan's tables); every schedule multiplies out to its size, uses the
    kernels' radices, and the tuned plan still matches the oracle."""
    torch = torch_cuda
    import dataclasses
    from paper_2008_00672_gb300 import Plan
    geom = dataclasses.replace(wl.config_mixed_20mhz(), flags=1)         # generic kernels
    plan = Plan(geom)
    before = {n: plan.radices(n) for n in (512, 1024, 2048)}
    assert before[1024] == [16, 8, 8] and before[2048] == [16, 16, 8] and before[512] == [8, 8, 8]
    S = 24
    plan.autotune(S, reps=2)
    for n in (512, 1024, 2048):
        r = plan.radices(n)
        assert int(np.prod(r)) == n and set(r) <= {2, 4, 8, 16}, (n, r)
    grid = c64(wl.qam_grid(geom, S, 9))
    w = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(torch.from_numpy(grid).cuda(), w)
    est = torch.empty((S, plan.grid_len), dtype=torch.complex64, device="cuda")
    plan.rx_analyze(w, est)
    torch.cuda.synchronize()
    for s in (0, S - 1):
        ref = fo.tx_frame(geom, grid[s].astype(np.complex128))
        parity.check(w[s].cpu().numpy(), ref, TOL, parity.wave_windows(geom), s)
        parity.check(est[s].cpu().numpy(), fo.rx_frame(geom, w[s].cpu().numpy().astype(np.complex128)), TOL,
                     parity.grid_windows(geom), s)
    plan.close()
