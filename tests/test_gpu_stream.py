"""GPU parity of the stream calls (fc_state) against one FP64 oracle frame of the
repeated geometry: K TX calls give samples [0, K T) of the K-slot frame and carry its
last D samples; K RX calls (after one priming call) decode the K-slot frame slot by
slot. Bar: RMS-normalised error <= 1e-5 per slot, as for the frame calls."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests import parity
from tests.test_stream_semantics import STREAMABLE, k_slots, slot_len, stack_grids

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


def run_stream_case(torch, geom, K, S, seed):
    from paper_2008_00672_gb300 import Plan, State
    plan = Plan(geom)
    T, D = plan.slot_len, plan.stream_delay
    assert T == slot_len(geom) and D == fo.frame_len(geom) - T
    st = State(plan, S)
    grids = [c64(wl.qam_grid(geom, S, seed + 17 * k)).astype(np.complex128) for k in range(K)]
    # ---- TX: K calls, then one call on a zero grid flushes the carried tail ----
    outs = []
    for k in range(K + 1):
        g = grids[k] if k < K else np.zeros_like(grids[0])
        dg = torch.from_numpy(c64(g)).cuda()
        o = torch.empty((S, T), dtype=torch.complex64, device="cuda")
        st.tx(dg, o)
        outs.append(o.cpu().numpy())
    tx_stream = np.concatenate(outs, axis=1)          # [S][(K + 1) T]
    big_geom = k_slots(geom, K)
    worst_tx = 0.0
    refs = []
    for s in range(S):
        ref = fo.tx_frame(big_geom, stack_grids(geom, [grids[k][s] for k in range(K)]))
        assert len(ref) == K * T + D
        refs.append(ref)
        for k in range(K):
            worst_tx = max(worst_tx, rel(tx_stream[s, k * T:(k + 1) * T], ref[k * T:(k + 1) * T]))
        if D:
            worst_tx = max(worst_tx, rel(tx_stream[s, K * T:K * T + D], ref[K * T:]))
        parity.check(tx_stream[s, :K * T + D], ref, TOL, parity.wave_windows(big_geom), ("tx", s))
    # ---- RX: the K-slot frame plus noise, one priming call, then K calls ----
    x = np.stack([c64(wl.awgn(refs[s], 30.0, seed + 7919 * (s + 1))).astype(np.complex128) for s in range(S)])
    prime = np.zeros((S, T), dtype=np.complex128)
    if D:
        prime[:, T - D:] = x[:, :D]
    grid_out = torch.empty((S, plan.grid_len), dtype=torch.complex64, device="cuda")
    st.rx(torch.from_numpy(c64(prime)).cuda(), grid_out)
    est = []
    for k in range(K):
        chunk = torch.from_numpy(c64(x[:, D + k * T:D + (k + 1) * T])).cuda()
        st.rx(chunk, grid_out)
        est.append(grid_out.cpu().numpy())
    worst_rx = 0.0
    for s in range(S):
        ref = fo.split_grid(big_geom, fo.rx_frame(big_geom, x[s]))
        for k in range(K):
            got = fo.split_grid(geom, est[k][s])
            want = []
            for m in range(len(geom.subbands)):
                B = geom.groups[geom.subbands[m].group].n_symbols
                worst_rx = max(worst_rx, rel(got[m], ref[m][k * B:(k + 1) * B]))
                want.append(ref[m][k * B:(k + 1) * B].reshape(-1))
            parity.check(est[k][s], np.concatenate(want), TOL, parity.grid_windows(geom), ("rx", s, k))
    st.close()
    plan.close()
    return worst_tx, worst_rx


@pytest.mark.parametrize("name,geom", STREAMABLE, ids=[n for n, _ in STREAMABLE])
def test_stream_small_geometries(torch_cuda, name, geom):
    wt, wr = run_stream_case(torch_cuda, geom, 3, 3, 51)
    assert wt <= TOL and wr <= TOL, (name, wt, wr)


@pytest.mark.parametrize("flags", [0, 1])
def test_stream_nr20mhz_mixed_numerology(torch_cuda, flags):
    """Warp-specialised kernels (flags 0) and generic kernels (flags 1)."""
    geom = dataclasses.replace(wl.config_mixed_20mhz(), flags=flags)
    wt, wr = run_stream_case(torch_cuda, geom, 2, 2, 61)
    assert wt <= TOL and wr <= TOL, (wt, wr)


def test_stream_nr5mhz_continuous(torch_cuda):
    wt, wr = run_stream_case(torch_cuda, wl.config_single_5mhz(), 3, 2, 71)
    assert wt <= TOL and wr <= TOL, (wt, wr)


def test_state_reset_restarts_the_stream(torch_cuda):
    """After fc_state_reset a call gives what the first call of a fresh state gives."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan, State
    geom = STREAMABLE[0][1]
    plan = Plan(geom)
    g = torch.from_numpy(c64(wl.qam_grid(geom, 2, 5))).cuda()
    st = State(plan, 2)
    first = torch.empty((2, plan.slot_len), dtype=torch.complex64, device="cuda")
    again = torch.empty_like(first)
    st.tx(g, first)
    st.tx(g, again)
    assert not torch.equal(first, again)            # the second call adds the carried tail
    st.reset()
    st.tx(g, again)
    assert rel(again.cpu().numpy(), first.cpu().numpy()) < 1e-6
    st.close()
    plan.close()


def test_state_checkpoint_resumes_the_stream(torch_cuda):
    """fc_state_export / fc_state_import: a stream interrupted after two slots and resumed
    from its checkpoint in a new state gives what the uninterrupted stream gives, TX and
    RX (to rounding: reductions may add in another order); a checkpoint of another size,
    or one whose header names another state, is refused."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import FcError, Plan, State
    geom = STREAMABLE[0][1]
    plan = Plan(geom)
    S, T, K = 2, plan.slot_len, 4
    assert plan.stream_delay > 0
    grids = [torch.from_numpy(c64(wl.qam_grid(geom, S, 90 + k))).cuda() for k in range(K)]
    rng = np.random.default_rng(91)
    slots = [torch.from_numpy(c64(rng.standard_normal((S, T)) + 1j * rng.standard_normal((S, T)))).cuda()
             for _ in range(K)]

    def step(st, k):
        o = torch.empty((S, T), dtype=torch.complex64, device="cuda")
        e = torch.empty((S, plan.grid_len), dtype=torch.complex64, device="cuda")
        st.tx(grids[k], o)
        st.rx(slots[k], e)
        return o.cpu().numpy(), e.cpu().numpy()

    whole = State(plan, S)
    ref = [step(whole, k) for k in range(K)]
    first = State(plan, S)
    got = [step(first, k) for k in range(2)]
    ckpt = first.export()
    assert ckpt.size == 48 + 2 * S * plan.stream_delay * 8
    first.close()
    resumed = State(plan, S)
    resumed.load(ckpt)
    got += [step(resumed, k) for k in range(2, K)]
    for k, ((ro, re), (go, ge)) in enumerate(zip(ref, got)):
        assert rel(go, ro) < 1e-6 and rel(ge, re) < 1e-6, (k, rel(go, ro), rel(ge, re))
    with pytest.raises(FcError):
        resumed.load(ckpt[:-8])
    forged = ckpt.copy()
    forged[4:8] = np.frombuffer(np.int32(S + 1).tobytes(), dtype=np.uint8)   # header: another stream count
    with pytest.raises(FcError):
        resumed.load(forged)
    whole.close()
    resumed.close()
    plan.close()


def test_state_refused_for_a_geometry_that_cannot_stream(torch_cuda):
    from paper_2008_00672_gb300 import FcError, Plan, State
    from tests.test_stream_semantics import small_sync
    plan = Plan(small_sync(5, (16, 8, 8, 9)))
    assert plan.slot_len == 0
    with pytest.raises(FcError) as e:
        State(plan, 1)
    assert e.value.status == 2          # FC_ERR_UNSUPPORTED
    plan.close()
