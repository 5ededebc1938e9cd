"""GPU: the serving loop with continuous batching. A carrier's results do not depend on
what else is served (alone vs mixed), they equal the carrier's own stream calls, requests
of different carriers that arrive together run in one batch whose device interval they
share, a request arena too small for everything still serves every request as memory
frees up, and admission refuses a carrier that does not fit above the HBM reserve."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import build
    build.build()
    return torch


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


def make_requests(torch, sizes, trace, seed):
    """Pinned host buffers per request: QAM grids for TX, noise-like slots for RX."""
    rng = np.random.default_rng(seed)
    reqs = []
    for t, cid, d in trace:
        z = sizes[cid]
        if d == 0:
            x = (rng.choice([-1.0, 1.0], z.grid_len) + 1j * rng.choice([-1.0, 1.0], z.grid_len)) / np.sqrt(2)
            out_len = z.slot_len
        else:
            x = (rng.standard_normal(z.slot_len) + 1j * rng.standard_normal(z.slot_len)) * 0.01
            out_len = z.grid_len
        h_in = torch.from_numpy(x.astype(np.complex64)).pin_memory()
        h_out = torch.zeros(out_len, dtype=torch.complex64).pin_memory()
        reqs.append((t, cid, d, h_in, h_out))
    return reqs


def serve(carriers, reqs, n_lanes=4):
    from paper_2008_00672_gb300 import Server
    srv = Server(n_lanes=n_lanes)
    for g in carriers:
        srv.add_carrier(g)
    lat = srv.run(reqs)
    srv.close()
    return lat


def test_alone_equals_mixed(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import fc
    carriers = wl.config_uneven_carriers(seed=1500, n_carriers=4, n_slots=1, whole_cp_period=True)
    sizes = [fc.fc_geometry_check(g) for g in carriers]
    trace = wl.serving_trace(len(carriers), 48, 4000.0, 9)
    mixed = make_requests(torch, sizes, trace, 1)
    lat = serve(carriers, mixed)
    assert all(0.0 < x < 1.0 for x in lat)
    for c in range(len(carriers)):
        mine = [(t, 0, d, h_in, torch.zeros_like(h_out).pin_memory())
                for (t, cid, d, h_in, h_out) in mixed if cid == c]
        if not mine:
            continue
        serve([carriers[c]], mine)
        got = [r[4].numpy() for r in mine]
        want = [r[4].numpy() for r in mixed if r[1] == c]
        for a, b in zip(got, want):
            assert rel(a, b) < 1e-6, carriers[c].name


def test_served_slots_equal_stream_calls(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan, State, fc
    geom = wl.config_uneven_carriers(seed=1501, n_carriers=1, n_slots=1, whole_cp_period=True)[0]
    z = fc.fc_geometry_check(geom)
    trace = [(1e-4 * k, 0, d) for k, d in enumerate([0, 0, 1, 0, 1, 1])]
    reqs = make_requests(torch, [z], trace, 2)
    serve([geom], reqs, n_lanes=1)
    plan = Plan(geom)
    st = State(plan, 1)
    for t, _, d, h_in, h_out in reqs:
        x = h_in.cuda().reshape(1, -1)
        y = torch.empty((1, h_out.numel()), dtype=torch.complex64, device="cuda")
        (st.tx if d == 0 else st.rx)(x, y)
        assert rel(h_out.numpy(), y.cpu().numpy()[0]) < 1e-6
    st.close()
    plan.close()


def test_admission_refused_above_the_reserve(torch_cuda):
    from paper_2008_00672_gb300 import FcError, Server
    srv = Server(n_lanes=1, hbm_reserve_bytes=1 << 60)
    with pytest.raises(FcError) as e:
        srv.add_carrier(wl.config_mixed_20mhz())
    assert e.value.status == 3          # FC_ERR_NOMEM
    srv.close()


def stream_reference(torch, geom, seq):
    """The carrier's own stream calls on the same inputs, in order."""
    from paper_2008_00672_gb300 import Plan, State
    plan = Plan(geom)
    st = State(plan, 1)
    out = []
    for d, h_in, n_out in seq:
        x = h_in.cuda().reshape(1, -1)
        y = torch.empty((1, n_out), dtype=torch.complex64, device="cuda")
        (st.tx if d == 0 else st.rx)(x, y)
        out.append(y.cpu().numpy()[0])
    st.close()
    plan.close()
    return out


def burst_trace(n_carriers, per_carrier):
    """Every request at t = 0: per carrier, TX and RX slots alternating."""
    return [(0.0, c, k % 2) for k in range(per_carrier) for c in range(n_carriers)]


def check_against_streams(torch, carriers, reqs):
    for c, geom in enumerate(carriers):
        mine = [r for r in reqs if r[1] == c]
        ref = stream_reference(torch, geom, [(d, h_in, h_out.numel()) for _, _, d, h_in, h_out in mine])
        for (_, _, d, _, h_out), want in zip(mine, ref):
            assert rel(h_out.numpy(), want) < 1e-6, (geom.name, d)


def test_burst_runs_as_batches_whose_device_work_overlaps(torch_cuda):
    """Requests of four carriers arriving together are batched: one batch holds requests
    of several carriers, and several slots of one carrier, all in its persistent launch,
    and they share its device interval; every result equals the carrier's own stream
    calls."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Server, fc
    carriers = wl.config_uneven_carriers(seed=1502, n_carriers=4, n_slots=1, whole_cp_period=True)
    sizes = [fc.fc_geometry_check(g) for g in carriers]
    reqs = make_requests(torch, sizes, burst_trace(len(carriers), 6), 3)
    srv = Server(n_lanes=4)
    for g in carriers:
        srv.add_carrier(g)
    rec = srv.serve(reqs)
    srv.close()
    by_batch = {}
    for (t, cid, d, _, _), r in zip(reqs, rec):
        by_batch.setdefault(r.batch, []).append((cid, d, r))
    multi = [b for b in by_batch.values() if len({cid for cid, _, _ in b}) >= 2]
    assert multi, "no batch held requests of two carriers"
    for b in multi:
        assert all(r.batched == 1 for _, _, r in b)
        starts = {round(r.device_start_ms, 6) for _, _, r in b}
        ends = {round(r.device_end_ms, 6) for _, _, r in b}
        assert len(starts) == 1 and len(ends) == 1 and b[0][2].device_end_ms > b[0][2].device_start_ms
    # consecutive slots of one carrier share a batch (their carries chained in the
    # batch's prologue and epilogue); batches are ordered on the device
    assert any(len([(cid, d) for cid, d, _ in b]) > len({(cid, d) for cid, d, _ in b}) for b in by_batch.values())
    ivals = sorted((b[0][2].device_start_ms, b[0][2].device_end_ms) for b in by_batch.values())
    assert all(ivals[i][1] <= ivals[i + 1][0] + 1e-3 for i in range(len(ivals) - 1))
    check_against_streams(torch, carriers, reqs)


def test_small_arena_admits_as_memory_frees(torch_cuda):
    """An arena that holds only a couple of requests at a time: every request is still
    served, in order per carrier, with the same results."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Server, fc
    carriers = wl.config_uneven_carriers(seed=1503, n_carriers=3, n_slots=1, whole_cp_period=True)
    sizes = [fc.fc_geometry_check(g) for g in carriers]
    reqs = make_requests(torch, sizes, burst_trace(len(carriers), 4), 4)
    srv = Server(n_lanes=2)
    for g in carriers:
        srv.add_carrier(g)
    def a256(b):
        return (b + 255) // 256 * 256

    def need(z):          # arena bytes of one request: input, output, workspace, frame
        return a256(8 * z.grid_len) + a256(8 * z.slot_len) + a256(z.workspace_per_stream) + a256(8 * z.wave_len)

    arena = 2 * max(need(z) for z in sizes)
    srv.set_limits(arena, max_batch=8, max_inflight=2)
    rec = srv.serve(reqs)
    srv.close()
    assert all(r.latency_s > 0 for r in rec)
    per_batch = {}
    for (_, cid, _, _, _), r in zip(reqs, rec):
        per_batch[r.batch] = per_batch.get(r.batch, 0) + need(sizes[cid])
    assert max(per_batch.values()) <= arena and len(per_batch) >= len(reqs) // 3
    check_against_streams(torch, carriers, reqs)


def test_continuous_carrier_served_beside_batched_ones(torch_cuda):
    """A continuous-mode carrier (its own stream calls on a lane) next to symbol-sync
    carriers in the persistent launch, in the same batches."""
    torch = torch_cuda
    from paper_2008_00672_gb300 import Server, fc
    carriers = wl.config_uneven_carriers(seed=1504, n_carriers=2, n_slots=1, whole_cp_period=True)
    carriers = list(carriers) + [wl.config_single_5mhz()]
    sizes = [fc.fc_geometry_check(g) for g in carriers]
    reqs = make_requests(torch, sizes, burst_trace(len(carriers), 4), 5)
    srv = Server(n_lanes=4)
    for g in carriers:
        srv.add_carrier(g)
    rec = srv.serve(reqs)
    srv.close()
    flags = {(cid, r.batched) for (_, cid, _, _, _), r in zip(reqs, rec)}
    assert (2, 0) in flags and (0, 1) in flags
    check_against_streams(torch, carriers, reqs)
