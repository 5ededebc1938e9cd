"""GPU: the serving loop. A carrier's results do not depend on what else is served
(alone vs mixed), they equal the carrier's own stream calls, and admission refuses a
carrier that does not fit above the HBM reserve."""
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
