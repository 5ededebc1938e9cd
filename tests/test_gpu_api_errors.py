"""GPU: the argument checks of the stream, pipeline, batch, server and autotuner calls
(each documented error returns FC_ERR_INVALID / FC_ERR_UNSUPPORTED and leaves the plan
usable), and their zero-stream no-ops."""
import ctypes

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


def status_of(fn, *args):
    from paper_2008_00672_gb300 import fc
    try:
        fn(*args)
    except fc.FcError as e:
        return e.status
    return fc.FC_OK


def test_pipeline_argument_checks(torch_cuda):
    from paper_2008_00672_gb300 import fc
    plan = fc.Plan(wl.config_mixed_20mhz())
    assert status_of(fc.fc_pipeline_create, plan.handle, 0, 2) == fc.FC_ERR_INVALID
    assert status_of(fc.fc_pipeline_create, plan.handle, 4, 0) == fc.FC_ERR_INVALID
    assert status_of(fc.fc_pipeline_create, plan.handle, 4, 17) == fc.FC_ERR_INVALID
    pipe = fc.fc_pipeline_create(plan.handle, 4, 2)
    fc.fc_tx_synthesize_host(pipe, 0, None, None)                       # zero streams: no-op
    assert status_of(fc.fc_tx_synthesize_host, pipe, 1, None, None) == fc.FC_ERR_INVALID
    assert status_of(fc.fc_rx_analyze_host, pipe, -1, None, None) == fc.FC_ERR_INVALID
    fc.fc_pipeline_destroy(pipe)
    plan.close()


def test_batch_argument_checks(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import fc
    plan = fc.Plan(wl.config_mixed_20mhz())
    g = torch.zeros((1, plan.grid_len), dtype=torch.complex64, device="cuda")
    w = torch.zeros((1, plan.wave_len), dtype=torch.complex64, device="cuda")
    item = fc.FcBatchItem(plan.handle.value, None, fc.FC_TX, 1, g.data_ptr(), w.data_ptr(), None, 0)
    assert status_of(fc.fc_batch_create, [], 4, True) == fc.FC_ERR_INVALID
    assert status_of(fc.fc_batch_create, [item], 0, True) == fc.FC_ERR_INVALID
    bad = fc.FcBatchItem(plan.handle.value, None, 7, 1, g.data_ptr(), w.data_ptr(), None, 0)
    assert status_of(fc.fc_batch_create, [bad], 2, True) == fc.FC_ERR_INVALID
    plan.close()


def test_state_and_choice_checks(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import fc
    a = fc.Plan(wl.config_mixed_20mhz())
    b = fc.Plan(wl.config_single_5mhz())
    st = fc.State(a, 1)
    g = torch.zeros((1, b.grid_len), dtype=torch.complex64, device="cuda")
    o = torch.zeros((1, b.slot_len), dtype=torch.complex64, device="cuda")
    # a state works only with plans of its frame sizes
    assert status_of(fc.fc_tx_synthesize_stream, b.handle, st.handle, g.data_ptr(), o.data_ptr()) \
        == fc.FC_ERR_INVALID
    assert status_of(fc.fc_state_create, a.handle, -1) == fc.FC_ERR_INVALID
    assert status_of(fc.fc_plan_set_choice, a.handle, 8, 5, 1, 0) == fc.FC_ERR_INVALID      # direction
    assert status_of(fc.fc_plan_set_choice, a.handle, 8, fc.FC_TX, 1, 2) == fc.FC_ERR_INVALID
    assert status_of(fc.fc_plan_autotune, a.handle, 0) == fc.FC_ERR_INVALID
    assert fc.load_library().fc_plan_device_status(a.handle) == fc.FC_OK
    st.close()
    a.close()
    b.close()


def test_server_argument_checks(torch_cuda):
    torch = torch_cuda
    from paper_2008_00672_gb300 import fc
    srv = fc.Server(n_lanes=1)
    cid = srv.add_carrier(wl.config_single_5mhz())
    z = srv.sizes[cid]
    h_in = torch.zeros(z.grid_len, dtype=torch.complex64).pin_memory()
    h_out = torch.zeros(z.slot_len, dtype=torch.complex64).pin_memory()
    unsorted = [fc.FcServeRequest(1e-3, cid, fc.FC_TX, h_in.data_ptr(), h_out.data_ptr()),
                fc.FcServeRequest(0.0, cid, fc.FC_TX, h_in.data_ptr(), h_out.data_ptr())]
    assert status_of(fc.fc_server_run, srv.handle, unsorted) == fc.FC_ERR_INVALID
    wrong = [fc.FcServeRequest(0.0, cid + 5, fc.FC_TX, h_in.data_ptr(), h_out.data_ptr())]
    assert status_of(fc.fc_server_run, srv.handle, wrong) == fc.FC_ERR_INVALID
    assert fc.fc_server_run(srv.handle, []) == []                       # no requests: returns at once
    srv.close()
    assert status_of(fc.fc_server_create, 0, 0, 0) == fc.FC_ERR_INVALID
