"""GPU: host-buffer execute calls (fc_pipeline): chunked, overlapped copies and
kernels give the same results as the device calls, for chunk counts that do not
divide the streams, for symbol-sync (warp kernels), continuous (workspace) and the
tensor-core path."""
import dataclasses

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


@pytest.mark.parametrize("name,chunk,depth", [("mixed20", 3, 2), ("single5", 4, 3), ("nr100t", 2, 3)])
def test_host_pipeline_equals_device_calls(torch_cuda, name, chunk, depth):
    torch = torch_cuda
    from paper_2008_00672_gb300 import FC_FLAG_TENSOR_DFT, Pipeline, Plan
    geom = dataclasses.replace(wl.config_100mhz(1), flags=FC_FLAG_TENSOR_DFT) if name == "nr100t" \
        else wl.NAMED[name]()
    S = 7
    plan = Plan(geom)
    grid = torch.from_numpy(wl.qam_grid(geom, S, 21).astype(np.complex64))
    h_grid = grid.pin_memory()
    h_wave = torch.zeros((S, plan.wave_len), dtype=torch.complex64).pin_memory()
    h_est = torch.zeros((S, plan.grid_len), dtype=torch.complex64).pin_memory()
    pipe = Pipeline(plan, chunk, depth)
    pipe.tx(h_grid, h_wave)
    pipe.rx(h_wave, h_est)
    torch.cuda.synchronize()
    d_wave = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    d_est = torch.empty((S, plan.grid_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(grid.cuda(), d_wave)
    plan.rx_analyze(h_wave.cuda(), d_est)
    torch.cuda.synchronize()
    assert rel(h_wave.numpy(), d_wave.cpu().numpy()) < 1e-6
    assert rel(h_est.numpy(), d_est.cpu().numpy()) < 1e-6
    pipe.close()
    plan.close()
