"""The allocation-free TX entry point against the ordinary one.

fc_tx_synthesize_static serves callers that cannot allocate device memory at
run time (its workspace is an array built into the library). This test calls it
through the C ABI twice in a row, with different inputs, and checks each output
against fc_tx_synthesize with a caller-allocated workspace on the same input, and
its first stream against the FP64 oracle. Around the second call it also checks the
property the entry point is named for: the device's free memory and torch's
allocated bytes do not change. It lives in its own file, collected last, and needs
nothing from earlier tests.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests import parity

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_workspace_tx_matches_allocating_tx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import build
    build.build()
    from paper_2008_00672_gb300 import fc

    lib = fc.load_library()
    geom = wl.config_single_5mhz()            # continuous mode: the TX path uses a workspace
    plan = fc.Plan(geom)
    assert plan.workspace_per_stream > 0
    n = 6
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((2100, 2200)):
        grid = torch.from_numpy(wl.qam_grid(geom, n, seed).astype(np.complex64)).cuda()
        ref = torch.empty((n, plan.wave_len), dtype=torch.complex64, device="cuda")
        plan.tx_synthesize(grid, ref)
        out = torch.full((n, plan.wave_len), float("nan"), dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        st = lib.fc_tx_synthesize_static(plan.handle, n, ctypes.c_void_p(grid.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == fc.FC_OK, lib.fc_last_error().decode()
        torch.cuda.synchronize()
        if call == 1:       # the first call may load kernel code; the second allocates nothing at all
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == used0
        err = rel(out.cpu().numpy(), ref.cpu().numpy())
        assert err <= TOL, (call, err)
        parity.check(out[0].cpu().numpy(), fo.tx_frame(geom, grid[0].cpu().numpy().astype(np.complex128)), TOL,
                     parity.wave_windows(geom), call)

    # more streams than the built-in workspace holds: a clear error, nothing launched
    too_many = (1 << 25) // plan.workspace_per_stream + 1
    st = lib.fc_tx_synthesize_static(plan.handle, too_many, ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 20),
                                     ctypes.c_void_p(stream))
    assert st == fc.FC_ERR_INVALID
    assert b"static workspace too small" in lib.fc_last_error()
    plan.close()


def test_static_tx_symbol_sync_needs_no_workspace():
    """The 20 MHz symbol-sync plan (one-warp kernels: the initialising launch, then its
    dependent launches) through the allocation-free entry point: no workspace, nothing
    allocated, the allocating call's result."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import fc

    lib = fc.load_library()
    geom = wl.config_mixed_20mhz()
    plan = fc.Plan(geom)
    assert plan.workspace_per_stream == 0 and plan.tx_kernels == 3
    n = 5
    stream = torch.cuda.current_stream().cuda_stream
    grid = torch.from_numpy(wl.qam_grid(geom, n, 2300).astype(np.complex64)).cuda()
    ref = torch.empty((n, plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(grid, ref)
    out = torch.full((n, plan.wave_len), float("nan"), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    st = lib.fc_tx_synthesize_static(plan.handle, n, ctypes.c_void_p(grid.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert st == fc.FC_OK, lib.fc_last_error().decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == used0
    # every sample written (the NaN fill is gone); equal up to the order of the reductions
    assert not torch.isnan(torch.view_as_real(out)).any()
    assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    parity.check(out[n - 1].cpu().numpy(), fo.tx_frame(geom, grid[n - 1].cpu().numpy().astype(np.complex128)), TOL,
                 parity.wave_windows(geom))
    plan.close()
