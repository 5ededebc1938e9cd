"""GPU parity on seeded random geometries: both modes, OLA/OLS on each side, short
transforms of 2^a 3^b points, interpolation ratios I in {1, 4/3, 3/2, 2, 3, 4}, one to
three numerology groups, one to three subbands per group, random CP lists, centre bins
and transition bands, and the kernel-selection flags. Every drawn geometry that the
planner accepts is compared with the FP64 oracle on two streams: RMS <= 1e-5 per stream,
per symbol window and per grid row, and 5e-5 of the signal RMS per sample
(`tests/parity.py`)."""
import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo
from tests import parity

pytestmark = pytest.mark.gpu
TOL = 1e-5
N_CASES = 24


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2008_00672_gb300 import build
    build.build()
    return torch


def draw_geometry(rng):
    mode = fo.SYMBOL_SYNC if rng.random() < 0.5 else fo.CONTINUOUS
    stx, srx = (fo.OLA, fo.OLS)[rng.integers(2)], (fo.OLA, fo.OLS)[rng.integers(2)]
    n_groups = int(rng.integers(1, 4))
    groups, subs = [], []
    n_sym = int(rng.integers(1, 5))
    for gi in range(n_groups):
        L = int(rng.choice([24, 32, 48, 64, 96, 128]))
        ratio = [(1, 1), (4, 3), (3, 2), (2, 1), (3, 1), (4, 1)][rng.integers(6)]
        if (L * ratio[0]) % ratio[1]:
            ratio = (2, 1)
        N = L * ratio[0] // ratio[1]
        if N > 512 or N % 4:
            N = 2 * L
        cps = []
        for _ in range(n_sym * (gi + 1)):
            if mode == fo.SYMBOL_SYNC:
                cps.append(int(rng.integers(0, N // 4 + 1)))
            else:                                    # continuous: N_CP L / N must be an integer
                step = N // np.gcd(N, L)
                cps.append(int(step * rng.integers(0, max(1, N // 8 // step) + 1)))
        groups.append(wl.Group(N, N // 2, tuple(cps)))
        for _ in range(int(rng.integers(1, 4)) if gi == 0 else 1):
            n_tb = int(rng.integers(0, 4))
            act = int(rng.integers(4, max(5, L - 2 * n_tb - 2)))
            c = int(rng.integers(-N // 2, N // 2))
            subs.append(wl.Subband(L, L, act, c, gi, wl.rc_transition_weights(L, act, n_tb)))
    flags = int(rng.choice([0, 1]))
    return wl.Geometry(mode, stx, srx, tuple(groups), tuple(subs), flags=flags)


def cases():
    rng = np.random.default_rng(20260301)
    out = []
    from paper_2008_00672_gb300 import fc
    fc.load_library()
    while len(out) < N_CASES:
        g = draw_geometry(rng)
        try:
            fc.fc_geometry_check(g)
            fo.frame_len(g)
        except Exception:
            continue                                   # geometry the paper's equations do not define
        out.append(g)
    return out


@pytest.fixture(scope="module")
def geometries(torch_cuda):
    return cases()


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_geometry(torch_cuda, geometries, k):
    torch = torch_cuda
    from paper_2008_00672_gb300 import Plan
    geom = geometries[k]
    S = 2
    grid = wl.qam_grid(geom, S, 900 + k).astype(np.complex64)
    plan = Plan(geom)
    w = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    plan.tx_synthesize(torch.from_numpy(grid).cuda(), w)
    x = np.stack([wl.awgn(fo.tx_frame(geom, grid[s].astype(np.complex128)), 30.0, 7 + s) for s in range(S)])
    x = x.astype(np.complex64)
    est = torch.empty((S, plan.grid_len), dtype=torch.complex64, device="cuda")
    plan.rx_analyze(torch.from_numpy(x).cuda(), est)
    torch.cuda.synchronize()
    w, est = w.cpu().numpy(), est.cpu().numpy()
    plan.close()
    ww, gw = parity.wave_windows(geom), parity.grid_windows(geom)
    for s in range(S):
        parity.check(w[s], fo.tx_frame(geom, grid[s].astype(np.complex128)), TOL, ww, (geom, "tx", s))
        parity.check(est[s], fo.rx_frame(geom, x[s].astype(np.complex128)), TOL, gw, (geom, "rx", s))
