"""Fixed invocations of the library's kernels for profilers.

    python -m paper_2008_00672_gb300.profile_cases CASE --streams S [--warm W]
        [--tx-chunks K --rx-chunks K] [--time R]

builds the case's plan, sets a fixed launch shape (the case's default, or the chunks
per stream given, e.g. the ones the benchmark's autotuner reports), runs W warm-up
TX + RX passes and then one more TX + RX pass, so that `ncu -k <kernel> -s <skip>`
can pick launches of a known shape. Inputs are seeded QAM grids; the RX input is the
TX output (its values do not change the kernels' work). With --time R it then times R
more TX calls and R more RX calls with CUDA events on the current stream and prints
the mean milliseconds of each (for comparing two builds of a kernel; not for ncu runs).

Cases:
  warp20     20 MHz mixed numerology, symbol-synchronized (one-warp-per-symbol kernels,
             which deal all streams' jobs to the resident CTAs whatever the chunk count)
  generic20  the same geometry on the generic shared-memory kernels
  tensor100  100 MHz / 273 PRB carrier, 10 slots, on the tensor-core passes
  fp32_100   the same carrier on the FP32 shared-memory kernels
"""
import argparse
import dataclasses

import numpy as np

import workloads as wl

from . import FC_FLAG_GENERIC_KERNELS, FC_FLAG_TENSOR_DFT, FC_RX, FC_TX, Plan, build


def make_case(name: str):
    if name == "warp20":
        return wl.config_mixed_20mhz(), {FC_TX: (1, 0), FC_RX: (2, 0)}
    if name == "generic20":
        return dataclasses.replace(wl.config_mixed_20mhz(), flags=FC_FLAG_GENERIC_KERNELS), {}
    if name == "tensor100":
        return dataclasses.replace(wl.config_100mhz(10), flags=FC_FLAG_TENSOR_DFT), {}
    if name == "fp32_100":
        return wl.config_100mhz(10), {}
    raise SystemExit(f"unknown case {name}")


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["warp20", "generic20", "tensor100", "fp32_100"])
    ap.add_argument("--streams", type=int, default=256)
    ap.add_argument("--warm", type=int, default=1)
    ap.add_argument("--tx-chunks", type=int, default=0, help="chunks per stream of the TX launch (0: the case's)")
    ap.add_argument("--rx-chunks", type=int, default=0, help="chunks per stream of the RX launch (0: the case's)")
    ap.add_argument("--time", type=int, default=0, help="then time this many TX and RX calls (CUDA events)")
    args = ap.parse_args()
    build.build()
    geom, shape = make_case(args.case)
    for d, k in ((FC_TX, args.tx_chunks), (FC_RX, args.rx_chunks)):
        if k:
            shape[d] = (k, 0)
    plan = Plan(geom)
    S = args.streams
    for d, (k, g) in shape.items():
        plan.set_choice(S, d, k, g)
    base = wl.qam_grid(geom, min(S, 64), wl.default_seed(2)).astype(np.complex64)
    grid = torch.from_numpy(base).cuda().repeat(-(-S // base.shape[0]), 1)[:S].contiguous()
    wave = torch.empty((S, plan.wave_len), dtype=torch.complex64, device="cuda")
    est = torch.empty_like(grid)
    for _ in range(args.warm + 1):
        plan.tx_synthesize(grid, wave)
        plan.rx_analyze(wave, est)
    torch.cuda.synchronize()
    timed = ""
    if args.time > 0:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        for _ in range(args.time):
            plan.tx_synthesize(grid, wave)
        ev[1].record()
        for _ in range(args.time):
            plan.rx_analyze(wave, est)
        ev[2].record()
        torch.cuda.synchronize()
        timed = (f"; mean of {args.time}: TX {ev[0].elapsed_time(ev[1]) / args.time:.4f} ms, "
                 f"RX {ev[1].elapsed_time(ev[2]) / args.time:.4f} ms")
    plan.close()
    print(f"{args.case}: {S} streams, {args.warm} warm-up passes + 1, launches per pass "
          f"TX {plan.tx_kernels} RX {plan.rx_kernels}{timed}")


if __name__ == "__main__":
    main()
