"""Time sharding of one carrier across ranks needs one halo step per direction (the
symbols of a symbol-synchronized frame are independent, Sec. III-C): the rank that
holds the earlier slots sends the D samples of its synthesis tail to the next rank,
which adds them to the start of its own output (TX); for RX, every rank but the first
sends the first D received samples of its shard to the rank before it, whose last slot
reads them. This checks the halo arithmetic with world_size-2 gloo ranks on the CPU and
the FP64 oracle (the GPU path runs replicas only): the ranks' concatenated outputs
equal one frame of the whole burst."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K_PER_RANK = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _geometry():
    import workloads as wl
    from oracle import fc_oracle as fo
    g = wl.Group(64, 32, (16, 8, 8, 8, 16, 8))                       # sum of CPs = N: whole phase per slot
    s = wl.Subband(32, 32, 20, 5, 0, wl.rc_transition_weights(32, 20, 3))
    return wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (g,), (s,))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import workloads as wl
    from oracle import fc_oracle as fo
    from tests.test_stream_semantics import k_slots, slot_len, stack_grids
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        geom = _geometry()
        T = slot_len(geom)
        D = fo.frame_len(geom) - T
        K = K_PER_RANK
        grids = [wl.qam_grid(geom, 1, 500 + k)[0] for k in range(world * K)]       # every rank can draw them
        # ---- TX: this rank's shard, then the halo (the D-sample tail) to the next rank ----
        mine = fo.tx_frame(k_slots(geom, K), stack_grids(geom, grids[rank * K:(rank + 1) * K]))
        out = mine[:K * T].copy()
        tail = torch.from_numpy(mine[K * T:].copy())
        if rank + 1 < world:
            dist.send(tail, dst=rank + 1)
        if rank > 0:
            prev = torch.empty_like(tail)
            dist.recv(prev, src=rank - 1)
            out[:D] += prev.numpy()
        # ---- RX: the received burst; rank r holds samples [r K T, (r+1) K T) (the last
        # rank also the final D). Slot k reads [k T, k T + Q), Q = T + D, so a shard's
        # last slot needs the first D samples of the next shard: that is the halo ----
        full = fo.tx_frame(k_slots(geom, world * K), stack_grids(geom, grids))
        x = full + 0.01 * np.random.default_rng(3).standard_normal(len(full))
        own = x[rank * K * T:(rank + 1) * K * T + (D if rank + 1 == world else 0)]
        if rank > 0:
            dist.send(torch.from_numpy(own[:D].copy()), dst=rank - 1)
        if rank + 1 < world:
            ahead = torch.empty(D, dtype=torch.complex128)
            dist.recv(ahead, src=rank + 1)
            own = np.concatenate([own, ahead.numpy()])
        est = fo.rx_frame(k_slots(geom, K), own)
        q.put((rank, out, est))
    finally:
        dist.destroy_process_group()


def test_time_shards_with_halo_equal_one_frame():
    import multiprocessing as mp
    sys.path.insert(0, ROOT)
    import workloads as wl
    from oracle import fc_oracle as fo
    from tests.test_stream_semantics import k_slots, stack_grids
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    geom = _geometry()
    grids = [wl.qam_grid(geom, 1, 500 + k)[0] for k in range(world * K_PER_RANK)]
    big = k_slots(geom, world * K_PER_RANK)
    full = fo.tx_frame(big, stack_grids(geom, grids))
    tx = np.concatenate([r[1] for r in res])
    assert np.max(np.abs(tx - full[:len(tx)])) < 1e-12 * np.max(np.abs(full))
    x = full + 0.01 * np.random.default_rng(3).standard_normal(len(full))
    want = fo.split_grid(big, fo.rx_frame(big, x))[0]
    got = np.concatenate([fo.split_grid(k_slots(geom, K_PER_RANK), r[2])[0] for r in res])
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
