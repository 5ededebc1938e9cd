"""Stream = frame: the semantics behind fc_state, pinned on the FP64 oracle alone.

A stream is a sequence of slots with the same geometry. The frame of K slots is the
frame of the geometry whose CP list is the slot's repeated K times (every group),
with the K slot grids stacked per subband. The library's stream calls rely on two
identities of that K-slot frame, which hold when the geometry is shift-invariant by
one slot (same slot duration T in every group; c_m T / N_m an integer, so theta_n and
phi_r repeat; continuous mode also needs whole hops per slot and S_L >= L_O):

  TX: frame_K = sum_k (frame_1 of slot k) delayed by k T          (all Q_K samples)
  RX: slot k of rx_frame_K(x) = rx_frame_1(x[k T : k T + Q_1])

So one stream call can run the one-slot frame, emit its first T samples plus the
carried tail, and carry the last D = Q_1 - T samples (TX); or run the one-slot
frame on D look-behind samples followed by the call's T new samples (RX). These
tests check both identities exactly, and that they fail when c_m T / N is not an
integer (the case the library refuses).
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo


def crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def k_slots(geom, K):
    groups = tuple(dataclasses.replace(g, n_cp=tuple(g.n_cp) * K) for g in geom.groups)
    return dataclasses.replace(geom, groups=groups)


def slot_len(geom):
    """T of the slot (high-rate samples); the same in every group or the geometry
    does not stream."""
    ts = set()
    for s in geom.subbands:
        g = geom.groups[s.group]
        n_ofdm = g.n_long if geom.mode == fo.SYMBOL_SYNC else s.l_ofdm * g.n_long // s.l_short
        ts.add(sum(g.n_cp) + len(g.n_cp) * n_ofdm)
    assert len(ts) == 1
    return ts.pop()


def stack_grids(geom, grids):
    """K per-slot grids (ABI layout) -> the K-slot frame's grid."""
    parts = [fo.split_grid(geom, g) for g in grids]
    return np.concatenate([np.concatenate([p[m] for p in parts]).reshape(-1)
                           for m in range(len(geom.subbands))])


def tx_identity_error(geom, K, seed):
    rng = np.random.default_rng(seed)
    T = slot_len(geom)
    q1 = fo.frame_len(geom)
    grids = [crand(rng, geom.grid_len()) for _ in range(K)]
    big = fo.tx_frame(k_slots(geom, K), stack_grids(geom, grids))
    assert len(big) == (K - 1) * T + q1
    acc = np.zeros(len(big), dtype=np.complex128)
    for k, g in enumerate(grids):
        acc[k * T:k * T + q1] += fo.tx_frame(geom, g)
    return float(np.max(np.abs(acc - big)) / np.max(np.abs(big)))


def rx_identity_error(geom, K, seed):
    rng = np.random.default_rng(seed)
    T = slot_len(geom)
    q1 = fo.frame_len(geom)
    x = crand(rng, (K - 1) * T + q1)
    big = fo.rx_frame(k_slots(geom, K), x)
    per = [fo.split_grid(geom, fo.rx_frame(geom, x[k * T:k * T + q1])) for k in range(K)]
    # the K-slot grid holds, per subband, K slots of rows
    bparts = fo.split_grid(k_slots(geom, K), big)
    err = 0.0
    for m in range(len(geom.subbands)):
        want = np.concatenate([p[m] for p in per])
        err = max(err, float(np.max(np.abs(bparts[m] - want)) / np.max(np.abs(want))))
    return err


def small_sync(c, n_cp, stx=fo.OLA, srx=fo.OLS):
    D = wl.rc_transition_weights(32, 20, 3)
    g = wl.Group(64, 32, tuple(n_cp))
    s = wl.Subband(32, 32, 20, c, 0, D)
    return wl.Geometry(fo.SYMBOL_SYNC, stx, srx, (g,), (s,))


def small_cont(c, n_cp, stx, srx, L=32, N=64):
    D = wl.rc_transition_weights(L, 20, 3)
    g = wl.Group(N, N // 2, tuple(n_cp))
    s = wl.Subband(L, L, 20, c, 0, D)
    return wl.Geometry(fo.CONTINUOUS, stx, srx, (g,), (s,))


def two_group_sync():
    ga = wl.Group(64, 32, (16, 16, 16, 16))          # T = 4 * (64 + 16) = 320
    gb = wl.Group(32, 16, (8,) * 8)                   # T = 8 * (32 + 8) = 320
    sa = wl.Subband(32, 32, 20, 6, 0, wl.rc_transition_weights(32, 20, 3))
    sb = wl.Subband(16, 16, 10, -4, 1, wl.rc_transition_weights(16, 10, 2))
    return wl.Geometry(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, (ga, gb), (sa, sb))


# every case has sum(N_CP) a multiple of N, so c_m T / N is an integer
STREAMABLE = [
    ("sync-OLA-OLS", small_sync(5, (16, 8, 8, 8, 16, 8))),
    ("sync-OLS-OLA", small_sync(-3, (16, 16, 16, 16), fo.OLS, fo.OLA)),
    ("continuous-OLA-OLA", small_cont(5, (8,) * 8, fo.OLA, fo.OLA)),
    ("continuous-OLS-OLS", small_cont(-7, (16, 16, 16, 16), fo.OLS, fo.OLS)),
    ("sync-two-groups", two_group_sync()),
]


def whole_phase(geom):
    T = slot_len(geom)
    return all((s.centre_bin * T) % geom.groups[s.group].n_long == 0 for s in geom.subbands)


@pytest.mark.parametrize("name,geom", STREAMABLE, ids=[n for n, _ in STREAMABLE])
def test_stream_identities_hold(name, geom):
    """Catches a stream design that drops the carried tail / look-behind, or a slot
    period that does not repeat the block grid and the phases."""
    assert whole_phase(geom), name
    assert tx_identity_error(geom, 3, 11) < 1e-12
    assert rx_identity_error(geom, 3, 12) < 1e-12


def test_stream_identities_nr_5mhz_continuous():
    """The 5 MHz continuous OLS workload (N = 512, L = 384, I = 4/3) streams per slot."""
    geom = wl.config_single_5mhz()
    assert slot_len(geom) == 7680 and whole_phase(geom)
    assert tx_identity_error(geom, 2, 13) < 1e-11
    assert rx_identity_error(geom, 2, 14) < 1e-11


def test_stream_identities_fail_without_whole_phase():
    """c_m T / N not an integer: theta_n does not repeat, so slot k of the long frame
    is slot 0's output times a phase that differs per subband; the library refuses
    this geometry for stream calls."""
    geom = small_sync(5, (16, 8, 8, 9))
    assert not whole_phase(geom)
    assert tx_identity_error(geom, 2, 15) > 1e-3
