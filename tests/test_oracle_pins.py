"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the mistake it is there to catch. None of them re-types an oracle
formula: they compare against printed numbers, closed forms, brute force,
exact operator identities or invariants.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle import fc_oracle as fo

GOLD = os.path.join(os.path.dirname(__file__), "golden", "plan_numbers.json")


def gold():
    with open(GOLD) as f:
        return json.load(f)


def crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def geom1(mode, stx, srx, N, N_O, L, L_ofdm, L_act, c, n_cp, D, lead_pad=-1):
    g = wl.Group(n_long=N, n_overlap=N_O, n_cp=tuple(n_cp), lead_pad=lead_pad)
    s = wl.Subband(l_short=L, l_ofdm=L_ofdm, n_active=L_act, centre_bin=c, group=0, weights=np.asarray(D, float))
    return wl.Geometry(mode, stx, srx, (g,), (s,))


# ---------------------------------------------------------------------------
# printed plan numbers
# ---------------------------------------------------------------------------

def test_cp_lengths_printed_sec3e():
    """Sec. III-E: L_CP,n = floor(N_CP,n/I). Catches a wrong I (N/L vs L/N) or rounding."""
    gd = gold()["cp_extrapolation_10mhz"]
    N = gd["n_long"]
    for L, fr1, fr2 in zip(gd["discontinuous_l_ofdm"], gd["fractional_l_cp_first"], gd["fractional_l_cp_other"]):
        g = wl.Group(N, N // 2, (gd["n_cp_first"], gd["n_cp_other"]))
        s = wl.Subband(L, L, 12, 0, 0, np.ones(L))
        d = fo.Dims(g, s)
        assert d.I == N / L
        assert gd["n_cp_first"] / d.I == pytest.approx(fr1)
        assert gd["n_cp_other"] / d.I == pytest.approx(fr2)
        assert fo.low_rate_cp(d, fo.SYMBOL_SYNC) == [math.floor(fr1), math.floor(fr2)]
        with pytest.raises(ValueError):       # continuous FC cannot use fractional CPs
            fo.low_rate_cp(d, fo.CONTINUOUS)
    L = gd["continuous_l_ofdm"]
    d = fo.Dims(wl.Group(N, N // 2, (gd["n_cp_first"], gd["n_cp_other"])), wl.Subband(L, L, 12, 0, 0, np.ones(L)))
    assert fo.low_rate_cp(d, fo.CONTINUOUS) == gd["continuous_l_cp"]


def test_fig_extrapol_numbers():
    gd = gold()["fig_extrapol"]
    L = gd["n_ofdm"] // gd["I"]
    d = fo.Dims(wl.Group(gd["n_ofdm"], gd["n_ofdm"] // 2, (gd["n_cp"],)), wl.Subband(L, L, 8, 0, 0, np.ones(L)))
    assert d.L == 16
    assert fo.low_rate_cp(d, fo.SYMBOL_SYNC) == [gd["l_cp"]]


def test_nr_cp_schedule_matches_paper():
    """The workload generator's NR CP schedule reproduces the paper's 80/72 pattern."""
    gd = gold()["nr_cp_schedule_10mhz"]
    assert list(wl.nr_normal_cp(gd["n_fft"], gd["scs_khz"], 14)) == gd["n_cp_14"]
    # one ms of samples at each rate: 15.36 Msps -> 15360
    assert sum(gd["n_cp_14"]) + 14 * gd["n_fft"] == 15360


def test_block_counts_two_symbols():
    """Fig. BlockProc: five continuous blocks for two symbols (lambda=0.5, no CP,
    S_L = L_O); symbol-synchronized processing uses two blocks per symbol."""
    gd = gold()["blocks_two_symbols"]
    L = N = 16
    d = fo.Dims(wl.Group(N, N // 2, (0, 0)), wl.Subband(L, L, 8, 0, 0, np.ones(L)))
    assert fo.continuous_block_count(2 * L, d.L_O, d) == gd["continuous"]
    assert 2 * 2 == gd["symbol_sync"]


# ---------------------------------------------------------------------------
# DFT closed forms and unitary OFDM
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 12, 16, 48])
def test_dft_closed_forms(n):
    """DFT(delta) = 1, DFT(exp(+j2pi k0 t/n)) = n delta_k0, IDFT inverts.
    Catches a sign or normalisation error in W_n."""
    d = np.zeros(n, complex)
    d[0] = 1
    assert np.allclose(fo.dft(d), np.ones(n), atol=1e-13)
    for k0 in range(n):
        t = np.arange(n)
        tone = np.exp(2j * np.pi * k0 * t / n)
        e = np.zeros(n, complex)
        e[k0] = n
        assert np.allclose(fo.dft(tone), e, atol=1e-10)
    x = crand(np.random.default_rng(n), n)
    assert np.allclose(fo.idft(fo.dft(x)), x, atol=1e-12)


def test_ofdm_mod_demod_unitary_parseval():
    rng = np.random.default_rng(3)
    for n, act in [(16, 12), (64, 44), (384, 288)]:
        x = crand(rng, act)
        t = fo.ofdm_modulate(x, n)
        assert np.sum(np.abs(t) ** 2) == pytest.approx(np.sum(np.abs(x) ** 2), rel=1e-12)
        assert np.allclose(fo.ofdm_demodulate(t, act), x, atol=1e-12)
    # a single active subcarrier at signed frequency f is a tone exp(+j 2 pi f t / n)/sqrt(n)
    n, act = 16, 5
    for i in range(act):
        x = np.zeros(act, complex)
        x[i] = 1
        f = i - act // 2
        assert np.allclose(fo.ofdm_modulate(x, n), np.exp(2j * np.pi * f * np.arange(n) / n) / math.sqrt(n))


def test_cp_insert():
    x = np.arange(8) + 0j
    assert np.array_equal(fo.cp_insert(x, 3), np.r_[5, 6, 7, np.arange(8)])


# ---------------------------------------------------------------------------
# Continuous FC: delayed identity, linear convolution, carrier, adjoint
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("L,N_O,c", [(16, 8, 0), (16, 8, 3), (24, 6, -5), (20, 10, 7)])
def test_continuous_identity_and_carrier(scheme, L, N_O, c):
    """I = 1, D = 1: output = padded input times exp(j2pi c t/N) (global time).
    Catches wrong phi_r, wrong block hop, window misplacement, OLS keep range."""
    N = L
    g = wl.Group(N, N_O, (0,))
    sb = wl.Subband(L, L, L, c, 0, np.ones(L))
    rng = np.random.default_rng(L + N_O)
    s = crand(rng, 5 * L + 3)
    out = fo.tx_continuous_subband(s, g, sb, scheme)
    d = fo.Dims(g, sb)
    u = np.zeros(len(out), complex)
    u[d.L_O:d.L_O + len(s)] = s
    t = np.arange(len(out))
    assert np.allclose(out, u * np.exp(2j * np.pi * c * t / N), atol=1e-12)


def _fir_weights(h, L):
    """Real zero-phase FIR h[-K..K] -> its L-point DFT in fftshifted order (real)."""
    K = (len(h) - 1) // 2
    hc = np.zeros(L)
    for i, v in enumerate(h):
        hc[(i - K) % L] = v
    H = np.fft.fft(hc)
    assert np.allclose(H.imag, 0, atol=1e-12)
    return H.real[(np.arange(L) - L // 2) % L]


@pytest.mark.parametrize("scheme", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("c", [0, 2])
def test_continuous_equals_linear_convolution(scheme, c):
    """I = 1, D = DFT of a zero-phase FIR with K <= min(L_L, L_T): FC = brute-force
    linear convolution (FC approximates linear convolution, Sec. II). Catches a wrong
    shift P, wrong bin map Xi, wrong D ordering, OLA/OLS windowing errors."""
    L = N = 32
    N_O = 16
    h = np.array([0.05, -0.1, 0.2, 0.7, 0.2, -0.1, 0.05, ])   # K = 3
    K = 3
    D = _fir_weights(h, L)
    g = wl.Group(N, N_O, (0,))
    sb = wl.Subband(L, L, L, c, 0, D)
    rng = np.random.default_rng(7)
    s = crand(rng, 150)
    out = fo.tx_continuous_subband(s, g, sb, scheme)
    u = np.zeros(len(out), complex)
    u[N_O:N_O + len(s)] = s
    # brute force: y[t] = sum_k h[k] u[t-k], then the carrier of the long bin c
    ref = np.zeros(len(out), complex)
    for t in range(len(out)):
        acc = 0
        for k in range(-K, K + 1):
            if 0 <= t - k < len(u):
                acc += h[k + K] * u[t - k]
        ref[t] = acc * np.exp(2j * np.pi * c * t / N)
    d = fo.Dims(g, sb)
    if scheme == fo.OLS:    # OLS output starts at N_L of block 0 and ends at N_L of the last hop
        lo, hi = d.N_L, (fo.continuous_block_count(len(s), d.L_O, d)) * d.N_S + d.N_L
        assert np.allclose(out[lo:hi], ref[lo:hi], atol=1e-12)
        assert np.allclose(out[:lo], 0) and np.allclose(out[hi:], 0)
    else:
        assert np.allclose(out, ref, atol=1e-12)


def _adjoint_case(N, N_O, L, c, seed):
    rng = np.random.default_rng(seed)
    D = rng.uniform(-1, 1, L)
    g = wl.Group(N, N_O, (0,))
    sb = wl.Subband(L, L, L, c, 0, D)
    return g, sb, rng


@pytest.mark.parametrize("N,N_O,L,c", [(64, 32, 48, 5), (64, 32, 32, -7), (64, 16, 32, 30),
                                       (48, 24, 36, 47), (40, 20, 40, 3)])
def test_continuous_adjoint_pairs(N, N_O, L, c):
    """RX_OLS = (TX_OLA)^H and RX_OLA = (TX_OLS)^H exactly (eq:ola_analysis,
    eq:ols_analysis with conj phase and 1/sqrt(I), readings R3/R4). Catches a
    missing conj, a wrong sqrt(I), mismatched windows, gather/scatter mismatch."""
    g, sb, rng = _adjoint_case(N, N_O, L, c, N + L + c)
    d = fo.Dims(g, sb)
    n_low = 4 * L + 5
    s = crand(rng, n_low)
    for stx, srx in [(fo.OLA, fo.OLS), (fo.OLS, fo.OLA)]:
        y_tx = fo.tx_continuous_subband(s, g, sb, stx)
        y = crand(rng, len(y_tx))
        s_rx = fo.rx_continuous_subband(y, g, sb, srx, n_low)
        lhs = np.vdot(y, y_tx)            # <TX s, y>
        rhs = np.vdot(s_rx, s)            # <s, RX y>
        assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1)


def test_block_operator_adjoint_matrix():
    """Per block: the analysis matrix is the conjugate transpose of the synthesis
    matrix (eq:ola_analysis '= conj(F)^T' with the R4 reading)."""
    g, sb, rng = _adjoint_case(32, 16, 24, 9, 1)
    d = fo.Dims(g, sb)
    ph = np.array([np.exp(2j * np.pi * 0.3)])
    F = np.stack([fo.synthesis_blocks(np.eye(d.L)[:, [j]], d, ph)[:, 0] for j in range(d.L)], axis=1)
    G = np.stack([fo.analysis_blocks(np.eye(d.N)[:, [j]], d, ph)[:, 0] for j in range(d.N)], axis=1)
    assert np.allclose(G, F.conj().T, atol=1e-13)


def test_block_matches_printed_matrices():
    """Transcription check: synthesis_blocks equals the product of the matrices as
    printed in Sec. III-B (1-based Xi, P as the printed block matrix), even L."""
    N, L, c = 32, 12, -4
    rng = np.random.default_rng(5)
    D = rng.uniform(0, 1, L)
    g = wl.Group(N, N // 2, (0,))
    sb = wl.Subband(L, L, L, c, 0, D)
    d = fo.Dims(g, sb)
    phi = np.exp(2j * np.pi * 0.17)
    WL = np.array([[np.exp(-2j * np.pi * k * t / L) for t in range(L)] for k in range(L)])
    WNi = np.array([[np.exp(2j * np.pi * k * t / N) / N for t in range(N)] for k in range(N)])
    fl, ce = L // 2, -(-L // 2)
    P = np.block([[np.zeros((fl, ce)), np.eye(fl)], [np.eye(ce), np.zeros((ce, fl))]])
    M = np.zeros((N, L), complex)
    for p1 in range(1, L + 1):                      # 1-based p, 1-based q
        q1 = ((c - ce + p1 - 1) % N) + 1
        M[q1 - 1, p1 - 1] = phi
    F = math.sqrt(N / L) * WNi @ M @ np.diag(D) @ P @ WL
    Fo = fo.synthesis_blocks(np.eye(L), d, np.full(L, phi))
    assert np.allclose(Fo, F, atol=1e-13)


# ---------------------------------------------------------------------------
# Symbol-synchronized processing
# ---------------------------------------------------------------------------

def sync_geom(N=32, L=16, c=3, n_cp=(6, 4, 4, 5), stx=fo.OLA, srx=fo.OLS, L_act=10, D=None):
    D = np.ones(L) if D is None else D
    return geom1(fo.SYMBOL_SYNC, stx, srx, N, N // 2, L, L, L_act, c, n_cp, D)


@pytest.mark.parametrize("stx", [fo.OLA, fo.OLS])
def test_sync_symbol_locality(stx):
    """Changing symbol n alters the TX output only inside [sigma_n, sigma_n + 3N/2)
    (symbols are processed independently, Sec. III)."""
    rng = np.random.default_rng(11)
    D = wl.rc_transition_weights(16, 10, 2)
    gm = sync_geom(stx=stx, D=D)
    grid = crand(rng, gm.grid_len())
    base = fo.tx_frame(gm, grid)
    d = fo.Dims(gm.groups[0], gm.subbands[0])
    sig = fo.sync_sigma(d)
    off = fo.frame_layout(gm)[0][0]
    for n in range(d.B):
        g2 = grid.copy()
        g2[n * 10:(n + 1) * 10] += crand(rng, 10)
        diff = np.abs(fo.tx_frame(gm, g2) - base)
        lo, hi = off + sig[n], off + sig[n] + 3 * d.N // 2
        assert np.all(diff[:lo] == 0) and np.all(diff[hi:] == 0)
        assert diff[lo:hi].max() > 1e-3


@pytest.mark.parametrize("N,L,c", [(32, 16, 3), (64, 16, -5), (48, 24, 0), (32, 32, 7)])
def test_sync_zero_cp_equals_continuous(N, L, c):
    """N_CP = 0, lambda = 0.5, continuous lead pad S_L = L_L: symbol-synchronized OLA
    TX equals continuous OLA TX (same blocks, same phases). Holds for any D, I, c;
    catches wrong segment offsets, wrong phi_r, wrong sigma_n."""
    rng = np.random.default_rng(N + L)
    D = rng.uniform(0, 1, L)
    n_cp = (0, 0, 0, 0, 0)
    gs = geom1(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, N, N // 2, L, L, L - 4, c, n_cp, D)
    gc = geom1(fo.CONTINUOUS, fo.OLA, fo.OLS, N, N // 2, L, L, L - 4, c, n_cp, D, lead_pad=N // 4)
    grid = crand(rng, gs.grid_len())
    a, b = fo.tx_frame(gs, grid), fo.tx_frame(gc, grid)
    assert len(a) == len(b)
    assert np.allclose(a, b, atol=1e-12)


@pytest.mark.parametrize("stx", [fo.OLA, fo.OLS])
@pytest.mark.parametrize("c", [3, -7, 10])
def test_sync_i1_is_cp_ofdm_on_continuous_carrier(stx, c):
    """I = 1, D = 1: the symbol-synchronized output is the plain CP-OFDM waveform
    (each symbol with its full CP at its nominal time) times a carrier whose phase
    is continuous across symbols. Pins theta_n: its sign, q running 1..n (R5),
    and the OLS keep windows (R17)."""
    N = L = 32
    n_cp = (8, 5, 6, 5, 7)
    gm = geom1(fo.SYMBOL_SYNC, stx, fo.OLS, N, N // 2, L, L, 20, c, n_cp, np.ones(L))
    rng = np.random.default_rng(c + 100)
    grid = crand(rng, gm.grid_len())
    out = fo.tx_frame(gm, grid)
    # brute force: concatenate CP-OFDM symbols starting at N/4 - N_CP,0 (group time)
    ref = np.zeros(len(out), complex)
    t0 = N // 4 - n_cp[0]
    pos = t0
    for n in range(len(n_cp)):
        x = np.zeros(N, complex)
        act = (np.arange(20) - 10) % N
        x[act] = grid[n * 20:(n + 1) * 20]
        body = np.fft.ifft(x) * math.sqrt(N)
        sym = np.r_[body[N - n_cp[n]:], body]
        ref[pos:pos + len(sym)] = sym
        pos += len(sym)
    t = np.arange(len(out))
    ref *= np.exp(2j * np.pi * c * t / N)
    assert np.allclose(out, ref, atol=1e-12)


@pytest.mark.parametrize("mode,stx,srx", [(fo.SYMBOL_SYNC, fo.OLA, fo.OLS), (fo.SYMBOL_SYNC, fo.OLS, fo.OLA),
                                          (fo.SYMBOL_SYNC, fo.OLA, fo.OLA), (fo.CONTINUOUS, fo.OLS, fo.OLS),
                                          (fo.CONTINUOUS, fo.OLA, fo.OLA), (fo.CONTINUOUS, fo.OLA, fo.OLS)])
def test_round_trip_exact_at_i1_full_band(mode, stx, srx):
    """I = 1 and D = 1: RX(TX(grid)) == grid exactly (the filter is the identity),
    for every TX/RX scheme pair. Catches CP-removal and concatenation offsets."""
    N = L = 32
    n_cp = (8, 4, 4, 8) if mode == fo.SYMBOL_SYNC else (8, 4, 4, 8)
    gm = geom1(mode, stx, srx, N, N // 2, L, L, 24, 5, n_cp, np.ones(L))
    grid = crand(np.random.default_rng(1), gm.grid_len())
    assert np.allclose(fo.rx_frame(gm, fo.tx_frame(gm, grid)), grid, atol=1e-12)


def test_round_trip_rc_filtered_small_error():
    """I = 2, RC transition bins: RX(TX(grid)) ~= grid up to FC distortion and the
    inter-symbol leakage of zero-phase weights (about -33 dB here); a wrong gain,
    sign or bin map gives O(1) error (0 dB or worse)."""
    for mode, stx, srx in [(fo.SYMBOL_SYNC, fo.OLA, fo.OLS), (fo.CONTINUOUS, fo.OLS, fo.OLS),
                           (fo.CONTINUOUS, fo.OLA, fo.OLS)]:
        N, L = 256, 128
        n_cp = (18, 16, 16, 16, 18, 16)
        D = wl.rc_transition_weights(L, 72, 8)
        gm = geom1(mode, stx, srx, N, N // 2, L, L, 72, -40, n_cp, D)
        grid = wl.qam_grid(gm, 1, 5)[0]
        est = fo.rx_frame(gm, fo.tx_frame(gm, grid))
        evm = 10 * np.log10(np.sum(np.abs(est - grid) ** 2) / np.sum(np.abs(grid) ** 2))
        assert evm < -28, (mode, stx, srx, evm)


def test_sync_matches_continuous_bodies_i2():
    """I = 2 with CPs: symbol-synchronized and continuous TX agree on the symbol
    bodies up to FC distortion; a wrong theta_n sign or index makes them differ by O(1)."""
    N, L = 256, 128
    n_cp = (20, 16, 16, 16, 20, 16)
    D = wl.rc_transition_weights(L, 72, 8)
    c = 37
    gs = geom1(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, N, N // 2, L, L, 72, c, n_cp, D)
    gc = geom1(fo.CONTINUOUS, fo.OLA, fo.OLS, N, N // 2, L, L, 72, c, n_cp, D)
    grid = wl.qam_grid(gs, 1, 9)[0]
    a, b = fo.tx_frame(gs, grid), fo.tx_frame(gc, grid)
    # align on symbol 0's CP start
    ta = N // 4 - n_cp[0]
    tb = N // 2
    n = sum(n_cp) + len(n_cp) * N
    # the continuous carrier is referenced to its own time origin: remove the offset phase
    ph = np.exp(2j * np.pi * c * (ta - tb) / N)
    err = a[ta:ta + n] - b[tb:tb + n] * ph
    rel = np.sum(np.abs(err) ** 2) / np.sum(np.abs(a[ta:ta + n]) ** 2)
    assert 10 * np.log10(rel) < -35


def test_single_subcarrier_tone_i2():
    """One active SC k, I = 2: the TX body is ~ exp(j2pi(c+k)t/N)/sqrt(N) at high rate
    (amplitude 1/sqrt(L) * 1/sqrt(I)). Pins the sqrt(I) gain and the direction of
    the bin map at I > 1."""
    N, L = 128, 64
    D = wl.rc_transition_weights(L, 40, 6)
    gm = geom1(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, N, N // 2, L, L, 40, 11, (0,), D)
    grid = np.zeros(40, complex)
    k = 7
    grid[k + 20] = 1
    out = fo.tx_frame(gm, grid)
    t0 = N // 4
    mid = np.arange(t0 + N // 8, t0 + N - N // 8)
    ref = np.exp(2j * np.pi * (11 + k) * (mid - t0) / N) / math.sqrt(N)
    # the carrier phase at the body start is exp(j2pi c t0/N)
    ref = ref * np.exp(2j * np.pi * 11 * t0 / N)
    assert np.max(np.abs(out[mid] - ref)) < 0.05 / math.sqrt(N)


def test_multi_group_frame_is_sum_of_groups():
    """x = sum_m w_m (Sec. III-B): a two-group frame equals the sum of single-group
    frames placed at the common symbol-0 CP time (reading R14)."""
    gm = wl.config_mixed_20mhz()
    # shrink to 2 symbols per group for speed
    ga = wl.Group(2048, 1024, gm.groups[0].n_cp[:2])
    gb = wl.Group(1024, 512, gm.groups[1].n_cp[:4])
    gm2 = wl.Geometry(gm.mode, gm.scheme_tx, gm.scheme_rx, (ga, gb), gm.subbands)
    grid = wl.qam_grid(gm2, 1, 3)[0]
    full = fo.tx_frame(gm2, grid)
    na = ga.n_symbols * gm.subbands[0].n_active
    only_a = wl.Geometry(gm.mode, gm.scheme_tx, gm.scheme_rx, (ga,), (gm.subbands[0],))
    sb_b = wl.Subband(512, 512, 288, 159, 0, gm.subbands[1].weights)
    only_b = wl.Geometry(gm.mode, gm.scheme_tx, gm.scheme_rx, (gb,), (sb_b,))
    wa = fo.tx_frame(only_a, grid[:na])
    wb = fo.tx_frame(only_b, grid[na:])
    offs, flen = fo.frame_layout(gm2)
    ref = np.zeros(flen, complex)
    ref[offs[0]:offs[0] + len(wa)] += wa
    ref[offs[1]:offs[1] + len(wb)] += wb
    assert np.allclose(full, ref, atol=1e-13)
    # symbol 0 CP start: A at 512-160 = 352, B at 256-88 = 168 -> B placed 184 later
    assert offs == [0, 184]


def test_linearity():
    gm = sync_geom(D=wl.rc_transition_weights(16, 10, 2))
    rng = np.random.default_rng(2)
    a, b = crand(rng, gm.grid_len()), crand(rng, gm.grid_len())
    al, be = 0.3 - 1.1j, -2.0 + 0.5j
    assert np.allclose(fo.tx_frame(gm, al * a + be * b), al * fo.tx_frame(gm, a) + be * fo.tx_frame(gm, b))
    w = crand(rng, fo.frame_len(gm))
    v = crand(rng, fo.frame_len(gm))
    assert np.allclose(fo.rx_frame(gm, al * w + be * v), al * fo.rx_frame(gm, w) + be * fo.rx_frame(gm, v))


def test_invalid_sync_geometry_rejected():
    with pytest.raises(ValueError):
        fo.tx_frame(sync_geom(n_cp=(9,)), np.zeros(10))          # N_CP > N/4
    with pytest.raises(ValueError):
        g = geom1(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, 32, 8, 16, 16, 10, 0, (2,), np.ones(16))
        fo.tx_frame(g, np.zeros(10))                              # lambda != 0.5


# ---------------------------------------------------------------------------
# Simplified RX (eq:reduc)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [16, 32, 64])
def test_halfband_complement(L):
    """C + Omega_{L/2} C Omega_{L/2} = I: the two half windows add to the identity
    (the lowpass/highpass pair behind eq:reduc)."""
    C = fo.halfband_C(L)
    O = np.diag(fo.omega(L, L // 2))
    assert np.allclose(C + O @ C @ O, np.eye(L), atol=1e-12)


@pytest.mark.parametrize("N,L,c,n_cp", [(32, 16, 3, (6, 4, 4, 5)), (64, 32, -9, (16, 8, 0, 13)),
                                        (2048, 1024, -300, (160, 144)), (48, 24, 5, (12, 3))])
def test_simplified_rx_equals_direct(N, L, c, n_cp):
    """eq:reduc == eq:FCcomb (direct RX: two short IDFTs, concatenation, OFDM DFT)
    exactly, for arbitrary received waveforms (reading R9: circular P^(+-L/4))."""
    rng = np.random.default_rng(N + L)
    D = rng.uniform(0, 1, L)
    gm = geom1(fo.SYMBOL_SYNC, fo.OLA, fo.OLS, N, N // 2, L, L, L - 4, c, n_cp, D)
    w = crand(rng, fo.frame_len(gm))
    a = fo.rx_frame(gm, w)
    b = fo.rx_frame(gm, w, simplified=True)
    assert np.allclose(a, b, atol=1e-10 * np.max(np.abs(a)))


# ---------------------------------------------------------------------------
# time-domain I/O (the FC part alone)
# ---------------------------------------------------------------------------

def _time_input_from_grid(geom, grid):
    """Concatenated low-rate CP-OFDM symbols of every subband, from a QAM grid."""
    parts = []
    for sub, rows in zip(geom.subbands, fo.split_grid(geom, grid)):
        d = fo.Dims(geom.groups[sub.group], sub)
        l_cp = fo.low_rate_cp(d, geom.mode)
        parts += [fo.cp_insert(fo.ofdm_modulate(rows[n], d.L_ofdm), l_cp[n]) for n in range(d.B)]
    return np.concatenate(parts)


@pytest.mark.parametrize("mode,stx,srx", [(fo.SYMBOL_SYNC, fo.OLA, fo.OLS), (fo.SYMBOL_SYNC, fo.OLS, fo.OLA),
                                          (fo.CONTINUOUS, fo.OLA, fo.OLA), (fo.CONTINUOUS, fo.OLS, fo.OLS)])
def test_time_io_is_the_fc_part_of_the_grid_path(mode, stx, srx):
    """Catches a time layout (CP, body, subband order) or a scale that differs from the
    OFDM stage: TX on the modulated symbols equals TX on the grid, and RX bodies
    demodulated equal RX on the grid."""
    rng = np.random.default_rng(5)
    g1 = wl.Group(64, 32, (16, 8, 8, 12) if mode == fo.SYMBOL_SYNC else (8, 8, 8, 8))
    subs = (wl.Subband(32, 32, 18, 7, 0, wl.rc_transition_weights(32, 18, 3)),
            wl.Subband(32, 32, 10, -12, 0, wl.rc_transition_weights(32, 10, 3)))
    geom = wl.Geometry(mode, stx, srx, (g1,), subs)
    grid = crand(rng, geom.grid_len())
    t_in = _time_input_from_grid(geom, grid)
    assert len(t_in) == sum(fo.time_lengths(geom)[0])
    w_grid = fo.tx_frame(geom, grid)
    w_time = fo.tx_frame(geom, t_in, io_time=True)
    assert np.max(np.abs(w_time - w_grid)) < 1e-12 * np.max(np.abs(w_grid))
    x = crand(rng, len(w_grid))
    bodies = fo.rx_frame(geom, x, io_time=True)
    assert len(bodies) == sum(fo.time_lengths(geom)[1])
    est, pos = [], 0
    for sub in geom.subbands:
        d = fo.Dims(geom.groups[sub.group], sub)
        for n in range(d.B):
            est.append(fo.ofdm_demodulate(bodies[pos:pos + d.L_ofdm], d.L_act))
            pos += d.L_ofdm
    ref = fo.rx_frame(geom, x)
    assert np.max(np.abs(np.concatenate(est) - ref)) < 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# the paper's complexity model (printed values)
# ---------------------------------------------------------------------------

def test_complexity_printed_values():
    """Sec. V prints mu(128) = 516 and mu(16) = 20, and the simplified RX replaces
    three low-rate transforms (two short IDFTs, one OFDM DFT) by two (beta = 1/2)."""
    assert fo.mu(128) == 516 and fo.mu(16) == 20
    L = 128
    direct = 2 * 1.0 * fo.mu(L) + fo.mu(L)           # transform part of C_low-rate, beta = 1
    reduced = 2 * 0.5 * fo.mu(L) + fo.mu(L)          # beta = 1/2
    assert abs((direct - reduced) / direct - 1 / 3) < 1e-12
    # the per-symbol total adds the weights (6 alpha N_tb) and the shared long transform
    c = fo.complexity_per_symbol(256, [(128, 128, 8)])
    assert c == 2 * fo.mu(256) + 2 * fo.mu(128) + 6 * 2 * 8 + fo.mu(128)


# ---------------------------------------------------------------------------
# the symbol-synchronized frame as explicit matrices from the printed equations
# ---------------------------------------------------------------------------

def _frame_matrix(geom):
    """TX of one subband as sum_n Gamma_{sigma_n} sum_r R_N^{(r)} [S_r] F_r(theta_n)
    [A_r] R_L^{(r)} Pad_n K_{CP,n} X_OFDM, each factor a dense matrix written from its
    equation (eq:TX_OFDMmod, eq:TX_CPins, eq:padding, eq:ola_proc windows, eq:ola_synthesis
    blocks, R placement, eq:multi-symb), for brute force over every basis input."""
    g, sub = geom.groups[0], geom.subbands[0]
    N, L, B, La, c = g.n_long, sub.l_short, len(g.n_cp), sub.n_active, sub.centre_bin
    I = N / L
    L_L, L_T, N_L, N_T = L // 4, L // 4, N // 4, N // 4
    L_S, N_S = L // 2, N // 2
    l_cp = [n_cp * L // N for n_cp in g.n_cp]
    W = lambda n: np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    Winv = lambda n: np.conj(W(n)) / n
    act = np.zeros((L, La))
    for a in range(La):
        act[(a - La // 2) % L, a] = 1.0                              # signed frequencies
    Xofdm = np.sqrt(L) * Winv(L) @ act
    Pshift = np.zeros((L, L))
    for p in range(L):
        Pshift[p, (p - L // 2) % L] = 1.0                            # P^(L/2)
    Dm = np.diag(np.asarray(sub.weights, float))
    Q = N_L + N_T + B * N + sum(g.n_cp[1:])
    T = np.zeros((Q, B * La), dtype=complex)
    cps = 0
    sigma = 0
    for n in range(B):
        if n > 0:
            cps += g.n_cp[n]
            sigma = n * N + cps
        theta = np.exp(2j * np.pi * c * cps / N)
        lc = l_cp[n]
        K = np.vstack([np.eye(L)[L - lc:], np.eye(L)]) if lc else np.eye(L)
        pad = np.zeros((3 * L // 2, lc + L))
        pad[L_L - lc: L_L + L, :] = np.eye(lc + L)
        for r in range(2):
            RL = np.zeros((L, 3 * L // 2))
            RL[:, r * L // 2: r * L // 2 + L] = np.eye(L)
            if geom.scheme_tx == fo.OLA:
                win = np.zeros(L)
                if r == 0:
                    win[L_L - lc: L_L + L_S] = 1.0
                else:
                    win[L_L: L_L + L_S] = 1.0
                A = np.diag(win)
            else:
                A = np.eye(L)
            phi = np.exp(2j * np.pi * r * c * L_S / L)
            Xi = np.zeros((N, L), dtype=complex)
            for p in range(L):
                Xi[(c + p - L // 2) % N, p] = phi * theta
            F = np.sqrt(I) * Winv(N) @ Xi @ Dm @ Pshift @ W(L)
            if geom.scheme_tx == fo.OLS:
                s_win = np.zeros(N)
                if r == 0:
                    s_win[N_L - g.n_cp[n]: N_L + N_S] = 1.0
                else:
                    s_win[N_L: N_L + N_S] = 1.0
                F = np.diag(s_win) @ F
            RN = np.zeros((3 * N // 2, N))
            RN[r * N // 2: r * N // 2 + N, :] = np.eye(N)
            Gam = np.zeros((Q, 3 * N // 2))
            Gam[sigma: sigma + 3 * N // 2, :] = np.eye(3 * N // 2)
            T[:, n * La:(n + 1) * La] += Gam @ RN @ F @ A @ RL @ pad @ K @ Xofdm
    return T


@pytest.mark.parametrize("stx", [fo.OLA, fo.OLS])
def test_sync_frame_matches_matrix_transcription(stx):
    """Catches an index, window, phase or placement slip anywhere in the symbol-sync
    assembly: every basis input through the oracle equals the column of the matrix."""
    D = wl.rc_transition_weights(16, 8, 2)
    geom = geom1(fo.SYMBOL_SYNC, stx, fo.OLS, 32, 16, 16, 16, 8, 5, (8, 4, 0), D)
    T = _frame_matrix(geom)
    for j in range(T.shape[1]):
        e = np.zeros(T.shape[1], dtype=complex)
        e[j] = 1.0
        assert np.max(np.abs(fo.tx_frame(geom, e) - T[:, j])) < 1e-12


def test_bf16_round_ties_bound_and_library():
    """BF16 rounding of the complex-BF16 I/O expected values: hand-worked ties to even
    (catches ties away from zero and a significand of 7 instead of 8 bits), the half-ulp
    bound and idempotence (catches a binade off by one), and torch's CPU float32 ->
    bfloat16 conversion on float32 inputs, where one rounding is the whole conversion."""
    torch = pytest.importorskip("torch")
    # spacing 2^-7 on [1, 2), 1 on [128, 256), 2^-133 among the subnormals
    worked = [(1 + 2.0**-8, 1.0), (1 + 3 * 2.0**-8, 1 + 2.0**-6), (-(1 + 2.0**-8), -1.0),
              (1 + 2.0**-7, 1 + 2.0**-7), (1 + 2.0**-8 + 2.0**-30, 1 + 2.0**-7), (254.5, 254.0), (255.5, 256.0),
              (1.5 * 2.0**-133, 2.0**-132), (0.0, 0.0), (3.0, 3.0)]
    for v, want in worked:
        assert fo.bf16_round(np.array([v]))[0] == want, (v, want)
    z = fo.bf16_round(np.array([1 + 2.0**-8 + 1j * (255.5)]))[0]
    assert z == 1.0 + 256.0j
    rng = np.random.default_rng(7)
    v = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32)
    k = rng.integers(128, 256, 4000)
    e = rng.integers(-120, 120, 4000)
    ties = (np.ldexp(k + 0.5, e - 7) * rng.choice([-1.0, 1.0], 4000)).astype(np.float32)   # exact in float32
    v = np.concatenate([v, ties])
    lib = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    mine = fo.bf16_round(v.astype(np.float64))
    assert np.array_equal(mine, lib)
    w = rng.standard_normal(20000) * 10.0 ** rng.uniform(-20, 20, 20000)
    r = fo.bf16_round(w)
    assert np.all(np.abs(r - w) <= 2.0**-8 * np.abs(w))
    assert np.array_equal(fo.bf16_round(r), r)
