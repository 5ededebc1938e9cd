"""Seeded synthetic 5G-NR-shaped workloads for FC-filtered CP-OFDM.

This module is shared by the FP64 oracle, the tests and the benchmark. It holds
only *descriptions* of the processing geometry (numerology, subband placement,
CP schedules, transition weights chosen as an input) and seeded random data
(QAM grids, AWGN). It contains none of the fast-convolution arithmetic: no
transform, window, bin map, phase or block assembly lives here.

Conventions shared with the C ABI (``include/fcofdm.h``):

* ``mode``: 0 = continuous FC processing (Sec. II), 1 = symbol-synchronized
  discontinuous FC processing (Sec. III-IV).
* ``scheme_tx`` / ``scheme_rx``: 0 = overlap-and-add, 1 = overlap-and-save.
* A QAM grid for one stream is the concatenation, subband by subband in the
  order given, of ``[B_g][L_act,m]`` complex symbols, where ``B_g`` is the
  symbol count of the subband's numerology group. Active subcarriers are stored
  in ascending signed frequency ``f = -floor(L_act/2) ... ceil(L_act/2)-1``.
* Weights ``D_m`` are real, one per short-transform bin, in fftshifted order
  (index ``p`` holds signed bin ``p - floor(L_m/2)``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

CONTINUOUS, SYMBOL_SYNC = 0, 1
OLA, OLS = 0, 1


@dataclass(frozen=True)
class Group:
    """One numerology group: shares the long transform size and symbol timing."""
    n_long: int                 # N, long (high-rate) transform size
    n_overlap: int              # N_O = lambda*N high-rate overlap samples
    n_cp: tuple                 # N_CP,n per symbol, high-rate samples (len = B)
    lead_pad: int = -1          # continuous mode: S_L*I_m in high-rate samples; -1 -> N_O

    @property
    def n_symbols(self) -> int:
        return len(self.n_cp)


@dataclass(frozen=True)
class Subband:
    """One FC subband (Sec. II, Sec. III-A); ``weights`` is D_m in fftshifted order."""
    l_short: int                # L_m
    l_ofdm: int                 # L_OFDM,m
    n_active: int               # L_act,m
    centre_bin: int             # c_m on the long grid (may be negative)
    group: int                  # index into Geometry.groups
    weights: np.ndarray = field(compare=False, repr=False)


@dataclass(frozen=True)
class Geometry:
    mode: int
    scheme_tx: int
    scheme_rx: int
    groups: tuple
    subbands: tuple
    name: str = ""
    qam_order: int = 4
    flags: int = 0               # ABI flags (e.g. force the generic kernels); no effect on the result

    def grid_len(self) -> int:
        """Complex QAM symbols per stream (sum over subbands of B_g * L_act,m)."""
        return sum(self.groups[s.group].n_symbols * s.n_active for s in self.subbands)

    def nominal_samples(self) -> int:
        """High-rate samples of the nominal signal duration (symbols + CPs) per stream."""
        g = self.groups[0]
        per_sym = g.n_long if self.mode == SYMBOL_SYNC else None
        if per_sym is None:
            sb = next(s for s in self.subbands if s.group == 0)
            per_sym = sb.l_ofdm * g.n_long // sb.l_short
        return sum(per_sym + c for c in g.n_cp)


# ---------------------------------------------------------------------------
# 5G NR numerology helpers (3GPP normal CP): the first symbol of every 0.5 ms
# carries a longer CP. These are signal-format constants, not FC arithmetic.
# ---------------------------------------------------------------------------

def nr_normal_cp(n_fft: int, scs_khz: int, n_symbols: int) -> tuple:
    """Normal-CP lengths at a sampling rate of ``n_fft * scs``.

    The base CP is 144/2048 of the useful symbol; the first symbol of each
    half subframe gets an extra 16/2048 of the 15 kHz symbol (i.e. 16*64*Tc).
    """
    base = 144 * n_fft // 2048
    # the half-subframe extension is 16 samples at 30.72 Msps, scaled to fs = n_fft*scs
    if (16 * n_fft * scs_khz) % 30720:
        raise ValueError("CP extension is not an integer number of samples at this rate")
    ext = 16 * n_fft * scs_khz // 30720
    syms_per_half = 7 * (scs_khz // 15)
    return tuple(base + (ext if (n % syms_per_half) == 0 else 0) for n in range(n_symbols))


def rc_transition_weights(l_short: int, n_active: int, n_tb: int) -> np.ndarray:
    """Frequency window D_m: ones on the active bins, raised-cosine transition bins.

    Transition bin j = 1..n_tb counted outward from the passband edge gets
    0.5*(1 + cos(pi*j/(n_tb+1))); all other bins are zero. Returned in fftshifted
    order (index p <-> signed bin p - floor(L/2)). The paper leaves the weight
    values to the designer, so these are an input choice, not part of the method.
    """
    w = np.zeros(l_short, dtype=np.float64)
    lo = -(n_active // 2)
    hi = lo + n_active            # exclusive
    half = l_short // 2
    if hi - lo + 2 * n_tb > l_short:
        raise ValueError("passband plus transition bands exceed the short transform")
    w[lo + half: hi + half] = 1.0
    for j in range(1, n_tb + 1):
        v = 0.5 * (1.0 + math.cos(math.pi * j / (n_tb + 1)))
        w[hi - 1 + j + half] = v
        w[lo - j + half] = v
    return w


def full_band_weights(l_short: int) -> np.ndarray:
    return np.ones(l_short, dtype=np.float64)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def config_single_5mhz() -> Geometry:
    """5 MHz NR, 15 kHz SCS, 24 PRB (288 SC), N=512 at 7.68 Msps, L=384,
    50% overlap-save on TX and RX, 14 symbols (one slot), QPSK, 8 RC bins."""
    n_cp = nr_normal_cp(512, 15, 14)                      # 40, 36 x6, 40, 36 x6
    g = Group(n_long=512, n_overlap=256, n_cp=n_cp)
    sb = Subband(l_short=384, l_ofdm=384, n_active=288, centre_bin=0, group=0,
                 weights=rc_transition_weights(384, 288, 8))
    return Geometry(CONTINUOUS, OLS, OLS, (g,), (sb,), name="nr5mhz_15khz_24prb_L384_N512_ols", qam_order=4)


def config_mixed_20mhz() -> Geometry:
    """20 MHz at 30.72 Msps, 1 ms subframe, symbol-synchronized FC.

    Group A: 15 kHz SCS, N=2048, 51 PRB (612 SC), L=1024, 14 symbols.
    Group B: 30 kHz SCS, N=1024, 24 PRB (288 SC), L=512, 28 symbols.
    A occupies 15 kHz bins [-606, 6), B occupies [30, 606) (B's own 30 kHz grid:
    [15, 303)), a 24-bin (2 PRB) guard between them. OLA TX, OLS RX, 16-QAM.
    """
    ga = Group(n_long=2048, n_overlap=1024, n_cp=nr_normal_cp(2048, 15, 14))
    gb = Group(n_long=1024, n_overlap=512, n_cp=nr_normal_cp(1024, 30, 28))
    sa = Subband(l_short=1024, l_ofdm=1024, n_active=612, centre_bin=-300, group=0,
                 weights=rc_transition_weights(1024, 612, 8))
    sbb = Subband(l_short=512, l_ofdm=512, n_active=288, centre_bin=159, group=1,
                  weights=rc_transition_weights(512, 288, 8))
    return Geometry(SYMBOL_SYNC, OLA, OLS, (ga, gb), (sa, sbb),
                    name="nr20mhz_mixed_15k51prb_30k24prb_symsync", qam_order=16)


def config_100mhz(n_slots: int = 10) -> Geometry:
    """100 MHz NR, 30 kHz SCS, 273 PRB (3276 SC), N=L=4096 at 122.88 Msps,
    50% overlap (OLA TX, OLS RX), ``n_slots`` slots of 14 symbols, 64-QAM."""
    g = Group(n_long=4096, n_overlap=2048, n_cp=nr_normal_cp(4096, 30, 14 * n_slots))
    sb = Subband(l_short=4096, l_ofdm=4096, n_active=3276, centre_bin=0, group=0,
                 weights=rc_transition_weights(4096, 3276, 8))
    return Geometry(CONTINUOUS, OLA, OLS, (g,), (sb,), name=f"nr100mhz_30khz_273prb_N4096_{n_slots}slots",
                    qam_order=64)


def config_nr10mhz_52prb(mode: int = CONTINUOUS) -> Geometry:
    """10 MHz NR at 15.36 Msps, N=1024, 15 kHz SCS, one subband of 52 PRB (624 SC) with
    8 raised-cosine transition bins per side, one slot of 14 symbols, 16-QAM: the
    wide-band scenario of the paper's EVM figures (continuous or symbol-synchronized
    processing on both sides). The paper does not state its short transform; L=768
    (I = 4/3, the smallest 3 x 2^k above 624 + 16 bins) is this workload's choice.
    OLA TX, OLS RX."""
    g = Group(n_long=1024, n_overlap=512, n_cp=nr_normal_cp(1024, 15, 14))
    sb = Subband(l_short=768, l_ofdm=768, n_active=624, centre_bin=0, group=0,
                 weights=rc_transition_weights(768, 624, 8))
    tag = "cont" if mode == CONTINUOUS else "symsync"
    return Geometry(mode, OLA, OLS, (g,), (sb,), name=f"nr10mhz_15khz_52prb_L768_N1024_{tag}", qam_order=16)


# NR sampling rates with power-of-two FFT sizes per channel bandwidth (MHz -> Msps)
NR_RATE_MSPS = {5: 7.68, 10: 15.36, 20: 30.72, 50: 61.44, 100: 122.88}
# (bandwidth MHz, SCS kHz) pairs NR defines: no 100 MHz at 15 kHz, no 5 MHz at 60 kHz
NR_BW_SCS = tuple((bw, scs) for bw in (5, 10, 20, 50, 100) for scs in (15, 30, 60)
                  if (bw, scs) not in ((100, 15), (5, 60)))


def _short_len(n_active: int, n_long: int, n_tb: int = 8) -> int:
    """Smallest power of two holding the active bins plus both transition bands."""
    L = 16
    while L < n_active + 2 * n_tb:
        L *= 2
    return min(L, n_long)


def config_uneven_carriers(seed: int = 1400, n_carriers: int = 64, n_slots: int = 4,
                           whole_cp_period: bool = False) -> list:
    """Independent carriers of uneven shape, one geometry each.

    Per carrier (seeded PCG64): a (bandwidth, SCS) pair NR defines, drawn uniformly;
    the NR sampling rate of that bandwidth, so N = f_s / SCS is a power of two
    (128 .. 4096); 1-8 subbands of 1-273 PRB each, drawn one after another while
    the total, with a 2-PRB guard between neighbours, stays within 90 % of the
    bandwidth; each subband's short transform is the smallest power of two holding
    its active subcarriers and 8 raised-cosine transition bins per side. Subbands sit
    side by side from the low band edge, centred on DC as a whole. Symbol-synchronized
    FC (OLA TX, OLS RX), n_slots slots of 14 symbols with NR normal CP, QPSK/16/64-QAM.
    whole_cp_period: a 60 kHz carrier gets 2 n_slots slots, so that every frame holds
    whole 0.5 ms CP periods (the long CP every 28 symbols) and repeats slot after slot.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_carriers):
        bw, scs = NR_BW_SCS[int(rng.integers(len(NR_BW_SCS)))]
        n_long = int(round(NR_RATE_MSPS[bw] * 1000 / scs))
        budget = int(0.9 * bw * 1000 // (12 * scs))
        prbs = []
        for _ in range(int(rng.integers(1, 9))):
            left = budget - sum(prbs) - 2 * len(prbs)
            if left < 1:
                break
            prbs.append(int(rng.integers(1, min(273, left) + 1)))
        width = 12 * (sum(prbs) + 2 * (len(prbs) - 1))
        lo = -(width // 2)
        subs = []
        for prb in prbs:
            n_act = 12 * prb
            L = _short_len(n_act, n_long)
            subs.append(Subband(l_short=L, l_ofdm=L, n_active=n_act, centre_bin=lo + n_act // 2, group=0,
                                weights=rc_transition_weights(L, n_act, 8)))
            lo += n_act + 24
        slots = n_slots * (2 if whole_cp_period and scs == 60 else 1)
        g = Group(n_long=n_long, n_overlap=n_long // 2, n_cp=nr_normal_cp(n_long, scs, 14 * slots))
        qam = (4, 16, 64)[int(rng.integers(3))]
        out.append(Geometry(SYMBOL_SYNC, OLA, OLS, (g,), tuple(subs),
                            name=f"carrier{i}_{bw}MHz_{scs}kHz_{len(subs)}sb", qam_order=qam))
    return out


TDD_PATTERNS = ("DDDSU", "DDSUU", "DDDDDDDSUU", "DSUUU")


def serving_trace(n_carriers: int, n_requests: int, rate_hz: float, seed: int) -> list:
    """Slot requests for a serving run: Poisson arrivals at rate_hz over all carriers,
    each arrival for a carrier drawn uniformly; a carrier's k-th request is its slot k,
    whose direction follows the carrier's seeded TDD pattern (D and S slots -> TX,
    U -> RX). Returns sorted (arrival_s, carrier, direction 0=TX / 1=RX) tuples."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pattern = [TDD_PATTERNS[int(rng.integers(len(TDD_PATTERNS)))] for _ in range(n_carriers)]
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_requests))
    who = rng.integers(0, n_carriers, n_requests)
    count = [0] * n_carriers
    out = []
    for ti, c in zip(t, who):
        c = int(c)
        p = pattern[c]
        out.append((float(ti), c, 1 if p[count[c] % len(p)] == "U" else 0))
        count[c] += 1
    return out


NAMED = {
    "single5": config_single_5mhz,
    "mixed20": config_mixed_20mhz,
    "nr100": config_100mhz,
    "nr10_52prb": config_nr10mhz_52prb,
}


# ---------------------------------------------------------------------------
# Seeded data
# ---------------------------------------------------------------------------

def _qam_levels(order: int) -> np.ndarray:
    m = int(round(math.sqrt(order)))
    if m * m != order:
        raise ValueError("square QAM only")
    lv = np.arange(-(m - 1), m, 2, dtype=np.float64)
    norm = math.sqrt(2.0 * np.mean(lv ** 2))
    return lv / norm


def qam_grid(geom: Geometry, n_streams: int, seed: int) -> np.ndarray:
    """Uniform random square-QAM symbols at unit average power.

    Returns complex128 ``[n_streams, grid_len]``; stream ``s`` uses
    ``Generator(PCG64(seed + s))`` so any stream can be regenerated alone.
    """
    lv = _qam_levels(geom.qam_order)
    out = np.empty((n_streams, geom.grid_len()), dtype=np.complex128)
    for s in range(n_streams):
        rng = np.random.Generator(np.random.PCG64(seed + s))
        i = rng.integers(0, len(lv), size=(2, out.shape[1]))
        out[s] = lv[i[0]] + 1j * lv[i[1]]
    return out


def gaussian_vector(n: int, seed: int) -> np.ndarray:
    """Circular complex Gaussian vector, unit variance per complex sample."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2.0)


def awgn(wave: np.ndarray, snr_db: float, seed: int) -> np.ndarray:
    """Complex AWGN with variance set from the mean power of ``wave`` (per row)."""
    wave = np.asarray(wave)
    flat = wave.reshape(-1, wave.shape[-1])
    out = np.empty_like(flat, dtype=np.complex128)
    for i in range(flat.shape[0]):
        p = float(np.mean(np.abs(flat[i]) ** 2))
        sigma = math.sqrt(p / (10.0 ** (snr_db / 10.0)))
        out[i] = flat[i] + sigma * gaussian_vector(flat.shape[1], seed + i)
    return out.reshape(wave.shape)


def default_seed(config_index: int) -> int:
    """Seed convention: 1000 + 100*config; stream s adds s."""
    return 1000 + 100 * config_index
