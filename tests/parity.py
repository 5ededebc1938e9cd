"""Element-wise parity bounds shared by the GPU-vs-oracle tests.

A whole-stream norm ||gpu - ref|| / ||ref|| dilutes an error confined to a few
samples by the square root of the stream length (about 180 on a 20 MHz subframe),
so every comparison here also bounds

* each window: the RMS of the error over one symbol's span of the waveform
  (sigma_n .. sigma_n + 3N/2 of eq:multi-symb in symbol-synchronized mode, one FC
  block of N samples at hop N_S in continuous mode, eq:BDM) or over one symbol row of
  the QAM grid (eq:concat2 and the OFDM DFT), relative to the RMS of the whole
  reference. Windows at the frame edges hold the filter ramps and little signal, so
  they are measured against the stream's signal level, not their own;
* each sample: max_i |gpu_i - ref_i| <= SAMPLE_FACTOR * tol * rms(ref).

Why SAMPLE_FACTOR = 5. Each output is a sum of many independently rounded FP32
products and additions through a chain of at most five transforms of up to 2^12
points, plus one rounding to complex64 relative to the sample's own magnitude. The
error is therefore close to Gaussian, with its largest values on the signal's peaks:
rounding an oracle waveform to complex64 alone gives a largest sample error about six
times its RMS error. The path's own RMS errors are 2e-7 (FP32) and 8e-6 (BF16x3 tensor
path), so its largest sample errors sit near 1.5e-6 and 5e-5 of rms(ref), against
bounds of 5e-5 and 1.5e-4: a margin of about 30x and 3x. A single sample off by
1e-4 rms (twice the FP32 bound) fails, which `tests/test_parity_helper.py` checks on
the CPU, together with an error spread over part of one window that passes the
whole-stream bound and fails the window bound.

This module holds no arithmetic of the method: windows come from the oracle's own
layout functions, and the comparison is plain numpy.
"""
import numpy as np

from oracle import fc_oracle as fo

SAMPLE_FACTOR = 5.0


def _rms(a) -> float:
    a = np.asarray(a)
    return float(np.sqrt(np.mean(np.abs(a) ** 2))) if a.size else 0.0


def parity_stats(got, ref, windows=None) -> dict:
    """Error of `got` against `ref` (1-D): whole-array RMS relative error, the worst
    window RMS error and the worst single-sample error, both relative to rms(ref)."""
    got = np.asarray(got).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    d = got.astype(np.complex128) - ref.astype(np.complex128)
    scale = max(_rms(ref), 1e-300)
    stats = {
        "rel": float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300)),
        "window": 0.0,
        "window_at": None,
        "sample": float(np.max(np.abs(d))) / scale if d.size else 0.0,
        "sample_at": int(np.argmax(np.abs(d))) if d.size else None,
    }
    for a, b in windows or ():
        a, b = max(0, int(a)), min(d.size, int(b))
        if b > a:
            w = _rms(d[a:b]) / scale
            if w > stats["window"]:
                stats["window"], stats["window_at"] = w, (a, b)
    return stats


def check(got, ref, tol, windows=None, what="") -> dict:
    """Assert the three bounds (whole array, every window, every sample) and return
    the statistics."""
    s = parity_stats(got, ref, windows)
    assert s["rel"] <= tol, (what, "stream RMS", s)
    assert s["window"] <= tol, (what, "window RMS", s)
    assert s["sample"] <= SAMPLE_FACTOR * tol, (what, "per sample", s)
    return s


def merge(worst: dict, s: dict) -> dict:
    """Keep the largest of each statistic over several checks (for reporting)."""
    out = dict(worst)
    for k in ("rel", "window", "sample"):
        out[k] = max(out.get(k, 0.0), s[k])
    return out


# ---------------------------------------------------------------------------
# windows from the geometry (oracle layout functions only)
# ---------------------------------------------------------------------------

def _first_sub(geom, gi):
    for s in geom.subbands:
        if s.group == gi:
            return s
    return None


def wave_windows(geom) -> list:
    """Symbol-synchronized: [sigma_n, sigma_n + 3N/2) of every group's symbols
    (eq:multi-symb); continuous: every FC block's N output samples at hop N_S (eq:BDM);
    both placed at the group's offset in the frame."""
    offs, flen = fo.frame_layout(geom)
    out = []
    for gi, g in enumerate(geom.groups):
        sub = _first_sub(geom, gi)
        if sub is None:
            continue
        d = fo.Dims(g, sub)
        o = offs[gi]
        if geom.mode == fo.SYMBOL_SYNC:
            for s in fo.sync_sigma(d):
                out.append((o + s, min(flen, o + s + 3 * d.N // 2)))
        else:
            _, glen = fo.group_lead_and_len(geom, gi)
            r = 0
            while r * d.N_S < glen:
                out.append((o + r * d.N_S, min(flen, o + r * d.N_S + d.N)))
                r += 1
    return out


def grid_windows(geom) -> list:
    """One window per symbol row of every subband in the grid layout (subband after
    subband, [B][L_act] each)."""
    out, pos = [], 0
    for s in geom.subbands:
        b = geom.groups[s.group].n_symbols
        for _ in range(b):
            out.append((pos, pos + s.n_active))
            pos += s.n_active
    return out


def body_windows(geom) -> list:
    """One window per recovered OFDM symbol body of the time-domain RX output
    (subband after subband, B bodies of L_OFDM each)."""
    out, pos = [], 0
    for s in geom.subbands:
        b = geom.groups[s.group].n_symbols
        for _ in range(b):
            out.append((pos, pos + s.l_ofdm))
            pos += s.l_ofdm
    return out


def chunk_windows(n: int, size: int) -> list:
    """Consecutive windows of `size` samples covering [0, n)."""
    size = max(1, int(size))
    return [(a, min(n, a + size)) for a in range(0, n, size)]
