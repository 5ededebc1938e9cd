"""The boundary is a C ABI: a plain C11 program (`tests/c_client/abi_client.c`, gcc,
-pedantic -Werror, no C++ or CUDA headers) includes `include/fcofdm.h`, links the
built library, validates a geometry and tries to create a plan. Its sizes must equal
the Python binding's for the same geometry; plan creation returns FC_OK on a GPU
machine and FC_ERR_CUDA (with the plan pointer left NULL) without one. On a GPU
(`-m gpu`) the same client also runs one TX and one RX of 4 streams through the
host-buffer calls, and its output files are compared with the FP64 oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def client_geometry():
    n_cp = tuple(40 if n in (0, 7) else 36 for n in range(14))
    return wl.Geometry(wl.SYMBOL_SYNC, wl.OLS, wl.OLS, (wl.Group(512, 256, n_cp),),
                       (wl.Subband(384, 384, 288, 0, 0, np.ones(384)),))


def build_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2008_00672_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "abi_client")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "abi_client.c"),
                        "-L", os.path.dirname(lib), "-lfcofdm", f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_plain_c_client(tmp_path):
    from paper_2008_00672_gb300 import fc
    exe = build_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    lines = r.stdout.splitlines()
    assert lines[0] == "status 0 FC_OK"
    grid_len, wave_len, nominal = (int(v) for v in lines[1].split()[1:])
    z = fc.fc_geometry_check(client_geometry())
    assert (grid_len, wave_len, nominal) == (z.grid_len, z.wave_len, z.nominal_len)
    assert grid_len == 14 * 288 and nominal == 7680
    status = int(lines[2].split()[1])
    assert status in (fc.FC_OK, fc.FC_ERR_CUDA)


@pytest.mark.gpu
def test_plain_c_client_runs_tx_and_rx(tmp_path):
    """The C client's TX (grid -> waveform) and RX (its own waveform -> grid) through the
    host-buffer calls, against the FP64 oracle with the element-wise bounds."""
    from oracle import fc_oracle as fo
    from tests import parity
    exe = build_client(tmp_path)
    out = tmp_path / "out"
    out.mkdir()
    r = subprocess.run([exe, str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert all(line.startswith("status 0 ") for line in r.stdout.splitlines() if line.startswith("status"))
    geom = client_geometry()
    grid = np.fromfile(out / "grid.bin", dtype=np.complex64).reshape(4, -1)
    wave = np.fromfile(out / "wave.bin", dtype=np.complex64).reshape(4, -1)
    est = np.fromfile(out / "est.bin", dtype=np.complex64).reshape(4, -1)
    ww, gw = parity.wave_windows(geom), parity.grid_windows(geom)
    for s in range(4):
        parity.check(wave[s], fo.tx_frame(geom, grid[s].astype(np.complex128)), 1e-5, ww, ("tx", s))
        parity.check(est[s], fo.rx_frame(geom, wave[s].astype(np.complex128)), 1e-5, gw, ("rx", s))
