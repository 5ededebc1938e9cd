"""The boundary is a C ABI: a plain C11 program (`tests/c_client/abi_client.c`, gcc,
-pedantic -Werror, no C++ or CUDA headers) includes `include/fcofdm.h`, links the
built library, validates a geometry and tries to create a plan. Its sizes must equal
the Python binding's for the same geometry; plan creation returns FC_OK on a GPU
machine and FC_ERR_CUDA (with the plan pointer left NULL) without one."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2008_00672_gb300 import build, fc
    lib = build.build()
    exe = str(tmp_path / "abi_client")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "abi_client.c"),
                        "-L", os.path.dirname(lib), "-lfcofdm", f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.stdout, r.stderr)
    lines = r.stdout.splitlines()
    assert lines[0] == "status 0 FC_OK"
    grid_len, wave_len, nominal = (int(v) for v in lines[1].split()[1:])
    n_cp = tuple(40 if n in (0, 7) else 36 for n in range(14))
    geom = wl.Geometry(wl.SYMBOL_SYNC, wl.OLS, wl.OLS, (wl.Group(512, 256, n_cp),),
                       (wl.Subband(384, 384, 288, 0, 0, np.ones(384)),))
    z = fc.fc_geometry_check(geom)
    assert (grid_len, wave_len, nominal) == (z.grid_len, z.wave_len, z.nominal_len)
    assert grid_len == 14 * 288 and nominal == 7680
    status = int(lines[2].split()[1])
    assert status in (fc.FC_OK, fc.FC_ERR_CUDA)
