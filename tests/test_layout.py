"""Source-level separation rules, checked on the text of the files:

* the product package never imports the oracle (the oracle is test infrastructure:
  tests, smoke() and the bench's CPU legs only) and has no compiler or multi-backend
  layer on its path (no Triton, no torch.compile);
* the oracle and the input generators import nothing from the product package, so the
  two sides of every parity test share no code."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2008_00672_gb300")


def sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_use_the_oracle_or_a_compiler_layer():
    for p in sources(PKG, (".py", ".cu", ".cuh", ".h")):
        txt = open(p).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, flags=re.M), p
        assert "fc_oracle" not in txt, p
        assert not re.search(r"^\s*(from|import)\s+triton\b", txt, flags=re.M), p
        assert "torch.compile" not in txt, p


def test_oracle_and_inputs_do_not_import_the_package():
    for top in (os.path.join(ROOT, "oracle"), os.path.join(ROOT, "workloads")):
        for p in sources(top, (".py",)):
            txt = open(p).read()
            assert not re.search(r"^\s*(from|import)\s+paper_2008_00672_gb300\b", txt, flags=re.M), p
            assert "ctypes" not in txt and "cdll" not in txt.lower(), p


def test_workloads_hold_no_transform_arithmetic():
    """The seeded input module draws numbers and describes geometries; FFTs, the FC
    blocks and the oracle live elsewhere."""
    for p in sources(os.path.join(ROOT, "workloads"), (".py",)):
        txt = open(p).read()
        assert not re.search(r"\b(np|numpy|scipy)\.fft\b|\bfrom\s+(numpy|scipy)\s+import\s+fft\b", txt), p
        assert not re.search(r"^\s*(from|import)\s+oracle\b", txt, flags=re.M), p
