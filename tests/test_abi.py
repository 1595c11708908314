"""The C-ABI library builds for sm_103a, loads and exports every symbol that
include/overlap.h declares; the Python binding covers each of them.  No
compute call is made (no GPU here)."""
import ctypes
import os
import subprocess

import pytest

from paper_1106_4964_gb300 import binding
from paper_1106_4964_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return b.build()


def test_header_declares_boundary(libpath):
    names = binding.declared_symbols()
    for required in ("ov_set_gauge", "ov_apply_dslash", "ov_apply_Hw", "ov_apply_overlap", "ov_deflate",
                     "ov_cg_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in binding.declared_symbols() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_header(libpath):
    lib = ctypes.CDLL(libpath)
    for n in binding.declared_symbols():
        assert hasattr(lib, n)
    assert set(binding.declared_symbols()) == set(binding._SIGS)


def test_build_targets_sm103a_only():
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(ImportError):
        _fresh_load(str(tmp_path / "nope.so"))


def _fresh_load(path):
    saved = binding._lib
    binding._lib = None
    try:
        binding.load(path)
    finally:
        binding._lib = saved


def test_fast_division_host_side(tmp_path):
    """The invariant-divisor division behind the device coordinate maps, compiled for the host
    and compared with integer division on dense and random numerators below 2^31."""
    import shutil
    import subprocess

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "fastdiv")
    csrc = os.path.join(ROOT, "paper_1106_4964_gb300", "csrc")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", csrc, "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "fastdiv_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout


def test_binding_enums_match_header():
    """The status and precision codes of the Python binding are the header's."""
    import re

    text = open(os.path.join(ROOT, "include", "overlap.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(OV_[A-Z0-9]+)\s*=\s*(-?\d+)", text)}
    for value, name in binding.STATUS.items():
        assert codes[name] == value
    for name in ("OV_F64", "OV_F32", "OV_F16S", "OV_BF16S", "OV_DF64"):
        assert getattr(binding, name) == codes[name]
    assert set(binding.PREC.values()) == {codes[n] for n in ("OV_F64", "OV_F32", "OV_F16S", "OV_BF16S", "OV_DF64")}
