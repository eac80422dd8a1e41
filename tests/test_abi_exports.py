"""The C ABI library builds for sm_103a and exports every entry point that
include/pf1606.h declares (CPU only: no compute call is made)."""
from __future__ import annotations

import ctypes as ct
import re
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions() -> list[str]:
    text = (ROOT / "include" / "pf1606.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not Path("/usr/local/cuda/bin/nvcc").exists():
        pytest.skip("nvcc not available")
    from paper_1606_08281_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["pf_loglik", "pf_strerror", "pf_last_error", "pf_version", "pf_philox4x32_10"]:
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", str(libpath)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pf_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_without_a_gpu(libpath):
    lib = ct.CDLL(str(libpath))
    lib.pf_strerror.restype = ct.c_char_p
    lib.pf_version.restype = ct.c_char_p
    assert lib.pf_strerror(0) == b"ok"
    assert b"sm_103a" in lib.pf_version()


def test_binding_names_match_the_header():
    from paper_1606_08281_gb300 import pf
    for name in declared_functions():
        assert hasattr(pf, name), name
