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


STRUCTS = ["pf_network", "pf_model", "pf_options", "pf_fsp_options", "pf_ode_options",
           "pf_request", "pf_ctx_config"]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes struct of the binding has the C struct's size and field
    offsets (the header compiled by the host C compiler), so that an option
    added on one side only cannot shift the others."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1606_08281_gb300 import pf
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pf1606.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in getattr(pf, name)._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c_side = {tuple(line.split()[:2]): int(line.split()[2]) for line in out.splitlines()}
    for name in STRUCTS:
        cls = getattr(pf, name)
        assert c_side[(name, "size")] == ct.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert c_side[(name, fname)] == getattr(cls, fname).offset, (name, fname)
