"""The C-ABI library builds, loads and exports every entry point that
include/vbmc.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vbmc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vbmc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1907_12933_gb300 import build
    return build.build()


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("vbmc_verify_query", "vbmc_verify_batch", "vbmc_get_witness", "vbmc_get_coverage"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_linkage(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in declared_functions():
        assert n in syms, n


def test_binding_raises_without_library(tmp_path, monkeypatch):
    import paper_1907_12933_gb300 as vb
    monkeypatch.setattr(vb, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(vb, "_lib", None)
    with pytest.raises(ImportError):
        vb.lib()


def test_binding_names_match_c_abi():
    import paper_1907_12933_gb300 as vb
    for n in ("verify_query", "verify_query_device", "verify_batch", "get_witness",
              "get_coverage", "get_verdict_bitmap", "get_ties", "result_summary"):
        assert callable(getattr(vb, n))
        assert "vbmc_" + n in declared_functions()
