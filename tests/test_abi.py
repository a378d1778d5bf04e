"""The C-ABI library builds, loads and exports every symbol include/ep.h declares
(no compute call: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ep.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:ep_status|const char\s*\*|int64_t|int|void|double)\s+(ep_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_03816_gb300 import build, ep

    build.build()
    return ep.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("ep_rhs", "ep_shoot", "ep_match", "ep_adjoint"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1510_03816_gb300 import build, ep

    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) == set(ep.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ep_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_build_targets_sm_103a_only():
    from paper_1510_03816_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_error_string(lib):
    from paper_1510_03816_gb300 import ep

    assert ep.version() >= 10000
    assert isinstance(ep.last_error(), str)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1510_03816_gb300 import ep

    monkeypatch.setattr(ep, "_lib", None)
    monkeypatch.setattr(ep, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        ep.load()
