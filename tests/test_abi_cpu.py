"""Host-side checks that need no GPU: the library builds, loads and exports
every entry point declared in include/kv.h; host-side validation and the
memory model."""
import os
import re

import pytest

import paper_1804_01583_gb300 as kv
from paper_1804_01583_gb300 import build as kvbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            # entry points of the debug build only
            src = re.sub(r"#ifdef KV_DEBUG.*?#endif", "", src, flags=re.S)
            names |= set(re.findall(r"\b(kv_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    kvbuild.build()
    return kv.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(kv.EXPORTED) <= set(names)


def test_version_and_error_string(lib):
    assert "sm_103a" in kv.version()
    assert isinstance(kv.last_error(), str)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kv.KvError) as ei:
        kv.Context(1 << 20)
    assert ei.value.code in (kv.KV_ECUDA, kv.KV_EINVAL)


@pytest.mark.parametrize("std", [["gcc", "-std=c11", "-x", "c"], ["g++", "-std=c++17", "-x", "c++"]])
def test_header_compiles_standalone(std):
    """include/kv.h on its own, as C11 and as C++17, pedantic, warnings as
    errors: the boundary needs no CUDA or torch header."""
    import shutil
    import subprocess
    if not shutil.which(std[0]):
        pytest.skip(f"{std[0]} not found")
    hdr = os.path.join(ROOT, "include", "kv.h")
    r = subprocess.run([std[0], std[1], "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", *std[2:], hdr],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
