"""The C-ABI library builds, loads and exports every function include/mpdict.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpdict.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mp_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g

    g._load_build_module().build()
    return os.path.join(ROOT, "paper_2112_12965_gb300", "libmpdict.so")


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("mp_init", "mp_shutdown", "mp_dict_load", "mp_dict_free", "mp_ab_join", "mp_submit", "mp_poll",
                 "mp_last_error"):
        assert name in fns


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mp_\w+)", out))
    assert set(declared_functions()) <= exported


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "mpdict.h"\nint main(void){mp_config c; return mp_config_default(&c) == 0 ? 0 : 1;}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                    "-o", str(tmp_path / "t.o")], check=True)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """The Python binding has no CPU fallback: a missing library is an error."""
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "mp_binding_copy", os.path.join(ROOT, "paper_2112_12965_gb300", "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(os.path, "exists", lambda p: False if p.endswith("libmpdict.so") else True)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        spec.loader.exec_module(mod)
