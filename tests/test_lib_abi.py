"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/adg.h.

No compute calls: this runs without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^ADG_API\s+[\w\s\*]+?\b(adg_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2504_06889_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("adg_init_mesh", "adg_set_pde", "adg_set_kernel_precision", "adg_step",
                 "adg_error_vs_exact"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (adg_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    from paper_2504_06889_gb300 import adg

    lib = adg.load()
    for n in declared_symbols():
        assert hasattr(lib, n)
    # host-only calls that touch no device
    assert lib.adg_nvar(adg.EULER, 3) == 5
    assert lib.adg_nvar(adg.ELASTIC, 3) == 9
    assert lib.adg_nvar(adg.SWE, 3) == -1
    assert lib.adg_last_error(None) == b"null context"
    assert lib.adg_create(None) == adg.EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2504_06889_gb300 import adg, build

    monkeypatch.setattr(build, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(adg, "_lib", None)
    with pytest.raises(ImportError):
        adg.load()
