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


def _noalloc_args(adg, dim, N, cells, pde=None, params=(1.4,)):
    import ctypes as C

    cl = (C.c_int * dim)(*cells)
    lo = (C.c_double * dim)(*([0.0] * dim))
    hi = (C.c_double * dim)(*([1.0] * dim))
    par = (C.c_double * len(params))(*params)
    return cl, lo, hi, par


def test_noalloc_rejects_bad_sizes_before_touching_the_device(libpath):
    """adg_step_noalloc checks sizes on the host first: cell counts whose products overflow, more
    cells than adg_init_mesh allows, meshes whose traces exceed the static scratch, and more
    Picard sweeps than adg_set_numerics allows.  Here (no GPU) a check that let such a call
    through would reach the CUDA runtime and return ADG_ECUDA instead.  The state pointer is a
    dummy that no correct path dereferences, so this runs on CPU-only machines only."""
    import ctypes as C

    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("host-side checks only: run where no GPU is visible")
    except ImportError:
        pass
    from paper_2504_06889_gb300 import adg

    lib = adg.load()
    dummy = C.c_void_p(1 << 20)  # 16-byte aligned, never dereferenced
    t = C.c_double(0.0)
    cases = [
        # (cells, picard_iters, expected)
        ((2**20, 2**20, 2**20), 0, adg.EINVAL),      # 2^60 cells: overflow territory
        ((2**31 - 1, 2**31 - 1, 3), 0, adg.EINVAL),
        ((1024, 1024, 1025), 0, adg.EINVAL),          # just above 2^30 cells
        ((64, 64, 64), 0, adg.ENOMEM),                # traces far beyond 32 MiB
        ((1, 1, 2**30), 0, adg.ENOMEM),               # exactly 2^30 cells pass the count check
                                                      # and then exceed the scratch
        ((2, 2, 2), 1001, adg.EINVAL),                # more sweeps than adg_set_numerics allows
        ((2, 2, 2), 2**31 - 1, adg.EINVAL),
        ((0, 2, 2), 0, adg.EINVAL),
        ((-5, 2, 2), 0, adg.EINVAL),
    ]
    for cells, iters, want in cases:
        cl, lo, hi, par = _noalloc_args(adg, 3, 2, cells)
        rc = lib.adg_step_noalloc(adg.EULER, 3, 2, cl, lo, hi, par, 1, 0.5, iters, dummy, 1, C.byref(t),
                                  None, None)
        assert rc == want, (cells, iters, rc, want)
    assert t.value == 0.0
