"""The FP32 kernels convert between FP64 and FP32 with integer operations (the FP64 unit of this
part, which also converts, is slow).  adg_check_conversions compares them bit for bit with the
hardware conversions on seeded patterns: uniform bit patterns, the range around FP32's, exact
half-way cases and carries into the exponent."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_integer_conversions_match_the_hardware():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06889_gb300 import adg, build

    build.build()
    lib = adg.load()
    for seed in (1, 2):
        bad = C.c_longlong(-1)
        rc = lib.adg_check_conversions(1 << 24, seed, None, C.byref(bad))
        assert rc == adg.OK
        assert bad.value == 0
