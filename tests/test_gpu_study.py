"""The lake-at-rest precision study (Secs. 6.3 and 7, shallow water with bathymetry) on a short run:
the FP64 scheme stays well balanced, and the error grows as the precision of the kernels or
of the stored solution drops."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def study():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06889_gb300 import adg as A
    from paper_2504_06889_gb300 import build
    from paper_2504_06889_gb300 import study as S

    build.build()
    A.load()
    return S


def test_lake_table_orders_by_precision(study):
    out = study.lake_table(t_end=0.05, m=9)
    r = {row["mix"]: row for row in out["rows"]}
    assert all(row["t"] >= 0.05 for row in out["rows"] if row["finite"])
    assert r["fp64"]["finite"] and r["fp64"]["l2"] <= 1e-10
    assert r["all fp32"]["l2"] > 10 * r["fp64"]["l2"]
    assert r["storage fp32"]["l2"] < r["storage fp16"]["l2"]
    assert r["storage fp16"]["l2"] < r["storage bf16"]["l2"] or not r["storage bf16"]["finite"]
    assert r["predictor fp32"]["l2"] > r["fp64"]["l2"]
