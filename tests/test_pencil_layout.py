"""Layout constants of the pencil-task Picard sweep (pt_layout in adg_kernels.cuh), replayed on the
CPU: for every configuration the library builds, the shared-memory indices of the node threads and
of the tasks stay inside their regions, every slot is written once, the tasks read exactly what the
nodes write and write exactly what they read, and the 8-byte accesses are aligned.  The constants
are parsed from the kernel source, so a change there is checked before it runs on a GPU.  The
double-buffered phase schedule of picard_pt and the trace stores of the final stage
(predictor_final_pt) are replayed as well."""
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_06889_gb300", "csrc")


def model():
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("pencil_layout_model", os.path.join(here, "pencil_layout_model.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def table():
    src = open(os.path.join(CSRC, "adg_kernels.cuh")).read()
    rows = re.findall(r"\(D == (\d) && n == (\d+) && ncmb == (\d+)\)\s*\?\s*PtLayout\{(\d+), (\d+), (\d+), (\d+)\}", src)
    return {(int(D), int(n), int(c)): tuple(int(x) for x in (a, b, ms, cs)) for D, n, c, a, b, ms, cs in rows}


M = model()
TABLE = table()


def test_table_covers_the_built_configurations():
    keys = {(c.D, c.n, c.NC) for c in M.CONFIGS}
    assert keys <= set(TABLE), keys - set(TABLE)


@pytest.mark.parametrize("cfg", M.CONFIGS, ids=[c.name for c in M.CONFIGS])
def test_layout_indices(cfg):
    assert cfg.check(TABLE[(cfg.D, cfg.n, cfg.NC)])


@pytest.mark.parametrize("cfg", M.CONFIGS, ids=[c.name for c in M.CONFIGS])
def test_table_holds_the_models_best_layout(cfg):
    # the kernel's constants reach the fewest modelled wavefronts of the search space (ties allowed)
    best, _ = cfg.search()
    assert cfg.count(TABLE[(cfg.D, cfg.n, cfg.NC)]) == best


@pytest.mark.parametrize("cfg", M.CONFIGS, ids=[c.name for c in M.CONFIGS])
def test_final_stage_traces(cfg):
    assert cfg.check_final(TABLE[(cfg.D, cfg.n, cfg.NC)])


@pytest.mark.parametrize("cfg", M.CONFIGS, ids=[c.name for c in M.CONFIGS])
def test_default_layout_indices(cfg):
    NP, n = cfg.NP, cfg.n
    assert cfg.check((0, 0, NP + 2, ((n - 1) * (NP + 2) + NP + 3) // 4 * 4))


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("iters", [1, 2, 3, 7])
def test_pipelined_schedule(n, iters):
    # every read sees its slice; n + 1 barriers per sweep after the first (which takes 2)
    assert M.check_schedule(n, iters) == 2 + (iters - 1) * (n + 1)


def test_a_wrong_stride_is_caught():
    cfg = [c for c in M.CONFIGS if c.name == "Euler 3D N=5"][0]
    with pytest.raises(AssertionError):
        cfg.check((1, 1, 30, 228))  # MS below NP: positions of two pencils overlap
