"""Layout constants of the pencil-task Picard sweep (pt_layout in adg_kernels.cuh), replayed on the
CPU: for every configuration the library builds, the shared-memory indices of the node threads and
of the tasks stay inside their regions, every slot is written once, the tasks read exactly what the
nodes write and write exactly what they read, and the 8-byte accesses are aligned.  The constants
are parsed from the kernel source, so a change there is checked before it runs on a GPU; so is
the thread orders of the 3D Euler N=5 nodes and x tasks (kNodeOrderEuler3N5,
kXTaskOrderEuler3N5).  The double-buffered phase
schedule of picard_pt and the trace stores of the final stage
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


def node_order_words():
    src = open(os.path.join(CSRC, "adg_kernels.cuh")).read()
    body = re.search(r"kNodeOrderEuler3N5\[(\d+)\] = \{([^}]*)\}", src)
    words = [int(w, 16) for w in re.findall(r"0x([0-9a-f]+)u", body.group(2))]
    assert len(words) == int(body.group(1))
    return words


def kernel_node_order(cfg):
    # node_of_thread: thread 32 w + l takes node l + 32 K, K the bits l of words 3 w .. 3 w + 2
    words = node_order_words()
    order = []
    for t in range(cfg.NS):
        w, l = t // 32, t % 32
        K = sum(((words[3 * w + b] >> l) & 1) << b for b in range(3))
        order.append(l + 32 * K)
    return order


def test_node_order_is_a_conflict_free_permutation():
    # the kernel's thread order of the 3D Euler N=5 nodes: every node once, and every warp's node
    # accesses in 32 distinct banks in all three directions (7 wavefronts per flux component)
    cfg = [c for c in M.CONFIGS if c.name == "Euler 3D N=5"][0]
    lay = TABLE[(cfg.D, cfg.n, cfg.NC)]
    order = kernel_node_order(cfg)
    assert sorted(order) == list(range(cfg.NS))
    assert len(node_order_words()) == 3 * ((cfg.NS + 31) // 32)
    assert cfg.count_nodes(lay) == 135  # the natural order: the y accesses meet on banks
    assert cfg.count_nodes(lay, order) == cfg.NC * ((cfg.NS + 31) // 32) == 105
    assert cfg.count(lay, order) == 444 and cfg.count(lay) == 504


def test_node_order_construction():
    # node_order of the model rebuilds a conflict-free order from the layout alone; the
    # configurations whose offsets it cannot handle keep the natural order
    cfg = [c for c in M.CONFIGS if c.name == "Euler 3D N=5"][0]
    lay = TABLE[(cfg.D, cfg.n, cfg.NC)]
    order = cfg.node_order(lay)
    assert sorted(order) == list(range(cfg.NS)) and all(order[t] % 32 == t % 32 for t in range(cfg.NS))
    assert cfg.count_nodes(lay, order) == 105
    assert order == kernel_node_order(cfg)
    assert cfg.node_order((1, 1, 38, 228)) is None  # y offsets with 8 nodes on some banks


def x_task_order_table():
    src = open(os.path.join(CSRC, "adg_kernels.cuh")).read()
    body = re.search(r"kXTaskOrderEuler3N5\[(\d+)\] = \{([^}]*)\}", src)
    vals = [int(v) for v in re.findall(r"\d+", body.group(2))]
    assert len(vals) == int(body.group(1))
    return vals


def test_x_task_order_is_a_conflict_free_permutation():
    # the kernel's thread order of the 3D Euler N=5 x tasks: every task once, the index
    # arithmetic and the trace stores still exact, and with the node order the fewest wavefronts
    # for 7 warps of nodes and 6 of tasks per direction
    cfg = [c for c in M.CONFIGS if c.name == "Euler 3D N=5"][0]
    lay = TABLE[(cfg.D, cfg.n, cfg.NC)]
    xorder = x_task_order_table()
    assert sorted(xorder) == list(range(cfg.dir_of.count(0) * cfg.NP))
    assert xorder == cfg.x_task_order(lay)
    assert cfg.check(lay, xorder) and cfg.check_final(lay, xorder)
    order = kernel_node_order(cfg)
    assert cfg.count(lay, order, xorder) == 426 == 2 * (cfg.NC * 7 + 3 * 6 * 6)
    assert cfg.count(lay, None, xorder) == 486  # the x task order alone


def test_a_wrong_stride_is_caught():
    cfg = [c for c in M.CONFIGS if c.name == "Euler 3D N=5"][0]
    with pytest.raises(AssertionError):
        cfg.check((1, 1, 30, 228))  # MS below NP: positions of two pencils overlap
