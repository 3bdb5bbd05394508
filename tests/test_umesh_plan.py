"""The library's host plan for unstructured meshes (C ABI, no GPU) against the
oracle: edges, partitions and macro-edges must agree exactly (integer
decisions taken from the same fp64 comparisons)."""
import numpy as np
import pytest

from oracle import unstructured as U
from paper_1811_09909_gb300 import workloads as W

um = pytest.importorskip("paper_1811_09909_gb300.umesh")


@pytest.fixture(scope="module", autouse=True)
def _library():
    """Build the library if it is missing (host compilation only)."""
    import os
    from paper_1811_09909_gb300 import build, hdgmg
    if not os.path.exists(hdgmg.LIB_PATH):
        build.build()





@pytest.mark.parametrize("n,seeds", [(4, 7), (6, 4), (10, 7)])
def test_plan_matches_oracle_hierarchy(n, seeds):
    v, q, sp, _, _ = W.example2(n, 2, seeds=seeds)
    pl = um.Plan(v, q, 2, 1.0, sp)
    ev, _, _ = U.mesh_edges(q)
    assert np.array_equal(pl.edges(), ev)
    parts, levels = U.hierarchy_chains(v, q, sp)
    assert pl.n_parts == len(parts)
    for r, part in enumerate(parts):
        assert np.array_equal(pl.partition(r), part)
    for t, lev in enumerate(levels):
        info, items = pl.macro_edges(t)
        ch = lev["units"]
        assert len(info) == len(ch)
        for c, x in enumerate(ch):
            assert tuple(info[c, :5]) == (x.sides[0], x.sides[1], x.start, x.end, int(x.closed))
            o, m = info[c, 5], len(x.edges)
            assert np.array_equal(items[o:o + m, 0], x.edges)
            assert np.array_equal(items[o:o + m, 1], x.edirs)
    assert pl.n_levels == len(levels) + 1         # P_2 mesh, P_1 mesh, then the partitions
    free = np.sum(U.mesh_edges(q)[2][:, 1] >= 0)
    assert pl.trace_dofs == free * 3


def test_plan_on_uniform_grid_is_the_block_agglomeration():
    n = 8
    xs = np.arange(n + 1) / n
    verts = np.array([(x, y) for y in xs for x in xs])
    quads = np.array([(j * (n + 1) + i, j * (n + 1) + i + 1, (j + 1) * (n + 1) + i + 1, (j + 1) * (n + 1) + i)
                      for j in range(n) for i in range(n)])
    seeds = np.array([[0.25, 0.25], [0.75, 0.25], [0.25, 0.75], [0.75, 0.75]])
    pl = um.Plan(verts, quads, 1, 1.0, seeds)
    c = U.centroids(verts, quads)
    assert pl.n_parts == 2
    assert np.array_equal(pl.partition(0), (c[:, 0] > 0.5) + 2 * (c[:, 1] > 0.5))
    info, items = pl.macro_edges(2)          # P_0: 4 interior straight macro-edges of 4 mesh edges
    interior = info[info[:, 1] >= 0]
    assert len(interior) == 4 and not interior[:, 4].any()
    sizes = np.diff(np.append(info[:, 5], len(items)))
    assert np.all(sizes[info[:, 1] >= 0] == 4)


@pytest.mark.parametrize("bad", ["clockwise", "index", "p", "tau", "seeds"])
def test_plan_rejects_invalid_problems(bad):
    from paper_1811_09909_gb300 import hdgmg
    v, q = W.umesh(3, 3, 1.0, 1.0, 0.2, (), 1)
    p, tau, seeds = 2, 1.0, np.array([[0.5, 0.5]])
    if bad == "clockwise":
        q = q.copy()
        q[3] = q[3][::-1]
    elif bad == "index":
        q = q.copy()
        q[0, 0] = len(v)
    elif bad == "p":
        p = 9
    elif bad == "tau":
        tau = 0.0
    else:
        seeds = np.zeros((0, 2))
    with pytest.raises(hdgmg.HdgmgError) as ei:
        um.Plan(v, q, p, tau, seeds)
    assert ei.value.status == -1
