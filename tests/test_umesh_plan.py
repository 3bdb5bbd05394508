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


@pytest.mark.parametrize("bad", ["clockwise", "index", "p", "tau", "seeds", "empty", "nonconforming",
                                 "degenerate"])
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
    elif bad == "empty":
        q = q[:0]
    elif bad == "nonconforming":
        q = np.concatenate([q, q[:1]])               # a second copy of element 0: three sides per edge
    elif bad == "degenerate":
        v = v.copy()
        v[q[2, 1]] = v[q[2, 0]]                     # a zero-length edge
    else:
        seeds = np.zeros((0, 2))
    with pytest.raises(hdgmg.HdgmgError) as ei:
        um.Plan(v, q, p, tau, seeds)
    assert ei.value.status == -1


def test_plan_edge_cases():
    """One element (no interior edge), one seed, and four elements around one
    vertex: sizes, partitions and macro-edges as worked by hand."""
    verts = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    pl = um.Plan(verts, np.array([[0, 1, 2, 3]]), 2, 1.0, np.array([[0.5, 0.5]]))
    assert (pl.n_edges, pl.n_parts, pl.trace_dofs) == (4, 1, 0)
    info, items = pl.macro_edges(1)                 # P_0 = the element: one cycle around it
    assert len(info) == 1 and info[0, 1] == -1 and info[0, 4] == 1 and len(items) == 4
    # 2 x 2 elements, one seed: P_0 holds all four; no cut partition has <= 2 macro-elements
    xs = np.array([0.0, 0.5, 1.0])
    v = np.array([(x, y) for y in xs for x in xs])
    q = np.array([(0, 1, 4, 3), (1, 2, 5, 4), (3, 4, 7, 6), (4, 5, 8, 7)])
    pl = um.Plan(v, q, 1, 1.0, np.array([[0.3, 0.3]]))
    assert pl.n_parts == 1 and np.all(pl.partition(0) == 0)
    assert pl.trace_dofs == 4 * 2                  # the four interior edges, P_1
    info, _ = pl.macro_edges(1)
    assert len(info) == 1 and info[0, 1] == -1     # only the outer boundary
    # two seeds splitting the square left / right: one interior macro-edge of two mesh edges
    pl = um.Plan(v, q, 1, 1.0, np.array([[0.25, 0.5], [0.75, 0.5]]))
    info, items = pl.macro_edges(1)
    inner = info[info[:, 1] >= 0]
    assert len(inner) == 1 and not inner[0, 4]
    o = inner[0, 5]
    assert sorted(items[o:o + 2, 0].tolist()) == sorted(
        [i for i, (a, b) in enumerate(pl.edges().tolist()) if {a, b} in ({1, 4}, {4, 7})])
    assert inner[0, 2] == 1 and inner[0, 3] == 7    # starts at the lower free end


@pytest.mark.parametrize("field,value", [("krylov", 2), ("precision", 3), ("precision", 2), ("smoother", 1), ("m_fine", 0),
                                         ("omega", 0.0), ("local_corr", 7)])
def test_create_rejects_unsupported_options_before_touching_the_gpu(field, value):
    import ctypes
    from paper_1811_09909_gb300 import hdgmg
    lib = um.load()
    v, q = W.umesh(2, 2, 1.0, 1.0, 0.2, (), 1)
    pr = um._Problem(v, q, 2, 1.0, np.array([[0.5, 0.5]]))
    o = hdgmg.Opts()
    lib.hdgmg_umesh_default_opts(ctypes.byref(o))
    assert (o.omega, o.m_fine, o.m_max) == (0.8, 2, 4)
    setattr(o, field, value)
    h = ctypes.c_void_p()
    st = lib.hdgmg_umesh_create(ctypes.byref(h), ctypes.byref(pr.s), ctypes.byref(o), None)
    assert st == -1 and not h


@pytest.mark.parametrize("case", range(6))
def test_plan_matches_oracle_on_random_meshes(case):
    """Random jittered meshes (with and without holes) and random seed sets:
    the library's partitions and macro-edges equal the oracle's exactly."""
    rng = np.random.default_rng(100 + case)
    nx, ny = int(rng.integers(3, 9)), int(rng.integers(3, 7))
    holes = ((0.5, 0.5, 0.15),) if case % 2 else ()
    v, q = W.umesh(nx, ny, 1.0, 1.0, 0.25, holes, int(rng.integers(0, 1000)))
    seeds = rng.uniform(0.0, 1.0, size=(int(rng.integers(1, 9)), 2))
    pl = um.Plan(v, q, 1 + case % 3, 1.0, seeds)
    parts, levels = U.hierarchy_chains(v, q, seeds)
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
