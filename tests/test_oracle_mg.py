"""Pins of the oracle's multigrid hierarchy and V-cycle (Sec. 3, Sec. 4.1).

The hierarchy is checked against a dense global Schur complement with a
hand-derived injection (Proposition "DtN"), against the traces of linear
functions (which every DtN level must map to zero flux on interior edges),
against the energy identity, and the V-cycle against the iteration counts the
paper prints for Example I (tests/golden/paper_example1_iterations.txt)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import hdg, mg
from paper_1811_09909_gb300 import workloads as W
from conftest import load_paper_table

# child injection P1(macro) -> P1(half), worked by hand in the orthonormal
# Legendre basis: [child][fine mode][coarse mode]
_R2 = math.sqrt(2.0)
_JC = np.array([[[1 / _R2, -math.sqrt(3) / (2 * _R2)], [0.0, 1 / (2 * _R2)]],
                [[1 / _R2, +math.sqrt(3) / (2 * _R2)], [0.0, 1 / (2 * _R2)]]])


def _hier(n, p, seed, **kw):
    rng = np.random.default_rng(seed)
    pr = hdg.HDGProblem(n, p, np.exp(rng.normal(size=n * n)), rng.uniform(1, 4) * n)
    return pr, mg.Hierarchy(pr, **kw)


def test_child_injection_closed_form():
    assert np.abs(mg.child_injection() - _JC).max() < 1e-14


def _edge_class(n):
    """fine edge -> (is_interior_of_macro, coarse edge, child) from geometry."""
    nvf = n * (n + 1)
    nc = n // 2
    nvc = nc * (nc + 1)
    out = []
    for e in range(hdg.n_edges(n)):
        if e < nvf:
            j, i = divmod(e, n + 1)
            out.append((i % 2 == 1, (j // 2) * (nc + 1) + i // 2, j % 2))
        else:
            j, i = divmod(e - nvf, n)
            out.append((j % 2 == 1, nvc + (j // 2) * nc + i // 2, i % 2))
    return out


@pytest.mark.parametrize("n,p", [(8, 1), (8, 2), (8, 3)])
def test_coarse_operator_is_dense_schur_complement(n, p):
    """Eq. Akm1 / Proposition DtN: A_{k-1} = J^T (A_BB - A_BI A_II^-1 A_IB) J,
    with A_II^-1 by a dense global solve and J from the closed form above."""
    pr, Hh = _hier(n, p, 5, coarsest_n=2)
    first_h = 1 if p > 1 else 0
    for k in range(first_h, len(Hh.levels) - 1):
        L, Lc = Hh.levels[k], Hh.levels[k + 1]
        A = L.A.toarray()
        cls = _edge_class(L.n)
        fe = L.free // 2
        Iset = np.array([i for i, e in enumerate(fe) if cls[e][0]])
        Bset = np.array([i for i, e in enumerate(fe) if not cls[e][0]])
        cpos = {d: i for i, d in enumerate(Lc.free)}
        J = np.zeros((len(Bset), len(Lc.free)))
        for r, b in enumerate(Bset):
            e, l = divmod(L.free[b], 2)
            _, ce, c = cls[e]
            for kk in range(2):
                if ce * 2 + kk in cpos:
                    J[r, cpos[ce * 2 + kk]] = _JC[c, l, kk]
        S = A[np.ix_(Bset, Bset)] - A[np.ix_(Bset, Iset)] @ np.linalg.solve(
            A[np.ix_(Iset, Iset)], A[np.ix_(Iset, Bset)])
        ref = J.T @ S @ J
        assert np.abs(Lc.A.toarray() - ref).max() < 1e-10 * np.abs(ref).max()


def _linear_trace(n, fun):
    """Orthonormal P1 coefficients of fun on every edge of an n x n mesh of
    the unit square, edge-major [n_edges*2]."""
    s, w = npleg.leggauss(4)
    h = 1.0 / n
    sc = np.sqrt(np.array([1.0, 3.0]) / h)[:, None]
    P = np.stack([np.ones_like(s), s]) * sc
    out = np.zeros((hdg.n_edges(n), 2))
    nv = n * (n + 1)
    for j in range(n):
        for i in range(n + 1):
            out[j * (n + 1) + i] = P @ (w * fun(i * h + 0 * s, (j + 0.5 + 0.5 * s) * h)) * h / 2
    for j in range(n + 1):
        for i in range(n):
            out[nv + j * n + i] = P @ (w * fun((i + 0.5 + 0.5 * s) * h, j * h + 0 * s)) * h / 2
    return out.ravel()


@pytest.mark.parametrize("p", [1, 3])
def test_every_level_annihilates_linear_traces(p):
    """A linear u is harmonic and reproduced by HDG, so its DtN image has zero
    net flux across every interior edge: A_k l_k = 0 on rows of interior edges
    at every P1 level (Neumann operators, boundary edges kept).  A wrong
    injection J breaks this on the first coarse level."""
    n = 16
    rng = np.random.default_rng(1)
    pr = hdg.HDGProblem(n, p, 2.5, 3.0 * n)
    Hh = mg.Hierarchy(pr, coarsest_n=2, dirichlet=False)
    fun = lambda x, y: 0.3 + 1.7 * x - 2.2 * y
    for L in Hh.levels:
        if L.nd != 2:
            continue
        lin = _linear_trace(L.n, fun)
        y = L.A @ lin[L.free]
        interior = ~hdg.boundary_edge_mask(L.n)[L.free // 2]
        assert np.abs(y[interior]).max() < 1e-10 * np.abs(L.A).max(), L.n


@pytest.mark.parametrize("p", [1, 2])
def test_energy_preservation_and_adjointness(p):
    """Proposition "Energy preservation": a_k(I_k l, I_k l) = a_{k-1}(l, l);
    and Q_{k-1} = I_k^T for symmetric A (remark after eq. n_g1_Qk)."""
    pr, Hh = _hier(8, p, 9, coarsest_n=2)
    rng = np.random.default_rng(0)
    for k in range(len(Hh.levels) - 1):
        L, Lc = Hh.levels[k], Hh.levels[k + 1]
        lam = rng.normal(size=Lc.A.shape[0])
        v = L.I @ lam
        assert abs(v @ (L.A @ v) - lam @ (Lc.A @ lam)) < 1e-10 * abs(lam @ (Lc.A @ lam))
        assert abs(L.Q - L.I.T).max() < 1e-12 * abs(L.Q).max()


def test_symmetric_vcycle_is_symmetric_positive():
    pr, Hh = _hier(8, 2, 2, coarsest_n=2, local_corr="both")
    rng = np.random.default_rng(4)
    nf = Hh.levels[0].A.shape[0]
    V = rng.normal(size=(nf, 3))
    B = np.stack([Hh.vcycle(V[:, i]) for i in range(3)], axis=1)
    G = V.T @ B
    assert np.abs(G - G.T).max() < 1e-10 * np.abs(G).max()
    assert np.linalg.eigvalsh(0.5 * (G + G.T)).min() > 0


def _counts(p, L, tau_mode, local_corr, m_fine=3, smoother="block_jacobi", omega=1.0):
    n = 2 ** L
    wl = W.example1(n, p, tau_mode=tau_mode)
    pr = hdg.HDGProblem(n, p, 1.0, wl.tau())
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    Hh = mg.Hierarchy(pr, coarsest_n=2, m_fine=m_fine, m_growth=2, local_corr=local_corr,
                      smoother=smoother, omega=omega)
    _, it, _, ok = Hh.solve_fixed_point(bf, tol=1e-9)
    _, it2, _, ok2 = Hh.solve_gmres(bf, tol=1e-9, left=True)
    return (it if ok else None), (it2 if ok2 else None)


@pytest.mark.parametrize("section,tau_mode,ps", [
    ("hdg_tau_over_h_block_jacobi", "over_h", (1, 2, 4)),
    ("hdg_tau_one_block_jacobi", "const", (1, 2)),
])
def test_iteration_counts_match_paper_tables(section, tau_mode, ps):
    """Example I (Sec. 4.1): MG-as-solver and MG-GMRES counts at levels 2-4
    within max(1, 15%) of the printed tables (m_N = 3, beta = 2, local
    correction in step 3 only, tolerance 1e-9)."""
    table = load_paper_table(section)
    for p in ps:
        for L in (2, 3, 4):
            ours = _counts(p, L, tau_mode, "pre")
            ref = (table[p][0][L - 2], table[p][1][L - 2])
            for o, r in zip(ours, ref):
                assert o is not None and abs(o - r) <= max(1, 0.15 * r), (p, L, ours, ref)


def test_lu_sgs_counts_match_paper_table():
    """LU-SGS smoother (one forward and one backward point Gauss-Seidel sweep
    per step, multicolour edge order): Example I counts at levels 2-4 within
    max(1, 15%) of the printed table, as solver and with GMRES."""
    table = load_paper_table("hdg_tau_over_h_lu_sgs")
    for p in (1, 2, 3, 4):
        for L in (2, 3, 4):
            ours = _counts(p, L, "over_h", "pre", smoother="lu_sgs")
            ref = (table[p][0][L - 2], table[p][1][L - 2])
            for o, r in zip(ours, ref):
                assert o is not None and abs(o - r) <= max(1, 0.15 * r), (p, L, ours, ref)


def test_smoother_ranking_and_h_independence():
    """The paper's comparison (Sec. 4.1): every smoother converges with
    h-independent counts; LU-SGS needs the fewest iterations and point-Jacobi
    the most.  The printed point-Jacobi and Chebyshev counts depend on the
    trace basis (Jacobi uses the diagonal of A, which changes with the basis;
    the paper does not state its basis) and are checked only loosely: within
    a factor 2 of the table at p = 1, 2, levels 3-5."""
    pj_t = load_paper_table("hdg_tau_over_h_point_jacobi")
    ch_t = load_paper_table("hdg_tau_over_h_chebyshev")
    for p in (1, 2):
        rows = {}
        for sm, om, tab in (("point_jacobi", 2.0 / 3.0, pj_t), ("chebyshev", 1.0, ch_t),
                            ("block_jacobi", 1.0, None), ("lu_sgs", 1.0, None)):
            levels = (3, 4, 5)
            c = [_counts(p, L, "over_h", "pre", m_fine=1, smoother=sm, omega=om) for L in levels]
            assert all(a is not None and b is not None for a, b in c), (sm, p, c)
            mgc = [a for a, _ in c]
            assert max(mgc) - min(mgc) <= max(2, 0.25 * max(mgc)), (sm, p, mgc)
            if tab is not None:
                for i, L in enumerate(levels):
                    assert 0.5 * tab[p][0][L - 2] <= mgc[i] <= 2 * tab[p][0][L - 2], (sm, p, mgc)
            rows[sm] = sum(mgc)
        assert rows["lu_sgs"] < rows["block_jacobi"] < rows["point_jacobi"], rows


def test_smoothers_are_symmetric_for_cg():
    """Point-Jacobi, Chebyshev and LU-SGS (symmetric sweep) keep the V-cycle
    with local correction in steps 3 and 5 symmetric and positive, so PCG
    converges with them (Sec. 3.6)."""
    n, p = 8, 2
    wl = W.example1(n, p)
    pr = hdg.HDGProblem(n, p, 1.0, wl.tau())
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    rng = np.random.default_rng(3)
    for sm, om in (("point_jacobi", 2.0 / 3.0), ("chebyshev", 1.0), ("lu_sgs", 1.0)):
        Hh = mg.Hierarchy(pr, coarsest_n=2, m_fine=2, local_corr="both", smoother=sm, omega=om)
        x, y = rng.standard_normal((2, len(bf)))
        bx, by = Hh.vcycle(x), Hh.vcycle(y)
        assert abs(y @ bx - x @ by) <= 1e-10 * abs(y @ bx), sm
        assert x @ bx > 0
        _, it, _, ok = Hh.solve_pcg(bf, tol=1e-10)
        assert ok and it < 40, (sm, it)


def test_no_local_correction_diverges_at_p1():
    """Table without local correction: p = 1 MG solver prints "*" at every
    level; with the correction it converges (Sec. 3.4, Sec. 4.1)."""
    table = load_paper_table("hdg_tau_over_h_block_jacobi_no_local_correction")
    assert table[1][0][:3] == [None, None, None]
    for L in (2, 3):
        mg_it, _ = _counts(1, L, "over_h", "none")
        assert mg_it is None
        mg_it, _ = _counts(1, L, "over_h", "pre")
        assert mg_it is not None


def test_h_independent_pcg_counts():
    """Flat counts as h shrinks (Sec. 4.1, tau = 1/h) for the symmetric
    V-cycle (local correction in steps 3 and 5) inside PCG."""
    its = []
    for n in (8, 16, 32, 64):
        wl = W.example1(n, 2)
        pr = hdg.HDGProblem(n, 2, 1.0, wl.tau())
        _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
        Hh = mg.Hierarchy(pr, coarsest_n=2, m_fine=1, local_corr="both")
        _, it, _, ok = Hh.solve_pcg(bf, tol=1e-10)
        assert ok
        its.append(it)
    assert max(its) - min(its) <= 2, its
