"""GPU parity of the unstructured-mesh path (hdgmg_umesh_*) against the
oracle (oracle/unstructured.py): element operators, every coarse level, the
V-cycle, PCG and fixed-point iteration counts, the solution and its
recovery, at sizes spanning several macro-elements and ragged ones (holes,
cycles, single-element macro-elements)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unstructured as U
from paper_1811_09909_gb300 import hdgmg, umesh as um, workloads as W

TOL = 1e-10          # FP64, different summation orders: relative to the operator's scale
# the unstructured defaults (hdgmg_umesh_default_opts), passed to the oracle
SMOOTH = dict(omega=0.8, m_fine=2, m_max=4)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _setup(n, p, seeds=7, kappa_sigma=0.0, **opts):
    v, q, sp, logk, f = W.example2(n, p, seeds=seeds)
    if kappa_sigma:
        logk = np.random.default_rng(11).normal(0, kappa_sigma, len(q))
    s = um.USolver(v, q, p, 1.0, sp, **opts)
    s.setup(_dev(logk))
    pr = U.UHDGProblem(v, q, p, np.exp(logk), 1.0)
    return s, pr, sp, f


def _dense(s, level):
    A, dofs = s.element_matrices(level)
    A = A.cpu().numpy()
    n = s.level_sizes(level)[0]
    M = np.zeros((n, n))
    for e in range(A.shape[0]):
        d = dofs[e]
        ok = d >= 0
        M[np.ix_(d[ok], d[ok])] += A[e][np.ix_(ok, ok)]
    return M


@pytest.mark.parametrize("p", [1, 2, 4])
def test_element_operators_and_levels_match_oracle(p):
    s, pr, sp, _ = _setup(4, p, kappa_sigma=1.0)
    Ae, _ = pr.condense()
    A, dofs = s.element_matrices(0)
    A = A.cpu().numpy()
    scale = np.abs(Ae).max()
    assert np.abs(A - Ae).max() < TOL * scale
    hu = U.UHierarchy(pr, sp, Ae=Ae, local_corr="both")
    assert s.n_levels == len(hu.levels)
    for k, L in enumerate(hu.levels):
        M = _dense(s, k)
        ref = L.A.toarray()
        assert M.shape == ref.shape, k
        assert np.abs(M - ref).max() < TOL * np.abs(ref).max(), k


@pytest.mark.parametrize("p,lc", [(2, "both"), (3, "pre"), (1, "both")])
def test_vcycle_matches_oracle(p, lc):
    om = 0.8 if p == 1 else 1.0
    s, pr, sp, _ = _setup(4, p, kappa_sigma=0.5, omega=om, local_corr=hdgmg.LC_BOTH if lc == "both" else hdgmg.LC_PRE,
                          m_fine=1, m_growth=2, m_max=4)
    hu = U.UHierarchy(pr, sp, local_corr=lc, omega=om, m_fine=1, m_growth=2, m_max=4)
    r = np.random.default_rng(5).normal(size=hu.levels[0].A.shape[0])
    z = s.vcycle(_dev(r)).cpu().numpy()
    zo = hu.vcycle(r)
    assert np.abs(z - zo).max() < 1e-9 * np.abs(zo).max()


@pytest.mark.parametrize("p", [1, 3])
def test_pcg_solve_and_recovery_match_oracle(p):
    s, pr, sp, f = _setup(5, p, kappa_sigma=1.0, rtol=1e-11)
    lam, u, q, info = s.solve(_dev(f))
    assert info.converged and info.rel_res <= 1e-11
    lam_o = pr.solve_direct(f)
    lam = lam.cpu().numpy().ravel()
    assert np.abs(lam - lam_o).max() < 1e-8 * np.abs(lam_o).max()
    u_o, q_o = pr.recover(lam_o, f)
    assert np.abs(u.cpu().numpy() - u_o).max() < 1e-8 * np.abs(u_o).max()
    assert np.abs(q.cpu().numpy() - q_o).max() < 1e-7 * np.abs(q_o).max()
    Ae, ge = pr.condense(f)
    b = pr.assemble_rhs(ge)[pr.free_dofs()]
    hu = U.UHierarchy(pr, sp, Ae=Ae, local_corr="both", **SMOOTH)
    _, it, _, ok = hu.solve_pcg(b, tol=1e-11)
    assert ok and abs(info.iters - it) <= 1, (info.iters, it)


def test_fixed_point_iterations_match_oracle():
    s, pr, sp, f = _setup(4, 2, krylov=hdgmg.KRYLOV_NONE, local_corr=hdgmg.LC_PRE, rtol=1e-9)
    lam, _, _, info = s.solve(_dev(f), want_u=False, want_q=False)
    Ae, ge = pr.condense(f)
    b = pr.assemble_rhs(ge)[pr.free_dofs()]
    hu = U.UHierarchy(pr, sp, Ae=Ae, local_corr="pre", **SMOOTH)
    _, it, _, ok = hu.solve_fixed_point(b, tol=1e-9)
    assert ok and info.converged and abs(info.iters - it) <= 1, (info.iters, it)


def test_four_seed_strategy_and_single_seed():
    for seeds in (4,):
        s, pr, sp, f = _setup(4, 2, seeds=seeds)
        lam, _, _, info = s.solve(_dev(f), want_u=False, want_q=False)
        assert info.converged
        assert np.abs(lam.cpu().numpy().ravel() - pr.solve_direct(f)).max() < 1e-8
    v, q = W.umesh(3, 3, 1.0, 1.0, 0.2, (), 2)
    s = um.USolver(v, q, 2, 1.0, np.array([[0.5, 0.5]]))
    s.setup(_dev(np.zeros(len(q))))
    f = np.ones((len(q), 9))
    lam, _, _, info = s.solve(_dev(f))
    pr = U.UHDGProblem(v, q, 2, 1.0, 1.0)
    assert info.converged
    assert np.abs(lam.cpu().numpy().ravel() - pr.solve_direct(f)).max() < 1e-8


def test_large_mesh_sampled_elements_and_convergence():
    """About 27k elements (n = 48): sampled element operators (random kappa)
    against the oracle one by one; then Example II's kappa = 1, f = 1 solve:
    converged with the true residual, the oracle's trace equations satisfied
    on sampled interior edges (sum over the edge's two elements of
    A_e lambda_e - g_e, each element condensed by the oracle), and the
    recovered u, q equal to the oracle's local solves on sampled elements."""
    v, q, sp, logk1, f = W.example2(48, 3)
    logk = np.random.default_rng(2).normal(0, 1.0, len(q))
    s = um.USolver(v, q, 3, 1.0, sp, rtol=1e-10)
    s.setup(_dev(logk))
    pr = U.UHDGProblem(v, q, 3, np.exp(logk), 1.0)
    A = s.element_matrices(0)[0]
    rng = np.random.default_rng(0)
    for e in rng.choice(len(q), 12, replace=False):
        Ao = pr.element_operator(int(e))
        assert np.abs(A[int(e)].cpu().numpy() - Ao).max() < TOL * np.abs(Ao).max()
    s.setup(_dev(logk1))
    lam, u, qq, info = s.solve(_dev(f))
    assert info.converged and info.rel_res <= 1e-10 and info.iters < 200, info.iters
    pr1 = U.UHDGProblem(v, q, 3, 1.0, 1.0)
    lam = lam.cpu().numpy().ravel()
    dofs = pr1.element_dofs()
    nd = 4
    interior = np.nonzero(pr1.edge_elems[:, 1] >= 0)[0]
    gscale = 0.0
    for m in rng.choice(interior, 10, replace=False):
        res = np.zeros(nd)
        for e in pr1.edge_elems[m]:
            Ae, ge = pr1.element_operator(int(e), f)
            j = list(pr1.edges[e]).index(m)
            sl = slice(j * nd, (j + 1) * nd)
            res += (Ae @ lam[dofs[e]] - ge)[sl]
            gscale = max(gscale, np.abs(ge).max())
        assert np.abs(res).max() < 1e-8 * gscale, (m, res)
    u, qq = u.cpu().numpy(), qq.cpu().numpy()
    nv = pr1.nv
    for e in rng.choice(len(q), 10, replace=False):
        fr = pr1.forms(int(e))
        L, R, _ = fr.local(1.0, 1.0)
        z = np.linalg.solve(L, fr.load(f[e]) - R @ lam[dofs[e]])
        assert np.abs(u[e] - z[2 * nv:]).max() < 1e-9 * np.abs(z[2 * nv:]).max()
        assert np.abs(qq[e, 0] - z[:nv]).max() < 1e-8 * np.abs(z[:2 * nv]).max()
        assert np.abs(qq[e, 1] - z[nv:2 * nv]).max() < 1e-8 * np.abs(z[:2 * nv]).max()


def test_invalid_options_are_rejected():
    v, q, sp, _, _ = W.example2(3, 2)
    for kw in ({"krylov": hdgmg.KRYLOV_GMRES}, {"precision": hdgmg.PREC_BF16},
               {"precision": hdgmg.PREC_FP32_IR}, {"smoother": hdgmg.SMOOTH_POINT_JACOBI}):
        with pytest.raises(hdgmg.HdgmgError) as ei:
            um.USolver(v, q, 2, 1.0, sp, **kw)
        assert ei.value.status == -1


def test_breakdown_on_nan_kappa():
    v, q, sp, logk, f = W.example2(3, 2)
    s = um.USolver(v, q, 2, 1.0, sp)
    logk = logk.copy()
    logk[5] = np.nan
    with pytest.raises(hdgmg.HdgmgError) as ei:
        s.setup(_dev(logk))
    assert ei.value.status == -5


def test_fp32_cycle_inside_fp64_pcg():
    """PREC_FP32: the V-cycle on FP32 copies of every level, inside the FP64
    PCG.  One cycle within 1e-4 of the FP64 cycle (FP32 rounding amplified by
    the level conditioning); the solve reaches the same FP64 residual target
    with at most two more iterations and the oracle's solution."""
    v, q, sp, logk, f = W.example2(5, 3)
    s64 = um.USolver(v, q, 3, 1.0, sp, rtol=1e-10)
    s32 = um.USolver(v, q, 3, 1.0, sp, rtol=1e-10, precision=hdgmg.PREC_FP32)
    for s in (s64, s32):
        s.setup(_dev(logk))
    r = _dev(np.random.default_rng(8).normal(size=s64.level_sizes(0)[0]))
    z64, z32 = s64.vcycle(r), s32.vcycle(r)
    rel = float(torch.linalg.norm(z32 - z64) / torch.linalg.norm(z64))
    assert 0.0 < rel < 1e-4, rel
    lam64, _, _, i64 = s64.solve(_dev(f), want_u=False, want_q=False)
    lam32, _, _, i32 = s32.solve(_dev(f), want_u=False, want_q=False)
    assert i64.converged and i32.converged and i32.rel_res <= 1e-10
    assert i32.iters <= i64.iters + 2, (i32.iters, i64.iters)
    pr = U.UHDGProblem(v, q, 3, 1.0, 1.0)
    lam_o = pr.solve_direct(f)
    assert np.abs(lam32.cpu().numpy().ravel() - lam_o).max() < 1e-8 * np.abs(lam_o).max()


@pytest.mark.parametrize("p", [5, 6])
def test_higher_orders_element_operators_and_solve(p):
    """p = 5, 6: element operators against the oracle and a PCG solve against
    its direct solve on the Example II stand-in at n = 3."""
    s, pr, sp, f = _setup(3, p, kappa_sigma=0.5, rtol=1e-11)
    A = s.element_matrices(0)[0].cpu().numpy()
    for e in (0, 17, len(pr.quads) - 1):
        Ao = pr.element_operator(e)
        assert np.abs(A[e] - Ao).max() < TOL * np.abs(Ao).max()
    lam, _, _, info = s.solve(_dev(f), want_u=False, want_q=False)
    assert info.converged
    lam_o = pr.solve_direct(f)
    assert np.abs(lam.cpu().numpy().ravel() - lam_o).max() < 1e-8 * np.abs(lam_o).max()


def test_mesh_without_interior_edges():
    """One element: no trace unknowns; the solve is the local solve with
    lambda = 0 on the boundary, recovered u equal to the oracle's."""
    verts = np.array([[0, 0], [1, 0], [1.2, 1], [0, 0.8]], float)
    quads = np.array([[0, 1, 2, 3]])
    s = um.USolver(verts, quads, 2, 1.0, np.array([[0.5, 0.5]]))
    s.setup(_dev(np.zeros(1)))
    f = np.ones((1, 9))
    lam, u, q, info = s.solve(_dev(f))
    assert info.converged and info.iters == 0
    assert float(lam.abs().max()) == 0.0
    pr = U.UHDGProblem(verts, quads, 2, 1.0, 1.0)
    u_o, q_o = pr.recover(np.zeros(pr.ne * 3), f)
    assert np.abs(u.cpu().numpy() - u_o).max() < 1e-10 * np.abs(u_o).max()
    assert np.abs(q.cpu().numpy() - q_o).max() < 1e-9 * np.abs(q_o).max()
