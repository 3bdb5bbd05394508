"""GPU parity of the convection-diffusion path (non-symmetric trace operator,
full storage, LU condensation, restriction from A_BI) against the oracle's
upwind HDG element and its multigrid, through the C ABI.

Tolerances:
  * element operators and right-hand sides: 1e-10 max|A| (GPU: LU without
    pivoting of the n_v block after q is eliminated; oracle: LU with partial
    pivoting of the full 3 n_v block -- two FP64 factorisations of matrices
    whose condition numbers reach ~1e5 at eps = 1e-3);
  * level operators and one FP64 V-cycle: 1e-10 relative (max norm);
  * solutions: relative residual of the oracle's own A, g <= 1.5 rtol and
    relative L2 error of lambda, u, q <= 1e-8 against the oracle's sparse
    direct solve (solves to 1e-12);
  * GMRES and fixed-point counts within one of the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

LC = {"none": hdgmg.LC_NONE, "pre": hdgmg.LC_PRE, "both": hdgmg.LC_BOTH}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def workload(n, p, eps, seed=None, beta=(1.0, 0.5)):
    """Manufactured convection-diffusion; with a seed, eps varies per element
    (log eps + N(0, 0.3^2)) and f is random."""
    wl = W.convdiff(n, p, eps=eps, beta=beta)
    if seed is not None:
        rng = np.random.default_rng(seed)
        wl.log_kappa = wl.log_kappa + rng.normal(0.0, 0.3, n * n)
        wl.f = rng.standard_normal(wl.f.shape)
    return wl


def solver(wl, **opts):
    opts.setdefault("krylov", hdgmg.KRYLOV_GMRES)
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=hdgmg.TAU_OVER_H, tau_c=wl.tau_c, beta=wl.beta, **opts)
    s.setup(cuda(wl.log_kappa))
    return s


def oracle(wl):
    return hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau(), beta=wl.beta)


@pytest.mark.parametrize("n,p,eps", [(4, 1, 1e-2), (8, 2, 1e-3), (4, 3, 0.1), (4, 4, 1e-3),
                                     (4, 6, 1e-3), (2, 8, 1e-2)])
def test_element_operators_match_oracle(n, p, eps):
    wl = workload(n, p, eps, seed=10 + p)
    s = solver(wl, coarsest_n=n)
    A = host(s.element_matrices(0))                          # [nl][nl][E]
    Ae, _ = oracle(wl).condense()
    ref = np.transpose(Ae, (1, 2, 0))
    assert np.abs(A - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(ref - np.transpose(ref, (1, 0, 2))).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("p", [1, 3])
def test_condensed_rhs_with_dirichlet_lift(p):
    n = 8
    wl = workload(n, p, 1e-2, seed=3)
    gD = W.dirichlet(lambda x, y: np.exp(x) * (1 + y), n, p)
    s = solver(wl)
    b = host(s.condensed_rhs(cuda(wl.f[0]), cuda(gD)))
    pr = oracle(wl)
    _, bf, *_ = pr.system(wl.f[0], gD)
    b_em = hdg.api_to_edge_major(b, n, p + 1)[pr.free_dofs()]
    assert np.abs(b_em - bf).max() <= 1e-10 * np.abs(bf).max()


@pytest.mark.parametrize("n,p", [(8, 1), (16, 2)])
def test_level_operators_match_oracle_hierarchy(n, p):
    wl = workload(n, p, 1e-2, seed=5)
    s = solver(wl, coarsest_n=2)
    H = mg.Hierarchy(oracle(wl), coarsest_n=2)
    rng = np.random.default_rng(1)
    assert s.num_levels() == len(H.levels)
    for k, L in enumerate(H.levels):
        x = rng.standard_normal((L.nd, hdg.n_edges(L.n)))
        y = host(s.apply_operator(k, cuda(x)))
        ref = H.from_free(L.A @ H.to_free(x, k), k)
        assert np.abs(y - ref).max() <= 1e-10 * np.abs(ref).max(), k


@pytest.mark.parametrize("n,p,lc,m,cn", [(8, 1, "pre", 1, 2), (16, 2, "both", 1, 2),
                                          (8, 3, "pre", 2, 2), (16, 2, "none", 2, 2),
                                          (8, 6, "pre", 1, 2), (16, 2, "pre", 1, 8)])
def test_vcycle_matches_oracle(n, p, lc, m, cn):
    """cn = 8: the coarsest operator (224 unknowns) is inverted by the
    global-memory Gauss-Jordan kernel instead of in shared memory."""
    wl = workload(n, p, 1e-3, seed=20 + p)
    s = solver(wl, coarsest_n=cn, m_fine=m, local_corr=LC[lc])
    H = mg.Hierarchy(oracle(wl), coarsest_n=cn, m_fine=m, local_corr=lc)
    rng = np.random.default_rng(7)
    r = rng.standard_normal((p + 1, hdg.n_edges(n)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert np.abs(e - ref).max() <= 1e-10 * np.abs(ref).max()


def test_fp32_vcycle_close_to_oracle():
    wl = workload(32, 4, 1e-3, seed=2)
    s = solver(wl, coarsest_n=4, m_max=4, precision=hdgmg.PREC_FP32)
    H = mg.Hierarchy(oracle(wl), coarsest_n=4, m_max=4, local_corr="both")
    rng = np.random.default_rng(8)
    r = rng.standard_normal((5, hdg.n_edges(32)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert rel_l2(e, ref) <= 1e-4


def _check_solution(wl, lam, u, q, rtol_res, gD=None):
    pr = oracle(wl)
    f = wl.f[0]
    Aff, bf, *_ = pr.system(f, gD)
    lam_f = hdg.api_to_edge_major(lam, wl.n, wl.p + 1)[pr.free_dofs()]
    res = np.linalg.norm(bf - Aff @ lam_f) / np.linalg.norm(bf)
    assert res <= 1.5 * rtol_res, res
    lam_ref = pr.solve_direct(f, gD)
    u_ref, q_ref = pr.recover(lam_ref, f)
    assert rel_l2(lam, lam_ref) <= 1e-8
    assert rel_l2(u, u_ref) <= 1e-8
    assert rel_l2(q, q_ref) <= 1e-8
    return pr, Aff, bf


@pytest.mark.parametrize("n,p,eps,lc", [(16, 2, 1e-3, "pre"), (16, 1, 1e-2, "pre"),
                                         (8, 4, 1e-3, "both"), (16, 3, 0.1, "pre")])
def test_gmres_solution_and_count_match_oracle(n, p, eps, lc):
    wl = workload(n, p, eps)
    s = solver(wl, coarsest_n=2, local_corr=LC[lc], rtol=1e-12, max_it=300)
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    assert info.converged == 1
    pr, Aff, bf = _check_solution(wl, host(lam), host(u), host(q), 1e-12)
    H = mg.Hierarchy(pr, coarsest_n=2, local_corr=lc)
    _, it, _, ok = H.solve_gmres(bf, tol=1e-12, max_it=300, left=False)
    assert ok and abs(info.iters - it) <= 1, (info.iters, it)


def test_dirichlet_data_and_fixed_point_iteration():
    """Inhomogeneous Dirichlet data, and MG as a fixed-point solver (Sec. 3.6)
    on the non-symmetric operator: counts within one of the oracle's."""
    n, p = 16, 2
    wl = workload(n, p, 0.05, seed=9)
    gD = W.dirichlet(lambda x, y: np.sin(3 * x) + y * y, n, p)
    s = solver(wl, krylov=hdgmg.KRYLOV_NONE, local_corr=hdgmg.LC_PRE, m_fine=3, rtol=1e-10,
               max_it=300)
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(gD))
    pr = oracle(wl)
    _, bf, *_ = pr.system(wl.f[0], gD)
    H = mg.Hierarchy(pr, coarsest_n=2, m_fine=3, local_corr="pre")
    _, it, _, ok = H.solve_fixed_point(bf, tol=1e-10, max_it=300)
    assert info.converged == 1 and ok
    assert abs(info.iters - it) <= 1, (info.iters, it)
    _check_solution(wl, host(lam), host(u), host(q), 1e-10, gD=gD)


@pytest.mark.parametrize("prec", [hdgmg.PREC_FP32, hdgmg.PREC_FP64, hdgmg.PREC_BF16])
def test_p6_gmres_reaches_fp64_residual(prec):
    """p = 6 (28 x 28 element operators), eps = 1e-3, FGMRES(30) with the
    step-3 cycle: FP64 residual 1e-10 with the FP32 cycle and with the BF16
    fine-level operator too."""
    wl = workload(32, 6, 1e-3)
    s = solver(wl, coarsest_n=4, m_max=4, local_corr=hdgmg.LC_PRE, precision=prec, rtol=1e-10)
    lam, u, q, info = s.solve(cuda(wl.f[0]))
    assert info.converged == 1 and info.rel_res <= 1e-10
    assert info.iters <= 40, info.iters
    _check_solution(wl, host(lam), host(u), host(q), 1e-10)


def test_discretisation_error_of_the_manufactured_solution():
    """The recovered u approximates sin(pi x) sin(pi y) to O(h^{p+1})."""
    errs = []
    for n in (8, 16):
        wl = workload(n, 2, 0.1)
        s = solver(wl, rtol=1e-12)
        _, u, _, info = s.solve(cuda(wl.f[0]), want_q=False)
        errs.append(oracle(wl).l2_error(host(u), W.sine_u))
    assert np.log2(errs[0] / errs[1]) >= 2.8, errs


def test_cg_and_adjoint_are_rejected():
    wl = workload(8, 2, 1e-2)
    with pytest.raises(hdgmg.HdgmgError) as ei:
        hdgmg.Solver(8, 2, tau_c=wl.tau_c, beta=wl.beta, krylov=hdgmg.KRYLOV_CG)
    assert ei.value.status == -1
    s = solver(wl)
    with pytest.raises(hdgmg.HdgmgError):
        s.gradient(cuda(wl.f[0]), cuda(np.zeros(wl.f[0].shape)))
