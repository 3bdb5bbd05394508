"""GPU parity of the CUDA path against the CPU FP64 oracle, through the C ABI.

Tolerances, from the arithmetic:
  * FP64 element operators and level operators: |gpu - oracle| <= 1e-11 max|A|
    (two different FP64 factorisations of local blocks whose condition
    numbers stay below ~1e4);
  * one FP64 V-cycle: 1e-10 relative (max norm);
  * solutions: FP64 relative residual <= 1e-10 of the oracle's own A and g,
    relative L2 error of lambda, u, q <= 1e-8 against the oracle's direct solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TAU = {"const": hdgmg.TAU_CONST, "over_h": hdgmg.TAU_OVER_H}
LC = {"none": hdgmg.LC_NONE, "pre": hdgmg.LC_PRE, "both": hdgmg.LC_BOTH}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def make(wl, **opts):
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=TAU[wl.tau_mode], tau_c=wl.tau_c, **opts)
    s.setup(cuda(wl.log_kappa))
    return s


def oracle_problem(wl):
    return hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau())


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def random_kappa_workload(n, p, seed, tau_mode="over_h"):
    rng = np.random.default_rng(seed)
    wl = W.lognormal(n, p, sigma=1.0, seed=seed, tau_mode=tau_mode)
    wl.f = rng.standard_normal(wl.f.shape)
    return wl


# ----------------------------------------------------------------- K1
@pytest.mark.parametrize("n,p", [(4, 1), (8, 2), (8, 3), (8, 4), (4, 6), (4, 8), (3, 5)])
def test_element_condensation_matches_oracle(n, p):
    wl = random_kappa_workload(n, p, 100 + p)
    if n % 2:
        s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, coarsest_n=n)
        s.setup(cuda(wl.log_kappa))
    else:
        s = make(wl)
    A = host(s.element_matrices(0))                         # [nl][nl][E]
    Ae, _ = oracle_problem(wl).condense()
    ref = np.transpose(Ae, (1, 2, 0))
    assert np.abs(A - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("p", [1, 2, 4])
def test_condensed_rhs_with_dirichlet_lift(p):
    n = 8
    wl = W.example1(n, p)
    rng = np.random.default_rng(p)
    wl.log_kappa = rng.normal(size=n * n)
    s = make(wl)
    b = host(s.condensed_rhs(cuda(wl.f[0]), cuda(wl.gD[0])))
    pr = oracle_problem(wl)
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    bo = np.zeros(hdg.n_edges(n) * (p + 1))
    bo[pr.free_dofs()] = bf
    ref = hdg.edge_major_to_api(bo, n, p + 1)
    assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()


# ------------------------------------------------------- hierarchy K2-K4
@pytest.mark.parametrize("n,p", [(8, 1), (16, 2), (8, 4)])
def test_level_operators_match_oracle_hierarchy(n, p):
    wl = random_kappa_workload(n, p, 7 + p)
    s = make(wl, coarsest_n=2)
    H = mg.Hierarchy(oracle_problem(wl), coarsest_n=2)
    assert s.num_levels() == len(H.levels)
    rng = np.random.default_rng(3)
    for k, L in enumerate(H.levels):
        assert s.level_shape(k) == (L.n, L.nd)
        for _ in range(2):
            x = rng.standard_normal((L.nd, hdg.n_edges(L.n)))
            y = host(s.apply_operator(k, cuda(x)))
            ref = H.from_free(L.A @ H.to_free(x, k), k)
            assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max(), k


# ------------------------------------------------------------- V-cycle
@pytest.mark.parametrize("n,p,lc,m", [(8, 1, "pre", 1), (16, 2, "both", 1), (8, 3, "both", 2),
                                       (16, 4, "pre", 3), (8, 2, "none", 2)])
def test_vcycle_matches_oracle(n, p, lc, m):
    wl = random_kappa_workload(n, p, 11 + p)
    s = make(wl, coarsest_n=2, m_fine=m, local_corr=LC[lc])
    H = mg.Hierarchy(oracle_problem(wl), coarsest_n=2, m_fine=m, local_corr=lc)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((p + 1, hdg.n_edges(n)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert np.abs(e - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("n,p", [(32, 2), (64, 4)])
def test_fp32_vcycle_close_to_oracle(n, p):
    """The FP32 V-cycle (fused P1 tail included) approximates the FP64 one of
    the oracle to FP32 accuracy amplified by the hierarchy's conditioning."""
    wl = random_kappa_workload(n, p, 21 + p)
    s = make(wl, coarsest_n=4, m_fine=1, m_max=4, precision=hdgmg.PREC_FP32)
    H = mg.Hierarchy(oracle_problem(wl), coarsest_n=4, m_fine=1, m_max=4, local_corr="both")
    rng = np.random.default_rng(6)
    r = rng.standard_normal((p + 1, hdg.n_edges(n)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert rel_l2(e, ref) <= 1e-4


def test_bf16_fine_operator():
    """PREC_BF16: the finest level's V-cycle matvecs read BF16 operators
    (FP32 accumulation).  One cycle stays within 2e-2 of the FP64 cycle and
    is measurably less accurate than the FP32 cycle (the BF16 copy is what
    runs); the FP64 PCG around it still reaches the FP64 residual."""
    wl = random_kappa_workload(32, 4, 31)
    s16 = make(wl, coarsest_n=4, m_fine=1, m_max=4, precision=hdgmg.PREC_BF16, rtol=1e-11)
    s32 = make(wl, coarsest_n=4, m_fine=1, m_max=4, precision=hdgmg.PREC_FP32, rtol=1e-11)
    H = mg.Hierarchy(oracle_problem(wl), coarsest_n=4, m_fine=1, m_max=4, local_corr="both")
    rng = np.random.default_rng(9)
    r = rng.standard_normal((5, hdg.n_edges(32)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    err16 = rel_l2(host(s16.apply_vcycle(cuda(r))), ref)
    err32 = rel_l2(host(s32.apply_vcycle(cuda(r))), ref)
    print("V-cycle relative error: bf16 %.3e  fp32 %.3e" % (err16, err32))
    assert err16 <= 2e-2 and err16 > 10 * err32
    lam, u, q, i16 = s16.solve(cuda(wl.f[0]))
    _, _, _, i32 = s32.solve(cuda(wl.f[0]))
    print("PCG iterations: bf16 %d  fp32 %d" % (i16.iters, i32.iters))
    assert i16.converged == 1 and i16.rel_res <= 1e-11
    assert i16.iters <= i32.iters + 3
    _check_solution(wl, host(lam), host(u), host(q), rtol_res=1e-11, tol_sol=1e-7)


# ---------------------------------------------------------- end to end
def _check_solution(wl, lam, u, q, rtol_res=1e-10, tol_sol=1e-8):
    pr = oracle_problem(wl)
    Aff, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    lam_f = hdg.api_to_edge_major(lam, wl.n, wl.p + 1)[pr.free_dofs()]
    res = np.linalg.norm(bf - Aff @ lam_f) / np.linalg.norm(bf)
    assert res <= rtol_res * 1.5, res
    lam_ref = pr.solve_direct(wl.f[0], wl.gD[0])
    u_ref, q_ref = pr.recover(lam_ref, wl.f[0])
    assert rel_l2(lam, lam_ref) <= tol_sol
    assert rel_l2(u, u_ref) <= tol_sol
    assert rel_l2(q, q_ref) <= tol_sol


def test_poisson_sine_16_p2_three_level_cg():
    """16 x 16, p = 2, kappa = 1, tau = 1, V(1,1) with levels 16^2 P2 -> 16^2
    P1 -> 8^2 P1 (coarsest, direct), PCG to 1e-10."""
    wl = W.poisson_sine(16, 2)
    s = make(wl, coarsest_n=8, m_fine=1, local_corr=hdgmg.LC_BOTH, rtol=1e-13)
    assert s.num_levels() == 3
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    assert info.converged == 1
    _check_solution(wl, host(lam), host(u), host(q))
    # iteration count of the same PCG on the oracle's hierarchy
    s2 = make(wl, coarsest_n=8, m_fine=1, local_corr=hdgmg.LC_BOTH, rtol=1e-10)
    _, _, _, info2 = s2.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    pr = oracle_problem(wl)
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=8, m_fine=1, local_corr="both")
    _, it, _, ok = H.solve_pcg(bf, tol=1e-10)
    assert ok and abs(info2.iters - it) <= 1, (info2.iters, it)


@pytest.mark.parametrize("p,prec", [(1, hdgmg.PREC_FP64), (3, hdgmg.PREC_FP64), (2, hdgmg.PREC_FP32),
                                    (4, hdgmg.PREC_FP32)])
def test_example1_with_dirichlet_data(p, prec):
    wl = W.example1(16, p)
    s = make(wl, precision=prec, rtol=1e-13, max_it=100)
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    assert info.converged == 1, info.as_dict()
    _check_solution(wl, host(lam), host(u), host(q))


@pytest.mark.parametrize("prec", [hdgmg.PREC_FP32, hdgmg.PREC_FP32_IR])
def test_lognormal_mixed_precision_reaches_fp64_residual(prec):
    wl = W.lognormal(64, 4, seed=2)
    s64 = make(wl, precision=hdgmg.PREC_FP64)
    s32 = make(wl, precision=prec)
    f = cuda(wl.f[0])
    l64, u64, q64, i64 = s64.solve(f)
    l32, u32, q32, i32 = s32.solve(f)
    assert i64.converged and i32.converged
    assert i64.rel_res <= 1e-10 and i32.rel_res <= 1e-10
    assert i64.refinements == 0
    if prec == hdgmg.PREC_FP32:
        # FP64 PCG with the FP32 V-cycle: the count of the FP64 V-cycle
        assert abs(i32.iters - i64.iters) <= 2, (i32.iters, i64.iters)
    else:
        # refinement: a few FP64 outer steps around inner FP32 PCG solves
        assert 1 <= i32.refinements <= 8
        assert i32.iters <= 3 * i64.iters, (i32.iters, i64.iters)
    _check_solution(wl, host(l32), host(u32), host(q32), tol_sol=1e-7)


def test_fixed_point_counts_match_oracle():
    """MG as a solver (Sec. 3.6), Example I, tau = 1/h, m_N = 3, step-3 local
    correction: same iteration count as the oracle (and the paper's table)."""
    for p in (1, 2):
        wl = W.example1(16, p)
        s = make(wl, krylov=hdgmg.KRYLOV_NONE, local_corr=hdgmg.LC_PRE, m_fine=3, rtol=1e-9)
        _, _, _, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
        pr = oracle_problem(wl)
        _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
        H = mg.Hierarchy(pr, coarsest_n=2, m_fine=3, local_corr="pre")
        _, it, _, ok = H.solve_fixed_point(bf, tol=1e-9)
        assert info.converged and ok
        assert abs(info.iters - it) <= 1, (p, info.iters, it)


# ---------------------------------------------------------- edge cases
def test_single_level_direct_solve():
    """n = coarsest_n with p = 1: the hierarchy is one level and B = A^-1."""
    wl = W.example1(4, 1)
    s = make(wl, coarsest_n=4, rtol=1e-12)
    assert s.num_levels() == 1
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    assert info.iters <= 2
    _check_solution(wl, host(lam), host(u), host(q))


def test_zero_data_gives_zero_solution():
    wl = W.lognormal(8, 2, seed=1)
    s = make(wl)
    lam, u, q, info = s.solve(cuda(np.zeros_like(wl.f[0])))
    assert info.iters == 0 and info.converged == 1
    assert float(lam.abs().max()) == 0.0 and float(u.abs().max()) == 0.0


def test_several_right_hand_sides():
    wl = W.lognormal(8, 3, seed=4)
    rng = np.random.default_rng(0)
    f = rng.standard_normal((3,) + wl.f.shape[1:])
    s = make(wl, rtol=1e-12)
    lam, u, q, info = s.solve(cuda(f))
    for k in range(3):
        wk = W.Workload("k", wl.n, wl.p, wl.log_kappa, f[k:k + 1], wl.gD, wl.tau_mode, wl.tau_c)
        _check_solution(wk, host(lam[k]), host(u[k]), host(q[k]))


def test_nan_kappa_reports_breakdown():
    wl = W.lognormal(8, 2, seed=1)
    logk = wl.log_kappa.copy()
    logk[5] = np.nan
    s = hdgmg.Solver(8, 2)
    with pytest.raises(hdgmg.HdgmgError) as ei:
        s.setup(cuda(logk))
    assert ei.value.status == -5
    with pytest.raises(hdgmg.HdgmgError):
        s.solve(cuda(wl.f[0]))


def test_run_host_matches_device_call():
    wl = W.example1(16, 2)
    s = make(wl, rtol=1e-12)
    lam_d, u_d, q_d, _ = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    lam = np.zeros((3, hdg.n_edges(16)))
    u = np.zeros((9, 256))
    q = np.zeros((2, 9, 256))
    st, info = s.run_host(np.ascontiguousarray(wl.log_kappa), np.ascontiguousarray(wl.f[0]),
                          np.ascontiguousarray(wl.gD[0]), lam, u, q)
    assert st == 0
    assert np.abs(lam - host(lam_d)).max() == 0.0
    assert np.abs(u - host(u_d)).max() == 0.0
    assert np.abs(q - host(q_d)).max() == 0.0
