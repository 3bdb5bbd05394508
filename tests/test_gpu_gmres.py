"""Flexible GMRES(m) right-preconditioned by the V-cycle (the paper's Krylov
method, Sec. 4) on the GPU against the oracle's restarted GMRES with the same
V-cycle as right preconditioner (oracle/mg.py, solve_gmres(left=False)).

The two orthogonalise differently (classical Gram-Schmidt applied twice on
the GPU, modified Gram-Schmidt once in the oracle) and so agree on the
iteration count within one step per restart cycle, not bit for bit.
Solutions: FP64 relative residual <= rtol of the oracle's own A and g and
relative L2 error <= 1e-8 against the oracle's direct solve."""
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


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _solve_both(wl, lc, m_fine, restart, tol, coarsest_n=2, precision=hdgmg.PREC_FP64):
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=TAU[wl.tau_mode], tau_c=wl.tau_c, coarsest_n=coarsest_n,
                     m_fine=m_fine, local_corr=LC[lc], krylov=hdgmg.KRYLOV_GMRES,
                     gmres_restart=restart, rtol=tol, max_it=300, precision=precision)
    s.setup(cuda(wl.log_kappa))
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    pr = hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau())
    Aff, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=coarsest_n, m_fine=m_fine, local_corr=lc)
    _, it, _, ok = H.solve_gmres(bf, tol=tol, max_it=300, restart=restart, left=False)
    assert ok
    lam_h = host(lam)
    lam_f = hdg.api_to_edge_major(lam_h, wl.n, wl.p + 1)[pr.free_dofs()]
    res = np.linalg.norm(bf - Aff @ lam_f) / np.linalg.norm(bf)
    return s, info, it, res, pr, lam_h, host(u), host(q)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_example1_step3_correction_matches_oracle(p):
    """Example I, tau = 1/h, m_N = 3, local correction in step 3 only (the
    non-symmetric cycle that the paper pairs with GMRES)."""
    wl = W.example1(16, p)
    s, info, it, res, pr, lam, u, q = _solve_both(wl, "pre", 3, 30, 1e-10)
    assert info.converged == 1
    assert abs(info.iters - it) <= 1, (info.iters, it)
    assert res <= 1.5e-10
    lam_ref = pr.solve_direct(wl.f[0], wl.gD[0])
    u_ref, q_ref = pr.recover(lam_ref, wl.f[0])
    assert rel_l2(lam, lam_ref) <= 1e-8
    assert rel_l2(u, u_ref) <= 1e-8
    assert rel_l2(q, q_ref) <= 1e-8


@pytest.mark.parametrize("restart", [1, 3, 8])
def test_restarts_match_oracle(restart):
    """Short restart lengths force several restart cycles (restart = 1 is the
    degenerate GMRES(1)): the Arnoldi count agrees with the oracle's within
    one step per cycle."""
    rng = np.random.default_rng(31)
    wl = W.lognormal(32, 2, sigma=1.0, seed=31)
    wl.f = rng.standard_normal(wl.f.shape)
    s, info, it, res, *_ = _solve_both(wl, "both", 1, restart, 1e-9, coarsest_n=4)
    assert info.converged == 1
    cycles = -(-it // restart)
    assert abs(info.iters - it) <= max(1, cycles // 2 + 1), (info.iters, it)
    assert res <= 1.5e-9


def test_no_local_correction_and_p4():
    wl = W.lognormal(16, 4, sigma=0.5, seed=8)
    s, info, it, res, *_ = _solve_both(wl, "none", 2, 30, 1e-10)
    assert info.converged == 1
    assert abs(info.iters - it) <= 1, (info.iters, it)
    assert res <= 1.5e-10


def test_fp32_cycle_as_flexible_preconditioner():
    """With the FP32 V-cycle the preconditioner is not exactly linear;
    flexible GMRES still reaches the FP64 tolerance with about the FP64
    count."""
    wl = W.lognormal(64, 4, seed=2)
    s, info, it, res, *_ = _solve_both(wl, "both", 1, 30, 1e-10, coarsest_n=4,
                                       precision=hdgmg.PREC_FP32)
    assert info.converged == 1
    assert info.iters <= it + 2, (info.iters, it)
    assert res <= 1.5e-10


def test_gmres_agrees_with_cg_on_the_symmetric_cycle():
    wl = W.lognormal(32, 3, seed=5)
    f = cuda(wl.f[0])
    sols = []
    for kr in (hdgmg.KRYLOV_CG, hdgmg.KRYLOV_GMRES):
        s = hdgmg.Solver(32, 3, krylov=kr, rtol=1e-12, coarsest_n=4)
        s.setup(cuda(wl.log_kappa))
        lam, _, _, info = s.solve(f)
        assert info.converged == 1
        sols.append(host(lam))
    assert rel_l2(sols[1], sols[0]) <= 1e-10


def test_zero_rhs_and_several_rhs():
    wl = W.lognormal(8, 2, seed=1)
    s = hdgmg.Solver(8, 2, krylov=hdgmg.KRYLOV_GMRES, gmres_restart=4, rtol=1e-12)
    s.setup(cuda(wl.log_kappa))
    lam, u, _, info = s.solve(cuda(np.zeros_like(wl.f[0])))
    assert info.iters == 0 and info.converged == 1 and float(lam.abs().max()) == 0.0
    rng = np.random.default_rng(3)
    f = rng.standard_normal((3,) + wl.f.shape[1:])
    lam, _, _, info = s.solve(cuda(f))
    pr = hdg.HDGProblem(8, 2, np.exp(wl.log_kappa), wl.tau())
    for k in range(3):
        ref = pr.solve_direct(f[k])
        assert rel_l2(host(lam[k]), ref) <= 1e-9
