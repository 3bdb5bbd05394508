"""GPU parity of the point smoothers of Sec. 4.1 (damped point-Jacobi,
Chebyshev-accelerated point-Jacobi, multicolour LU-SGS) against the oracle's
multigrid with the same smoother, through the C ABI.

Tolerances: one FP64 V-cycle 1e-10 relative (the Chebyshev interval comes
from 30 power iterations on both sides from the same start vector; the two
estimates agree to rounding); FP32 cycle 1e-4; solutions as in
test_gpu_parity.py; iteration counts within one of the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

SM = {"point_jacobi": (hdgmg.SMOOTH_POINT_JACOBI, 2.0 / 3.0),
      "chebyshev": (hdgmg.SMOOTH_CHEBYSHEV, 1.0),
      "lu_sgs": (hdgmg.SMOOTH_LU_SGS, 1.0)}
LC = {"none": hdgmg.LC_NONE, "pre": hdgmg.LC_PRE, "both": hdgmg.LC_BOTH}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def pair(wl, sm, beta=None, coarsest_n=2, m_fine=1, local_corr="both", **solver_kw):
    """The library's solver and the oracle's hierarchy with the same options."""
    code, om = SM[sm]
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=hdgmg.TAU_OVER_H, tau_c=wl.tau_c, beta=beta,
                     smoother=code, omega=om, coarsest_n=coarsest_n, m_fine=m_fine,
                     local_corr=LC[local_corr], **solver_kw)
    s.setup(cuda(wl.log_kappa))
    pr = hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau(), beta=beta)
    H = mg.Hierarchy(pr, coarsest_n=coarsest_n, m_fine=m_fine, local_corr=local_corr, smoother=sm,
                     omega=om)
    return s, H, pr


@pytest.mark.parametrize("sm", list(SM))
@pytest.mark.parametrize("n,p,lc,m", [(16, 2, "both", 2), (8, 3, "pre", 1), (8, 1, "pre", 3)])
def test_vcycle_matches_oracle(sm, n, p, lc, m):
    rng = np.random.default_rng(40 + p)
    wl = W.lognormal(n, p, sigma=1.0, seed=40 + p)
    s, H, _ = pair(wl, sm, local_corr=lc, m_fine=m)
    r = rng.standard_normal((p + 1, hdg.n_edges(n)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert np.abs(e - ref).max() <= 1e-10 * np.abs(ref).max(), sm


@pytest.mark.parametrize("sm", list(SM))
def test_fp32_vcycle_close_to_oracle(sm):
    wl = W.lognormal(32, 4, seed=3)
    s, H, _ = pair(wl, sm, coarsest_n=4, precision=hdgmg.PREC_FP32)
    rng = np.random.default_rng(9)
    r = rng.standard_normal((5, hdg.n_edges(32)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert rel_l2(e, ref) <= 1e-4, sm


@pytest.mark.parametrize("sm", list(SM))
def test_fixed_point_counts_match_oracle(sm):
    """MG as a solver on Example I (tau = 1/h, m_N = 3, step-3 correction)."""
    wl = W.example1(16, 2)
    s, H, pr = pair(wl, sm, local_corr="pre", m_fine=3, krylov=hdgmg.KRYLOV_NONE, rtol=1e-9,
                    max_it=300)
    _, _, _, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    _, it, _, ok = H.solve_fixed_point(bf, tol=1e-9, max_it=300)
    assert ok and info.converged == 1
    assert abs(info.iters - it) <= 1, (sm, info.iters, it)


@pytest.mark.parametrize("sm", list(SM))
def test_pcg_solution_matches_direct_solve(sm):
    wl = W.lognormal(32, 2, seed=6)
    s, H, pr = pair(wl, sm, coarsest_n=4, rtol=1e-12)
    lam, u, q, info = s.solve(cuda(wl.f[0]))
    assert info.converged == 1
    lam_ref = pr.solve_direct(wl.f[0])
    u_ref, q_ref = pr.recover(lam_ref, wl.f[0])
    assert rel_l2(host(lam), lam_ref) <= 1e-8
    assert rel_l2(host(u), u_ref) <= 1e-8
    assert rel_l2(host(q), q_ref) <= 1e-8


def test_lu_sgs_on_convection_diffusion():
    """LU-SGS on the non-symmetric operator (full storage) inside GMRES."""
    wl = W.convdiff(16, 2, eps=1e-2)
    s, H, pr = pair(wl, "lu_sgs", beta=wl.beta, local_corr="pre", krylov=hdgmg.KRYLOV_GMRES,
                    rtol=1e-10)
    rng = np.random.default_rng(2)
    r = rng.standard_normal((3, hdg.n_edges(16)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert np.abs(e - ref).max() <= 1e-10 * np.abs(ref).max()
    lam, _, _, info = s.solve(cuda(wl.f[0]))
    assert info.converged == 1
    assert rel_l2(host(lam), pr.solve_direct(wl.f[0])) <= 1e-8
