"""GPU parity on Examples III and IV of Sec. 4 on quadrilateral meshes
(smooth kappa; a 1e6 checkerboard jump) against the oracle, through the C ABI.

Tolerances: iteration counts within one of the oracle's (fixed point; PCG;
right-preconditioned GMRES); solutions (relative L2 of lambda and u) 1e-8
against the oracle's sparse direct solve, 1e-7 on Example IV whose 1e6 jump
raises the condition number of the trace system by about that factor (solves
to 1e-12)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

SCHEME = {"hdg": hdgmg.SCHEME_HDG, "sipg": hdgmg.SCHEME_SIPG, "iipg": hdgmg.SCHEME_IIPG,
          "nipg": hdgmg.SCHEME_NIPG}
TAU = {"const": hdgmg.TAU_CONST, "over_h": hdgmg.TAU_OVER_H,
       "kappa_over_h": hdgmg.TAU_KAPPA_OVER_H}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def run(wl, scheme, krylov, prec=hdgmg.PREC_FP64, rtol=1e-12):
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=TAU[wl.tau_mode], tau_c=wl.tau_c, scheme=SCHEME[scheme],
                     krylov=krylov, local_corr=hdgmg.LC_PRE if krylov != hdgmg.KRYLOV_CG
                     else hdgmg.LC_BOTH, m_fine=3 if krylov == hdgmg.KRYLOV_NONE else 1,
                     coarsest_n=2, precision=prec, rtol=rtol, max_it=300)
    s.setup(cuda(wl.log_kappa))
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    pr = hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau(), scheme=scheme)
    return host(lam), host(u), info, pr


@pytest.mark.parametrize("scheme,c", [("hdg", 1.0), ("sipg", None)])
@pytest.mark.parametrize("p", [2, 4])
def test_example4_fixed_point_counts_and_solution(scheme, c, p):
    c = c if c is not None else float((p + 1) * (p + 2))
    wl = W.checkerboard(32, p, tau_mode="kappa_over_h", tau_c=c)
    lam, u, info, pr = run(wl, scheme, hdgmg.KRYLOV_NONE, rtol=1e-9)
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=2, m_fine=3, local_corr="pre")
    _, it, _, ok = H.solve_fixed_point(bf, tol=1e-9, max_it=300)
    assert info.converged == 1 and ok and abs(info.iters - it) <= 1, (info.iters, it)


@pytest.mark.parametrize("scheme,c", [("hdg", 1.0), ("sipg", None)])
@pytest.mark.parametrize("prec", [hdgmg.PREC_FP64, hdgmg.PREC_FP32])
def test_example4_pcg(scheme, c, prec):
    """PCG with the symmetric cycle; the FP32 cycle reaches the FP64 residual
    on the 1e6 jump with the FP64 cycle's count (+1)."""
    p = 3
    c = c if c is not None else float((p + 1) * (p + 2))
    wl = W.checkerboard(32, p, tau_mode="kappa_over_h", tau_c=c)
    lam, u, info, pr = run(wl, scheme, hdgmg.KRYLOV_CG, prec=prec)
    assert info.converged == 1
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=2, local_corr="both")
    _, it, _, ok = H.solve_pcg(bf, tol=1e-12, max_it=300)
    assert ok and abs(info.iters - it) <= 1, (info.iters, it)
    lam_ref = pr.solve_direct(wl.f[0], wl.gD[0])
    u_ref, _ = pr.recover(lam_ref, wl.f[0])
    assert rel_l2(lam, lam_ref) <= 1e-7
    assert rel_l2(u, u_ref) <= 1e-7


@pytest.mark.parametrize("scheme,mode,c", [("iipg", "kappa_over_h", None), ("nipg", "kappa_over_h", None),
                                           ("hdg", "const", 1.0)])
def test_example3_gmres(scheme, mode, c):
    p, n = 3, 32
    c = c if c is not None else float((p + 1) * (p + 2))
    wl = W.example3(n, p, tau_mode=mode, tau_c=c)
    lam, u, info, pr = run(wl, scheme, hdgmg.KRYLOV_GMRES)
    assert info.converged == 1
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=2, local_corr="pre")
    _, it, _, ok = H.solve_gmres(bf, tol=1e-12, max_it=300, left=False)
    assert ok and abs(info.iters - it) <= 1, (info.iters, it)
    lam_ref = pr.solve_direct(wl.f[0], wl.gD[0])
    u_ref, _ = pr.recover(lam_ref, wl.f[0])
    assert rel_l2(lam, lam_ref) <= 1e-8
    assert rel_l2(u, u_ref) <= 1e-8
    assert pr.l2_error(u, W.ex1_u) < 1e-3     # O(h^2) from the element-centre kappa
