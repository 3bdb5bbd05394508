"""GPU tests of the matrix-free FP32 finest-level apply (opts.matrix_free):
A_e x = kappa K x + tau x - sum_i (kappa P_i + tau Q_i)^T (kappa P_i + tau Q_i) x / s_i
through the shared eigenbasis, used by the V-cycle's finest-level matvecs.

Tolerances:
  * one V-cycle against the oracle's FP64 V-cycle: 2e-3 relative, max norm.
    The FP32 sum subtracts terms of size kappa |K| |x| to form A_e x; for the
    smooth parts of x the result is ~1e3-1e4 times smaller than the terms, so
    FP32 rounding of the terms (6e-8 each, ~nt of them) leaves up to ~1e-4
    relative error in A_e x, which the cycle carries into e;
  * PCG (FP64 outer iteration): lambda within 1e-8 relative L2 of the
    oracle's direct solve at rtol 1e-12 (the preconditioner's rounding does
    not enter the FP64 residual), and at most 3 iterations more than the
    stored operator's count."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("n,p", [(16, 2), (32, 4), (16, 6), (32, 1)])
def test_matrix_free_vcycle_close_to_oracle(n, p):
    wl = W.lognormal(n, p, sigma=1.0, seed=51 + p, tau_mode="over_h")
    s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=wl.tau_c, coarsest_n=4, m_fine=1, m_max=2,
                     precision=hdgmg.PREC_FP32, matrix_free=1)
    s.setup(cuda(wl.log_kappa))
    H = mg.Hierarchy(hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau()), coarsest_n=4, m_fine=1,
                     m_max=2, local_corr="both")
    r = np.random.default_rng(52).standard_normal((p + 1, hdg.n_edges(n)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert float(np.abs(e - ref).max() / np.abs(ref).max()) <= 2e-3


@pytest.mark.parametrize("n,p", [(32, 3), (64, 4)])
def test_matrix_free_pcg_solution_and_iterations(n, p):
    wl = W.lognormal(n, p, seed=53 + p)
    f = np.random.default_rng(54).standard_normal(((p + 1) ** 2, n * n))
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-12, precision=hdgmg.PREC_FP32,
              tau_mode=hdgmg.TAU_OVER_H)
    res = {}
    for mf in (1, 0):
        s = hdgmg.Solver(n, p, matrix_free=mf, **kw)
        s.setup(cuda(wl.log_kappa))
        lam, _, _, info = s.solve(cuda(f), want_u=False, want_q=False)
        assert info.converged == 1 and info.rel_res <= 1e-12, (mf, info.as_dict())
        res[mf] = (host(lam).copy(), info.iters)
    assert res[1][1] <= res[0][1] + 3
    ref = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau()).solve_direct(f)
    assert rel(res[1][0], ref) <= 1e-8


def test_matrix_free_blocked_solve_matches_single():
    n, p, k = 32, 3, 3
    wl = W.lognormal(n, p, seed=55)
    F = np.random.default_rng(56).standard_normal((k, (p + 1) ** 2, n * n))
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-12, precision=hdgmg.PREC_FP32, matrix_free=1,
              tau_mode=hdgmg.TAU_OVER_H)
    sb = hdgmg.Solver(n, p, rhs_block=4, **kw)
    sb.setup(cuda(wl.log_kappa))
    lam, _, _, info = sb.solve(cuda(F), want_u=False, want_q=False)
    assert info.converged == 1
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau())
    for j in range(k):
        assert rel(host(lam[j]), pr.solve_direct(F[j])) <= 1e-8


@pytest.mark.parametrize("kw", [dict(p=7, precision=hdgmg.PREC_FP32),
                                dict(p=3, precision=hdgmg.PREC_FP64),
                                dict(p=3, precision=hdgmg.PREC_BF16)])
def test_matrix_free_rejected_outside_its_range(kw):
    p = kw.pop("p")
    with pytest.raises(hdgmg.HdgmgError):
        hdgmg.Solver(8, p, matrix_free=1, **kw)


def test_matrix_free_under_fp32_refinement():
    """PREC_FP32_IR: the inner FP32 PCG's V-cycle applies the finest operator
    matrix-free, the inner matvec and the FP64 residual stay stored."""
    n, p = 32, 3
    wl = W.lognormal(n, p, seed=57)
    f = np.random.default_rng(58).standard_normal(((p + 1) ** 2, n * n))
    s = hdgmg.Solver(n, p, coarsest_n=4, m_fine=1, m_max=2, rtol=1e-11, precision=hdgmg.PREC_FP32_IR,
                     matrix_free=1, tau_mode=hdgmg.TAU_OVER_H)
    s.setup(cuda(wl.log_kappa))
    lam, _, _, info = s.solve(cuda(f), want_u=False, want_q=False)
    assert info.converged == 1 and info.rel_res <= 1e-11
    ref = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau()).solve_direct(f)
    assert rel(host(lam), ref) <= 1e-8
