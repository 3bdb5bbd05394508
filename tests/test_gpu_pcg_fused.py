"""GPU tests of the fused PCG iteration (opts.pcg_fuse = 1, the default):
the direction update, the FP64 matvec and p.Ap in one kernel (p.Ap summed
element by element as sum_e p_e^T A_e p_e), then x, r and p in one update
kernel.  Against the unfused iteration (pcg_fuse = 0: separate direction,
matvec, dot and update kernels) it runs the same recurrence with a
different summation order, so:
  * the PCG count within one of the unfused count;
  * lambda within 1e-10 relative L2 of the unfused solution (both solved to
    1e-12) and within 1e-8 of the oracle's direct solve (the suite's solution
    tolerance);
  * the reported residual (recomputed in FP64 after the loop) at or below rtol;
  * the same solve twice gives the same bits (fixed reduction order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("precision,pcg_graph", [(hdgmg.PREC_FP32, 1), (hdgmg.PREC_FP64, 1),
                                                 (hdgmg.PREC_BF16, 1), (hdgmg.PREC_FP32, 0)])
@pytest.mark.parametrize("n,p", [(32, 3), (48, 4), (32, 1), (24, 2)])
def test_fused_pcg_matches_unfused_and_direct(precision, pcg_graph, n, p):
    """p = 1: the finest level is the persistent cycle's first P1 level, so
    r.z falls back to its own kernel; p = 2, 3, 4: r.z in the finest level's
    last block-Jacobi step."""
    wl = W.lognormal(n, p, seed=31 + p)
    f = np.random.default_rng(32).standard_normal(((p + 1) ** 2, n * n))
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-12, precision=precision, pcg_graph=pcg_graph,
              tau_mode=hdgmg.TAU_OVER_H)
    out = {}
    for fuse in (1, 0):
        s = hdgmg.Solver(n, p, pcg_fuse=fuse, **kw)
        s.setup(cuda(wl.log_kappa))
        lam, _, _, info = s.solve(cuda(f), want_u=False, want_q=False)
        assert info.converged == 1 and info.rel_res <= 1e-12, (fuse, info.as_dict())
        out[fuse] = (host(lam).copy(), info.iters)
        if fuse:
            lam2, _, _, info2 = s.solve(cuda(f), want_u=False, want_q=False)
            assert np.array_equal(host(lam2), out[1][0]) and info2.iters == info.iters
        s.close()
    assert abs(out[1][1] - out[0][1]) <= 1
    assert rel(out[1][0], out[0][0]) <= 1e-10
    ref = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau()).solve_direct(f)
    assert rel(out[1][0], ref) <= 1e-8


def test_fused_pcg_with_dirichlet_data():
    """Non-zero boundary data: the lift enters the right-hand side, the
    Dirichlet entries of the direction stay zero in the fused matvec."""
    n, p = 32, 2
    wl = W.lognormal(n, p, seed=41)
    rng = np.random.default_rng(42)
    f = rng.standard_normal(((p + 1) ** 2, n * n))
    gD = rng.standard_normal((p + 1, hdg.n_edges(n)))
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-12, precision=hdgmg.PREC_FP32,
              tau_mode=hdgmg.TAU_OVER_H)
    lams = []
    for fuse in (1, 0):
        s = hdgmg.Solver(n, p, pcg_fuse=fuse, **kw)
        s.setup(cuda(wl.log_kappa))
        lam, _, _, info = s.solve(cuda(f), cuda(gD), want_u=False, want_q=False)
        assert info.converged == 1
        lams.append(host(lam).copy())
    assert rel(lams[0], lams[1]) <= 1e-10
