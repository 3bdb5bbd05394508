"""GPU adjoint (hdgmg_gradient / hdgmg_adjoint / the torch.autograd binding)
against the oracle's gradient (uncondensed adjoint, oracle/adjoint.py) and
against central finite differences of the GPU forward map.

Tolerance: 1e-6 relative to max|gradient| (finite differences with step 1e-5
on solves converged to 1e-13; the oracle comparison is tighter in practice)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import adjoint, hdg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _problem(n, p, seed):
    rng = np.random.default_rng(seed)
    logk = rng.normal(size=n * n)
    f = 1.0 + 0.3 * rng.standard_normal(((p + 1) ** 2, n * n))
    pr = hdg.HDGProblem(n, p, np.exp(logk), float(n))
    _, u, _ = adjoint.forward(pr, f)
    u_obs = u * (1.0 + 0.01 * rng.standard_normal(u.shape))
    return rng, logk, f, pr, u_obs


@pytest.mark.parametrize("prec", [hdgmg.PREC_FP64, hdgmg.PREC_FP32])
def test_gradient_matches_oracle(prec):
    n, p = 16, 2
    rng, logk, f, pr, u_obs = _problem(n, p, 54)
    s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=1.0, rtol=1e-13, precision=prec)
    s.setup(cuda(logk))
    J, gk, gf, info = s.gradient(cuda(f), cuda(u_obs))
    J_o, gk_o, gf_o = adjoint.gradient(pr, f, u_obs)
    assert abs(J - J_o) <= 1e-9 * abs(J_o)
    gk, gf = gk.cpu().numpy(), gf.cpu().numpy()
    assert np.abs(gk - gk_o).max() <= 1e-6 * np.abs(gk_o).max()
    assert np.abs(gf - gf_o).max() <= 1e-6 * np.abs(gf_o).max()


def test_gradient_matches_finite_differences():
    n, p = 16, 2
    rng, logk, f, pr, u_obs = _problem(n, p, 7)
    s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=1.0, rtol=1e-13)
    s.setup(cuda(logk))
    J, gk, _, _ = s.gradient(cuda(f), cuda(u_obs))
    gk = gk.cpu().numpy()
    M = np.diag(pr.forms.Mv)

    def misfit(lk):
        s.setup(cuda(lk))
        _, u, _, _ = s.solve(cuda(f), want_q=False)
        d = u.cpu().numpy() - u_obs
        return 0.5 * float(np.sum(M[:, None] * d * d))

    eps = 1e-5
    for e in rng.choice(n * n, 12, replace=False):
        lp, lm = logk.copy(), logk.copy()
        lp[e] += eps
        lm[e] -= eps
        fd = (misfit(lp) - misfit(lm)) / (2 * eps)
        assert abs(gk[e] - fd) <= 1e-6 * np.abs(gk).max(), (e, gk[e], fd)


def test_autograd_function():
    n, p = 8, 3
    rng, logk, f, pr, u_obs = _problem(n, p, 11)
    s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=1.0, rtol=1e-13)
    lk = cuda(logk).requires_grad_(True)
    ft = cuda(f).requires_grad_(True)
    weights = cuda(rng.standard_normal(f.shape))
    u = hdgmg.hdg_solve(s, lk, ft)
    loss = (u * weights).sum()
    loss.backward()
    g_lk = lk.grad.cpu().numpy()
    g_f = ft.grad.cpu().numpy()

    def loss_of(lk_np, f_np):
        with torch.no_grad():
            uu = hdgmg.hdg_solve(s, cuda(lk_np), cuda(f_np))
            return float((uu * weights).sum())

    eps = 1e-5
    for e in rng.choice(n * n, 6, replace=False):
        lp, lm = logk.copy(), logk.copy()
        lp[e] += eps
        lm[e] -= eps
        fd = (loss_of(lp, f) - loss_of(lm, f)) / (2 * eps)
        assert abs(g_lk[e] - fd) <= 1e-6 * np.abs(g_lk).max()
    for _ in range(4):
        a, e = rng.integers(f.shape[0]), rng.integers(n * n)
        fp, fm = f.copy(), f.copy()
        fp[a, e] += eps
        fm[a, e] -= eps
        fd = (loss_of(logk, fp) - loss_of(logk, fm)) / (2 * eps)
        assert abs(g_f[a, e] - fd) <= 1e-6 * np.abs(g_f).max()
