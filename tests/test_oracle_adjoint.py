"""Pin of the oracle's adjoint gradient: central finite differences of the
oracle's own forward map J(m, f) (an independent route: no adjoint algebra)."""
import numpy as np
import pytest

from oracle import adjoint, hdg


def _setup(n, p, seed):
    rng = np.random.default_rng(seed)
    logk = rng.normal(size=n * n)
    tau = float(n)                              # tau = 1/h on the unit square
    f = 1.0 + 0.3 * rng.standard_normal(((p + 1) ** 2, n * n))
    pr = hdg.HDGProblem(n, p, np.exp(logk), tau)
    _, u, _ = adjoint.forward(pr, f)
    u_obs = u * (1.0 + 0.01 * rng.standard_normal(u.shape))
    return rng, logk, tau, f, pr, u_obs


@pytest.mark.parametrize("n,p,sample", [(4, 2, None), (4, 1, None), (16, 2, 24)])
def test_gradient_matches_central_differences(n, p, sample):
    rng, logk, tau, f, pr, u_obs = _setup(n, p, 3 + n + p)
    J, gm, gf = adjoint.gradient(pr, f, u_obs)
    assert abs(J - adjoint.misfit_of(n, p, logk, tau, f, u_obs)) < 1e-14 * max(1.0, abs(J))
    eps = 1e-5
    idx = np.arange(n * n) if sample is None else rng.choice(n * n, sample, replace=False)
    for e in idx:
        lp, lm = logk.copy(), logk.copy()
        lp[e] += eps
        lm[e] -= eps
        fd = (adjoint.misfit_of(n, p, lp, tau, f, u_obs) - adjoint.misfit_of(n, p, lm, tau, f, u_obs)) / (2 * eps)
        assert abs(gm[e] - fd) <= 1e-6 * np.abs(gm).max(), (e, gm[e], fd)
    for _ in range(6):
        a, e = rng.integers(f.shape[0]), rng.integers(n * n)
        fp, fm = f.copy(), f.copy()
        fp[a, e] += eps
        fm[a, e] -= eps
        fd = (adjoint.misfit_of(n, p, logk, tau, fp, u_obs) - adjoint.misfit_of(n, p, logk, tau, fm, u_obs)) / (2 * eps)
        assert abs(gf[a, e] - fd) <= 1e-6 * np.abs(gf).max(), (a, e, gf[a, e], fd)


def test_gradient_vanishes_at_the_data():
    """u_obs = u(m) makes J = 0 a minimum: the gradient is zero."""
    rng, logk, tau, f, pr, _ = _setup(4, 2, 1)
    _, u, _ = adjoint.forward(pr, f)
    J, gm, gf = adjoint.gradient(pr, f, u.copy())
    assert J < 1e-28 and np.abs(gm).max() < 1e-12 and np.abs(gf).max() < 1e-12
