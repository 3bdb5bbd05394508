"""Pins of the oracle's HDG discretisation and condensation (Sec. 2).

Each test fixes a property the mathematics demands independently of how the
oracle computes it, chosen so that a dropped term, a sign error or a wrong
index in the local equations fails at least one of them."""
import numpy as np
import pytest

from oracle import hdg
from paper_1811_09909_gb300 import workloads as W


def _solve(n, p, kappa, tau, f_fun, g_fun):
    pr = hdg.HDGProblem(n, p, kappa, tau)
    f = W.nodal(f_fun, n, p)
    gD = W.dirichlet(g_fun, n, p)
    lam = pr.solve_direct(f, gD)
    u, q = pr.recover(lam, f)
    return pr, lam, u, q


@pytest.mark.parametrize("p,tau", [(2, 1.0), (3, 7.0), (2, 0.3)])
def test_patch_quadratic_exact(p, tau):
    """u = x^2 + y^2 (q = -(2x, 2y), f = -4) lies in the discrete spaces for
    p >= 2: HDG reproduces it to roundoff on any mesh and any tau > 0."""
    pr, lam, u, q = _solve(4, p, 1.0, tau, lambda x, y: -4.0 + 0 * x, lambda x, y: x ** 2 + y ** 2)
    X, Y = pr.node_coords()
    assert np.abs(u - (X ** 2 + Y ** 2)).max() < 1e-12
    assert np.abs(q[0] + 2 * X).max() < 1e-11
    assert np.abs(q[1] + 2 * Y).max() < 1e-11
    lam_exact = W.dirichlet(lambda x, y: x ** 2 + y ** 2, 4, p)
    # interior traces too: compare against the exact trace on every edge
    lam_all = _all_edge_coeffs(lambda x, y: x ** 2 + y ** 2, 4, p)
    assert np.abs(lam - lam_all).max() < 1e-12
    assert lam_exact.shape == lam.shape


def _all_edge_coeffs(fun, n, p, nq=12):
    from numpy.polynomial import legendre as npleg
    s, w = npleg.leggauss(nq)
    h = 1.0 / n
    P = np.stack([npleg.legval(s, np.eye(p + 1)[k]) for k in range(p + 1)])
    sc = np.sqrt((2 * np.arange(p + 1) + 1) / h)[:, None]
    out = np.zeros((p + 1, hdg.n_edges(n)))
    for j in range(n):
        for i in range(n + 1):
            out[:, j * (n + 1) + i] = (P * sc) @ (w * fun(i * h + 0 * s, (j + 0.5) * h + 0.5 * h * s)) * h / 2
    for j in range(n + 1):
        for i in range(n):
            out[:, n * (n + 1) + j * n + i] = (P * sc) @ (w * fun((i + 0.5) * h + 0.5 * h * s, j * h + 0 * s)) * h / 2
    return out


def test_patch_linear_p1_variable_kappa():
    """u = 1 + 2x - 3y with piecewise-constant kappa: q = -kappa grad u is
    discontinuous but q.n is continuous only if kappa is constant, so use
    kappa constant per test and several values."""
    for kap in (0.01, 1.0, 50.0):
        pr, lam, u, q = _solve(4, 1, kap, 2.0, lambda x, y: 0 * x, lambda x, y: 1 + 2 * x - 3 * y)
        X, Y = pr.node_coords()
        assert np.abs(u - (1 + 2 * X - 3 * Y)).max() < 1e-11
        assert np.abs(q[0] + 2 * kap).max() < 1e-9 * max(1, kap)
        assert np.abs(q[1] - 3 * kap).max() < 1e-9 * max(1, kap)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_convergence_rates_u_and_q(p):
    """Manufactured u = sin(pi x) sin(pi y), tau = 1: L2 errors of u and q
    decrease like h^{p+1} (HDG literature; the paper cites the rates)."""
    errs = []
    for n in (4, 8, 16):
        pr, lam, u, q = _solve(n, p, 1.0, 1.0, W.sine_f, lambda x, y: 0 * x)
        eu = pr.l2_error(u, W.sine_u)
        eq = np.hypot(pr.l2_error(q[0], lambda x, y: W.sine_q(x, y)[0]),
                      pr.l2_error(q[1], lambda x, y: W.sine_q(x, y)[1]))
        errs.append((eu, eq))
    ru = np.log2(errs[1][0] / errs[2][0])
    rq = np.log2(errs[1][1] / errs[2][1])
    assert abs(ru - (p + 1)) < 0.25, ru
    assert abs(rq - (p + 1)) < 0.25, rq


@pytest.mark.parametrize("p", [1, 2, 4])
def test_element_matrix_properties(p):
    rng = np.random.default_rng(7)
    pr = hdg.HDGProblem(3, p, np.exp(rng.normal(size=9)), rng.uniform(0.5, 5, size=9),
                        x1=0.6, y1=0.9)
    Ae, _ = pr.condense()
    scale = np.abs(Ae).max()
    # symmetric positive semi-definite
    assert np.abs(Ae - Ae.transpose(0, 2, 1)).max() < 1e-12 * scale
    ev = np.linalg.eigvalsh(Ae)
    assert ev.min() > -1e-12 * scale
    # exactly one zero eigenvalue: the constant trace (DtN of a constant is 0)
    c = np.zeros(pr.nt)
    for le, length in enumerate((pr.hy, pr.hy, pr.hx, pr.hx)):
        c[le * (p + 1)] = np.sqrt(length)
    assert np.abs(Ae @ c).max() < 1e-12 * scale
    assert (ev[:, 1] > 1e-8 * scale).all()


def test_homogeneity_in_kappa_tau():
    """A_e(c kappa, c tau) = c A_e(kappa, tau) (the local problem is linear in
    (kappa, tau) after scaling q)."""
    a = hdg.HDGProblem(2, 3, 1.3, 2.1).condense()[0]
    b = hdg.HDGProblem(2, 3, 1.3 * 7.0, 2.1 * 7.0).condense()[0]
    assert np.abs(b - 7.0 * a).max() < 1e-12 * np.abs(b).max()


def test_p0_closed_form():
    """p = 0 on one element of side h: worked by hand from HDG_local1/2,
    HDG_flux and conservation:
    A_e = (kappa/h)[[1,-1,0,0],[-1,1,0,0],[0,0,1,-1],[0,0,-1,1]] + tau (I - 11^T/4),
    g_e = f h^{3/2} / 4 (1,1,1,1)."""
    h, k, t, fv = 0.5, 2.0, 3.0, 1.7
    pr = hdg.HDGProblem(1, 0, k, t, x1=h, y1=h)
    Ae, ge = pr.condense(np.array([[fv]]))
    ref = (k / h) * np.array([[1, -1, 0, 0], [-1, 1, 0, 0], [0, 0, 1, -1], [0, 0, -1, 1]]) \
        + t * (np.eye(4) - 0.25)
    assert np.abs(Ae[0] - ref).max() < 1e-13
    assert np.allclose(ge[0], fv * h ** 1.5 / 4, atol=1e-14)


def test_global_trace_operator_spd():
    rng = np.random.default_rng(3)
    pr = hdg.HDGProblem(4, 2, np.exp(rng.normal(size=16)), 4.0)
    Aff, *_ = pr.system(np.zeros((9, 16)))
    M = Aff.toarray()
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 1e-6


@pytest.mark.parametrize("n,p", [(2, 1), (2, 2), (4, 1), (4, 2)])
def test_condensed_equals_uncondensed(n, p):
    """Static condensation + recovery equals a dense solve of the full
    (q, u, lambda) system (Sec. 2, last paragraph)."""
    rng = np.random.default_rng(11 + n + p)
    kap = np.exp(rng.normal(size=n * n))
    tau = rng.uniform(0.5, 3.0, size=n * n)
    pr = hdg.HDGProblem(n, p, kap, tau)
    f = rng.normal(size=((p + 1) ** 2, n * n))
    gD = W.dirichlet(lambda x, y: np.cos(x) + y ** 3, n, p)
    lam = pr.solve_direct(f, gD)
    u, q = pr.recover(lam, f)
    lam2, u2, q2 = pr.solve_uncondensed(f, gD)
    assert np.abs(lam - lam2).max() < 1e-11
    assert np.abs(u - u2).max() < 1e-11
    assert np.abs(q - q2).max() < 1e-10


def test_example1_forcing_matches_finite_differences():
    """The hand-derived -lap u of Example I agrees with a 4th-order finite
    difference Laplacian of u = x y exp(x^2 y^3)."""
    x = np.array([0.3, 0.7, 0.91])
    y = np.array([0.2, 0.55, 0.8])
    d = 1e-3
    u = W.ex1_u
    lap = (-u(x + 2 * d, y) + 16 * u(x + d, y) - 30 * u(x, y) + 16 * u(x - d, y) - u(x - 2 * d, y)) / (12 * d * d) \
        + (-u(x, y + 2 * d) + 16 * u(x, y + d) - 30 * u(x, y) + 16 * u(x, y - d) - u(x, y - 2 * d)) / (12 * d * d)
    assert np.allclose(W.ex1_f(x, y), -lap, rtol=1e-7)


def test_direct_solve_orderings_agree():
    """The minimum-degree column ordering used at full size gives the same
    direct solution as SuperLU's default ordering (symmetric HDG and the
    non-symmetric convection-diffusion system)."""
    from paper_1811_09909_gb300 import workloads as W
    wl = W.lognormal(8, 3, seed=5)
    pr = hdg.HDGProblem(8, 3, np.exp(wl.log_kappa), wl.tau())
    a = pr.solve_direct(wl.f[0])
    b = pr.solve_direct(wl.f[0], ordering="MMD_AT_PLUS_A")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    wc = W.convdiff(8, 2, eps=1e-2)
    pc = hdg.HDGProblem(8, 2, np.exp(wc.log_kappa), wc.tau(), beta=wc.beta)
    a = pc.solve_direct(wc.f[0])
    b = pc.solve_direct(wc.f[0], ordering="MMD_AT_PLUS_A")
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
