"""Pins of the oracle's convection-diffusion HDG element (the library's
extension of Sec. 2 to -div(eps grad u) + div(beta u) = f, constant beta,
upwind tau_f = tau_e + max(beta.n_f, 0)).

Every check follows from the mathematics, not from the oracle's own formulas:
reduction to the diffusion element at beta = 0, exactness on polynomial
solutions in the discrete spaces (a sign error in any convective term breaks
consistency), the closed form of the element's response to a constant trace,
the energy (positive-definite symmetric part) that the upwind tau guarantees,
optimal O(h^{p+1}) rates for u, and the uncondensed brute-force solve."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import hdg, mg
from paper_1811_09909_gb300 import workloads as W

BETA = (1.0, 0.5)


def _edge_coeffs(fun, n, p, nq=12):
    """Orthonormal-Legendre coefficients of fun on every edge (unit square)."""
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


def _problem(n, p, eps, tau_c=1.0, beta=BETA, seed=None):
    kap = eps if seed is None else eps * np.exp(np.random.default_rng(seed).normal(0, 0.3, n * n))
    return hdg.HDGProblem(n, p, kap, tau_c * n, beta=beta)


def test_zero_velocity_reduces_to_diffusion():
    n, p = 4, 3
    rng = np.random.default_rng(1)
    kap = np.exp(rng.normal(size=n * n))
    f = rng.standard_normal(((p + 1) ** 2, n * n))
    a = hdg.HDGProblem(n, p, kap, 2.5)
    b = hdg.HDGProblem(n, p, kap, 2.5, beta=(0.0, 0.0))
    Aa, ga = a.condense(f)
    Ab, gb = b.condense(f)
    assert np.abs(Aa - Ab).max() <= 1e-13 * np.abs(Aa).max()
    assert np.abs(ga - gb).max() <= 1e-13 * np.abs(ga).max()


@pytest.mark.parametrize("p,eps", [(1, 1.0), (1, 1e-3), (2, 0.05), (3, 1e-3)])
def test_patch_exact_with_convection(p, eps):
    """u linear (p = 1) or quadratic (p >= 2): q = -eps grad u,
    f = -eps lap u + beta.grad u is reproduced exactly, with lambda the exact
    trace on every edge (interior ones included)."""
    bx, by = BETA
    if p == 1:
        uf = lambda x, y: 1.0 + 2.0 * x - 3.0 * y            # noqa: E731
        gx, gy = (lambda x, y: 2.0 + 0 * x), (lambda x, y: -3.0 + 0 * x)
        ff = lambda x, y: bx * 2.0 - by * 3.0 + 0 * x          # noqa: E731
    else:
        uf = lambda x, y: x ** 2 + x * y - 2 * y ** 2          # noqa: E731
        gx, gy = (lambda x, y: 2 * x + y), (lambda x, y: x - 4 * y)
        ff = lambda x, y: -eps * (2.0 - 4.0) + bx * (2 * x + y) + by * (x - 4 * y)   # noqa: E731
    n = 4
    pr = _problem(n, p, eps)
    f = W.nodal(ff, n, p)
    gD = W.dirichlet(uf, n, p)
    lam = pr.solve_direct(f, gD)
    u, q = pr.recover(lam, f)
    X, Y = pr.node_coords()
    scale = 1.0 + np.abs(uf(X, Y)).max()
    assert np.abs(u - uf(X, Y)).max() < 1e-11 * scale
    assert np.abs(q[0] + eps * gx(X, Y)).max() < 1e-10 * scale
    assert np.abs(q[1] + eps * gy(X, Y)).max() < 1e-10 * scale
    assert np.abs(lam - _edge_coeffs(uf, n, p)).max() < 1e-11 * scale


@pytest.mark.parametrize("p", [1, 2, 4])
def test_constant_trace_closed_form(p):
    """lambda = 1, f = 0 has the local solution u = 1, q = 0 (beta is
    divergence-free), so the element's conservation rows give <beta.n, mu>:
    (beta.n_f) sqrt(|e_f|) on mode 0 of face f, zero else.  The trace
    operator is minus these rows (A_e lambda = g_e - flux rows, the sign that
    makes the diffusion part positive), so A_e 1 = -<beta.n, mu>."""
    n, eps = 3, 0.02
    pr = _problem(n, p, eps, seed=3)
    Ae, _ = pr.condense()
    h = 1.0 / n
    bn = np.array([-BETA[0], BETA[0], -BETA[1], BETA[1]])
    want = np.zeros(4 * (p + 1))
    want[0::p + 1] = -bn * np.sqrt(h)
    one = np.zeros(4 * (p + 1))
    one[0::p + 1] = np.sqrt(h)                  # the constant 1 on every face
    resp = Ae @ one
    assert np.abs(resp - want[None]).max() < 1e-12 * np.abs(Ae).max()
    # and the operator is genuinely non-symmetric
    assert np.abs(Ae - np.transpose(Ae, (0, 2, 1))).max() > 1e-3 * np.abs(Ae).max()


@pytest.mark.parametrize("eps", [1e-3, 0.1])
def test_upwind_tau_gives_positive_definite_symmetric_part(eps):
    """Energy: lambda^T A lambda = sum_K [ eps^-1 |q|^2 + <(tau - beta.n/2)(u - lambda)^2> ]
    > 0 for interior traces (the beta.n lambda^2 terms cancel across edges),
    because tau_f - beta.n_f / 2 >= tau_e > 0."""
    pr = _problem(6, 2, eps, tau_c=eps)
    Aff, *_ = pr.system(np.zeros((9, 36)))
    A = Aff.toarray()
    sym = 0.5 * (A + A.T)
    assert np.linalg.eigvalsh(sym).min() > 0.0
    # without the upwind part the same mesh is not coercive for small eps
    if eps == 1e-3:
        bad = hdg.HDGProblem(6, 2, eps, eps * 6, beta=BETA)
        bad.tau_f = np.repeat(bad.tau[:, None], 4, axis=1)
        Ab, *_ = bad.system(np.zeros((9, 36)))
        Ab = Ab.toarray()
        assert np.linalg.eigvalsh(0.5 * (Ab + Ab.T)).min() < 0.0


@pytest.mark.parametrize("p", [1, 2])
def test_convergence_rates_u(p):
    eps = 0.1
    errs = []
    for n in (4, 8, 16):
        pr = _problem(n, p, eps, tau_c=eps)
        f = W.nodal(W.convdiff_f(eps, BETA), n, p)
        lam = pr.solve_direct(f)
        u, _ = pr.recover(lam, f)
        errs.append(pr.l2_error(u, W.sine_u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() >= p + 0.8, rates


def test_condensed_equals_uncondensed():
    n, p, eps = 4, 2, 0.01
    pr = _problem(n, p, eps, seed=5)
    rng = np.random.default_rng(9)
    f = rng.standard_normal(((p + 1) ** 2, n * n))
    gD = W.dirichlet(lambda x, y: np.cos(x) + y, n, p)
    lam = pr.solve_direct(f, gD)
    u, q = pr.recover(lam, f)
    lam2, u2, q2 = pr.solve_uncondensed(f, gD)
    assert np.abs(lam - lam2).max() < 1e-10 * np.abs(lam).max()
    assert np.abs(u - u2).max() < 1e-10 * np.abs(u).max()
    assert np.abs(q - q2).max() < 1e-10 * np.abs(q).max()


def test_nonsymmetric_galerkin_hierarchy():
    """A_{k-1} = J^T (A_BB - A_BI A_II^-1 A_IB) J against the dense global
    Schur complement (Proposition DtN holds without symmetry), and Q != I^T."""
    n, p = 8, 1
    pr = _problem(n, p, 0.01, seed=2)
    H = mg.Hierarchy(pr, coarsest_n=2, dirichlet=False)
    L0, L1 = H.levels[0], H.levels[1]
    A = L0.A.toarray()
    Iset, Bset = L0.Iset, np.setdiff1d(np.arange(A.shape[0]), L0.Iset)
    S = A[np.ix_(Bset, Bset)] - A[np.ix_(Bset, Iset)] @ np.linalg.solve(A[np.ix_(Iset, Iset)],
                                                                       A[np.ix_(Iset, Bset)])
    J = L0.I.toarray()[Bset]
    assert np.abs(J.T @ S @ J - L1.A.toarray()).max() < 1e-11 * np.abs(A).max()
    assert np.abs(L0.Q.toarray() - L0.I.toarray().T).max() > 1e-3


def test_mg_gmres_converges_for_small_eps():
    """The multigrid-preconditioned GMRES of Sec. 4 on the non-symmetric
    system (eps = 1e-3, mesh Peclet ~ 35 at n = 32): converges and matches the
    direct solve."""
    wl = W.convdiff(32, 2, eps=1e-3)
    pr = hdg.HDGProblem(32, 2, np.exp(wl.log_kappa), wl.tau(), beta=wl.beta)
    Aff, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=2, m_fine=1, local_corr="pre")
    x, it, _, ok = H.solve_gmres(bf, tol=1e-10, max_it=200, left=False)
    assert ok and it < 60, it
    lam = pr.solve_direct(wl.f[0], wl.gD[0])
    ref = hdg.api_to_edge_major(lam, 32, 3)[pr.free_dofs()]
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
