"""The two condensation routes of the symmetric path (Sec. 2 static
condensation) against each other and against the oracle, through the C ABI:
BASIS (one basis diagonalising every element's kappa G + tau E, no factor
stored) and FACTOR (local Cholesky of every element's volume block, factor
kept for the right-hand side and recovery).

Tolerances: element operators 1e-11 max|A| against the oracle and 1e-12
between the routes (two FP64 evaluations of the same Schur complement);
condensed right-hand sides likewise; solutions 1e-8 against the oracle's
direct solve and 1e-10 between the routes (solves to 1e-12)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

ROUTES = {"basis": hdgmg.CONDENSE_BASIS, "factor": hdgmg.CONDENSE_FACTOR}
SCHEME = {"hdg": hdgmg.SCHEME_HDG, "sipg": hdgmg.SCHEME_SIPG}
TAU = {"const": hdgmg.TAU_CONST, "over_h": hdgmg.TAU_OVER_H,
       "kappa_over_h": hdgmg.TAU_KAPPA_OVER_H}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def make(wl, route, scheme="hdg", **opts):
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=TAU[wl.tau_mode], tau_c=wl.tau_c, scheme=SCHEME[scheme],
                     condensation=ROUTES[route], **opts)
    s.setup(cuda(wl.log_kappa))
    return s


CASES = [("hdg", 1, "over_h", 1.0), ("hdg", 4, "over_h", 1.0), ("hdg", 3, "const", 1.0),
         ("hdg", 8, "over_h", 1.0), ("sipg", 2, "kappa_over_h", 12.0), ("sipg", 5, "kappa_over_h", 42.0)]


@pytest.mark.parametrize("scheme,p,mode,c", CASES)
def test_routes_agree_with_each_other_and_the_oracle(scheme, p, mode, c):
    n = 8 if p < 8 else 4
    wl = W.lognormal(n, p, sigma=1.0, seed=60 + p, tau_mode=mode, tau_c=c)
    rng = np.random.default_rng(p)
    f = rng.standard_normal(wl.f[0].shape)
    gD = W.dirichlet(lambda x, y: np.exp(x) * (1 + y), n, p)
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau(), scheme=scheme)
    Ae, _ = pr.condense()
    ref = np.transpose(Ae, (1, 2, 0))
    _, bf, *_ = pr.system(f, gD)
    out = {}
    for route in ROUTES:
        s = make(wl, route, scheme, coarsest_n=n, rtol=1e-12)
        A = host(s.element_matrices(0))
        assert np.abs(A - ref).max() <= 1e-11 * np.abs(ref).max(), route
        b = host(s.condensed_rhs(cuda(f), cuda(gD)))
        b_em = hdg.api_to_edge_major(b, n, p + 1)[pr.free_dofs()]
        assert np.abs(b_em - bf).max() <= 1e-11 * np.abs(bf).max(), route
        lam, u, q, info = s.solve(cuda(f), cuda(gD))
        assert info.converged == 1 and info.condense_kind == ROUTES[route]
        out[route] = (A, host(lam), host(u), host(q))
    Ab, Af = out["basis"][0], out["factor"][0]
    assert np.abs(Ab - Af).max() <= 1e-12 * np.abs(Af).max()
    for k in (1, 2, 3):
        assert rel_l2(out["basis"][k], out["factor"][k]) <= 1e-10, k
    lam_ref = pr.solve_direct(f, gD)
    u_ref, q_ref = pr.recover(lam_ref, f)
    for route in ROUTES:
        assert rel_l2(out[route][1], lam_ref) <= 1e-8
        assert rel_l2(out[route][2], u_ref) <= 1e-8
        assert rel_l2(out[route][3], q_ref) <= 1e-8


def test_auto_picks_basis_where_accurate():
    wl = W.lognormal(8, 2, seed=3)
    s = hdgmg.Solver(8, 2, tau_c=1.0)
    s.setup(cuda(wl.log_kappa))
    _, _, _, info = s.solve(cuda(wl.f[0]))
    assert info.condense_kind == hdgmg.CONDENSE_BASIS
    wl = W.convdiff(8, 2, eps=1e-2)
    s = hdgmg.Solver(8, 2, tau_c=wl.tau_c, beta=wl.beta, krylov=hdgmg.KRYLOV_GMRES)
    s.setup(cuda(wl.log_kappa))
    _, _, _, info = s.solve(cuda(wl.f[0]))
    assert info.condense_kind == hdgmg.CONDENSE_BASIS


@pytest.mark.parametrize("p,eps", [(2, 1e-2), (4, 1e-3), (6, 1e-3)])
def test_nonsymmetric_routes_agree(p, eps):
    """Convection-diffusion: the pencil basis (eps0 = kappa's geometric mean)
    and the local LU give the oracle's element operators, right-hand sides and
    solutions; kappa spread e^N(0, 0.3^2) around eps."""
    n = 8
    wl = W.convdiff(n, p, eps=eps)
    rng = np.random.default_rng(p)
    wl.log_kappa = wl.log_kappa + rng.normal(0.0, 0.3, n * n)
    f = rng.standard_normal(wl.f[0].shape)
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau(), beta=wl.beta)
    Ae, _ = pr.condense()
    ref = np.transpose(Ae, (1, 2, 0))
    _, bf, *_ = pr.system(f)
    lam_ref = pr.solve_direct(f)
    u_ref, q_ref = pr.recover(lam_ref, f)
    out = {}
    for route in ROUTES:
        s = hdgmg.Solver(n, p, tau_c=wl.tau_c, beta=wl.beta, krylov=hdgmg.KRYLOV_GMRES,
                         condensation=ROUTES[route], coarsest_n=2, rtol=1e-12, max_it=300)
        s.setup(cuda(wl.log_kappa))
        A = host(s.element_matrices(0))
        assert np.abs(A - ref).max() <= 1e-10 * np.abs(ref).max(), route
        b = host(s.condensed_rhs(cuda(f)))
        b_em = hdg.api_to_edge_major(b, n, p + 1)[pr.free_dofs()]
        assert np.abs(b_em - bf).max() <= 1e-10 * np.abs(bf).max(), route
        lam, u, q, info = s.solve(cuda(f))
        assert info.converged == 1 and info.condense_kind == ROUTES[route], route
        assert rel_l2(host(lam), lam_ref) <= 1e-8
        assert rel_l2(host(u), u_ref) <= 1e-8
        assert rel_l2(host(q), q_ref) <= 1e-8
        out[route] = A
    assert np.abs(out["basis"] - out["factor"]).max() <= 1e-11 * np.abs(ref).max()


def test_inaccurate_pencil_basis_falls_back_to_lu():
    """IIPG-H with a kappa-independent penalty at p = 4: the eigenvectors of
    the pencil are nearly dependent (the element's symmetries make eigenvalues
    coincide), the set-up's check fails, AUTO falls back to the local LU and
    an explicit BASIS request is EINVAL."""
    n, p = 8, 4
    wl = W.lognormal(n, p, sigma=0.3, seed=5, tau_mode="over_h", tau_c=60.0)
    s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=60.0, scheme=hdgmg.SCHEME_IIPG,
                     krylov=hdgmg.KRYLOV_GMRES, coarsest_n=2, rtol=1e-12)
    s.setup(cuda(wl.log_kappa))
    lam, _, _, info = s.solve(cuda(wl.f[0]))
    assert info.converged == 1
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau(), scheme="iipg")
    assert rel_l2(host(lam), pr.solve_direct(wl.f[0])) <= 1e-8
    kind = info.condense_kind
    s2 = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=60.0, scheme=hdgmg.SCHEME_IIPG,
                      krylov=hdgmg.KRYLOV_GMRES, condensation=hdgmg.CONDENSE_BASIS)
    if kind == hdgmg.CONDENSE_FACTOR:
        with pytest.raises(hdgmg.HdgmgError) as ei:
            s2.setup(cuda(wl.log_kappa))
        assert "EINVAL" in str(ei.value)
    else:                                   # the basis passed its check: it must then be exact
        s2.setup(cuda(wl.log_kappa))
        A = host(s2.element_matrices(0))
        Ae, _ = pr.condense()
        ref = np.transpose(Ae, (1, 2, 0))
        assert np.abs(A - ref).max() <= 1e-10 * np.abs(ref).max()


def test_factor_route_reports_indefinite_blocks():
    """SIPG-H with a tiny penalty: a non-positive Cholesky pivot (FACTOR) and
    a non-positive s_i (BASIS) both end in EBREAKDOWN."""
    wl = W.lognormal(8, 2, sigma=0.5, seed=2, tau_mode="const", tau_c=0.01)
    for route in ROUTES:
        s = hdgmg.Solver(8, 2, tau_mode=hdgmg.TAU_CONST, tau_c=0.01, scheme=hdgmg.SCHEME_SIPG,
                         condensation=ROUTES[route])
        with pytest.raises(hdgmg.HdgmgError) as ei:
            s.setup(cuda(wl.log_kappa))
        assert "EBREAKDOWN" in str(ei.value), route


def test_factor_route_adjoint_matches_basis_route():
    n, p = 8, 3
    wl = W.lognormal(n, p, seed=9)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(wl.f[0].shape)
    u_obs = rng.standard_normal(f.shape)
    g = {}
    for route in ROUTES:
        s = make(wl, route, rtol=1e-13, max_it=300)
        J, gk, gf, _ = s.gradient(cuda(f), cuda(u_obs))
        g[route] = (J, host(gk), host(gf))
    assert abs(g["basis"][0] - g["factor"][0]) <= 1e-10 * abs(g["factor"][0])
    assert rel_l2(g["basis"][1], g["factor"][1]) <= 1e-8
    assert rel_l2(g["basis"][2], g["factor"][2]) <= 1e-8
