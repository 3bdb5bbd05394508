"""GPU parity of the hybridized interior penalty schemes (Sec. 2, eq. IPG_H:
SIPG-H, NIPG-H, IIPG-H) against the oracle's primal element and its
multigrid, through the C ABI.

SIPG-H runs the symmetric path (packed operators, eigenbasis condensation, CG);
NIPG-H and IIPG-H the non-symmetric one (full storage, LU condensation,
restriction from A_BI, GMRES), with the scheme's own reference tables.

Tolerances:
  * element operators and right-hand sides: 1e-11 max|A| (FP64, the same
    forms integrated exactly on both sides; the oracle factors the volume
    block with partial pivoting, the GPU without);
  * level operators and one FP64 V-cycle: 1e-10 relative (max norm);
  * solutions: relative L2 error of lambda, u and q <= 1e-8 against the
    oracle's sparse direct solve and recovery (solves to 1e-12);
  * fixed-point counts within one of the oracle's;
  * adjoint gradient (SIPG-H): 1e-6 relative against central differences of
    the oracle's forward map (step 1e-5 in log kappa)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import adjoint, hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

CODE = {"sipg": hdgmg.SCHEME_SIPG, "nipg": hdgmg.SCHEME_NIPG, "iipg": hdgmg.SCHEME_IIPG}
TAU = {"const": hdgmg.TAU_CONST, "over_h": hdgmg.TAU_OVER_H,
       "kappa_over_h": hdgmg.TAU_KAPPA_OVER_H}
LC = {"none": hdgmg.LC_NONE, "pre": hdgmg.LC_PRE, "both": hdgmg.LC_BOTH}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def workload(n, p, sigma=0.7, seed=1, tau_mode="kappa_over_h"):
    """Log-normal kappa with the paper's penalty (p+1)(p+2)/h, proportional to
    kappa_e unless tau_mode says otherwise."""
    return W.lognormal(n, p, sigma=sigma, seed=seed, tau_mode=tau_mode,
                       tau_c=float((p + 1) * (p + 2)))


def solver(wl, scheme, **opts):
    opts.setdefault("krylov", hdgmg.KRYLOV_CG if scheme == "sipg" else hdgmg.KRYLOV_GMRES)
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=TAU[wl.tau_mode], tau_c=wl.tau_c, scheme=CODE[scheme],
                     **opts)
    s.setup(cuda(wl.log_kappa))
    return s


def oracle(wl, scheme):
    return hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau(), scheme=scheme)


@pytest.mark.parametrize("scheme", list(CODE))
@pytest.mark.parametrize("n,p,tau_mode", [(4, 1, "kappa_over_h"), (8, 2, "kappa_over_h"),
                                          (4, 3, "over_h"), (4, 4, "kappa_over_h"),
                                          (2, 6, "kappa_over_h"), (2, 8, "kappa_over_h")])
def test_element_operators_match_oracle(scheme, n, p, tau_mode):
    wl = workload(n, p, seed=10 + p, sigma=0.7 if tau_mode == "kappa_over_h" else 0.2,
                  tau_mode=tau_mode)
    s = solver(wl, scheme, coarsest_n=n)
    A = host(s.element_matrices(0))                          # [nl][nl][E]
    Ae, _ = oracle(wl, scheme).condense()
    ref = np.transpose(Ae, (1, 2, 0))
    assert np.abs(A - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("scheme", list(CODE))
@pytest.mark.parametrize("p", [1, 3])
def test_condensed_rhs_with_dirichlet_lift(scheme, p):
    n = 8
    wl = workload(n, p, seed=3)
    rng = np.random.default_rng(4)
    f = rng.standard_normal(wl.f[0].shape)
    gD = W.dirichlet(lambda x, y: np.exp(x) * (1 + y), n, p)
    s = solver(wl, scheme)
    b = host(s.condensed_rhs(cuda(f), cuda(gD)))
    pr = oracle(wl, scheme)
    _, bf, *_ = pr.system(f, gD)
    b_em = hdg.api_to_edge_major(b, n, p + 1)[pr.free_dofs()]
    assert np.abs(b_em - bf).max() <= 1e-11 * np.abs(bf).max()


@pytest.mark.parametrize("scheme", list(CODE))
def test_level_operators_match_oracle_hierarchy(scheme):
    wl = workload(16, 2, seed=5)
    s = solver(wl, scheme, coarsest_n=2)
    H = mg.Hierarchy(oracle(wl, scheme), coarsest_n=2)
    rng = np.random.default_rng(1)
    assert s.num_levels() == len(H.levels)
    for k, L in enumerate(H.levels):
        x = rng.standard_normal((L.nd, hdg.n_edges(L.n)))
        y = host(s.apply_operator(k, cuda(x)))
        ref = H.from_free(L.A @ H.to_free(x, k), k)
        assert np.abs(y - ref).max() <= 1e-10 * np.abs(ref).max(), k


@pytest.mark.parametrize("scheme", list(CODE))
@pytest.mark.parametrize("n,p,lc,m", [(8, 1, "pre", 1), (16, 2, "both", 1), (8, 3, "pre", 2),
                                      (8, 5, "both", 1)])
def test_vcycle_matches_oracle(scheme, n, p, lc, m):
    wl = workload(n, p, seed=20 + p)
    s = solver(wl, scheme, coarsest_n=2, m_fine=m, local_corr=LC[lc])
    H = mg.Hierarchy(oracle(wl, scheme), coarsest_n=2, m_fine=m, local_corr=lc)
    rng = np.random.default_rng(7)
    r = rng.standard_normal((p + 1, hdg.n_edges(n)))
    e = host(s.apply_vcycle(cuda(r)))
    ref = H.from_free(H.vcycle(H.to_free(r)))
    assert np.abs(e - ref).max() <= 1e-10 * np.abs(ref).max()


def _check_solution(wl, scheme, f, lam, u, q, gD=None):
    pr = oracle(wl, scheme)
    lam_ref = pr.solve_direct(f, gD)
    u_ref, q_ref = pr.recover(lam_ref, f)
    assert rel_l2(lam, lam_ref) <= 1e-8
    assert rel_l2(u, u_ref) <= 1e-8
    assert rel_l2(q, q_ref) <= 1e-8
    return pr


@pytest.mark.parametrize("scheme", list(CODE))
@pytest.mark.parametrize("prec", [hdgmg.PREC_FP64, hdgmg.PREC_FP32])
def test_solution_matches_direct_solve(scheme, prec):
    wl = workload(32, 3, seed=6)
    gD = W.dirichlet(lambda x, y: np.sin(2 * x) + y, 32, 3)
    s = solver(wl, scheme, coarsest_n=4, precision=prec, rtol=1e-12, max_it=300)
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(gD))
    assert info.converged == 1 and info.iters <= 40, info.iters
    _check_solution(wl, scheme, wl.f[0], host(lam), host(u), host(q), gD)


@pytest.mark.parametrize("scheme", list(CODE))
def test_example1_fixed_point_counts_match_oracle(scheme):
    """MG as a solver on Example I with the paper's NIPG-H settings
    (tau = (p+1)(p+2)/h_min, m_N = 3, step-3 correction, tolerance 1e-9)."""
    p, n = 2, 16
    wl = W.example1(n, p, tau_mode="over_h", tau_c=float((p + 1) * (p + 2)))
    s = solver(wl, scheme, krylov=hdgmg.KRYLOV_NONE, local_corr=hdgmg.LC_PRE, m_fine=3,
               coarsest_n=2, rtol=1e-9, max_it=300)
    lam, u, q, info = s.solve(cuda(wl.f[0]), cuda(wl.gD[0]))
    pr = oracle(wl, scheme)
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    H = mg.Hierarchy(pr, coarsest_n=2, m_fine=3, local_corr="pre")
    _, it, _, ok = H.solve_fixed_point(bf, tol=1e-9, max_it=300)
    assert info.converged == 1 and ok
    assert abs(info.iters - it) <= 1, (info.iters, it)
    # the discrete solution approximates the exact one (Example I) to O(h^p)
    assert pr.l2_error(host(u), W.ex1_u) < 1e-3


def test_sipg_gradient_matches_finite_differences():
    """hdgmg_gradient on SIPG-H with tau_e = c kappa_e/h: the derivative in
    log kappa_e includes the penalty's dependence on kappa_e."""
    n, p = 4, 2
    wl = workload(n, p, seed=8)
    rng = np.random.default_rng(9)
    f = rng.standard_normal(wl.f[0].shape)
    u_obs = rng.standard_normal(f.shape)
    s = solver(wl, "sipg", rtol=1e-13, max_it=300)
    J, gk, gf, _ = s.gradient(cuda(f), cuda(u_obs))
    gk = host(gk)

    def J_of(logk):
        pr = hdg.HDGProblem(n, p, np.exp(logk), wl.tau_c * np.exp(logk) * n, scheme="sipg")
        _, u, _ = adjoint.forward(pr, f)
        return adjoint.misfit(pr, u, u_obs)

    h = 1e-5
    for e in (0, 5, 15):
        lp, lm = wl.log_kappa.copy(), wl.log_kappa.copy()
        lp[e] += h
        lm[e] -= h
        fd = (J_of(lp) - J_of(lm)) / (2 * h)
        assert abs(gk[e] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gk).max()), (e, gk[e], fd)


@pytest.mark.parametrize("scheme", ["nipg", "iipg"])
def test_adjoint_rejected_for_nonsymmetric_schemes(scheme):
    wl = workload(4, 1)
    s = solver(wl, scheme)
    with pytest.raises(hdgmg.HdgmgError):
        s.gradient(cuda(wl.f[0]), cuda(wl.f[0]))


def test_batch_mixes_schemes():
    """One batch with HDG, SIPG-H, NIPG-H and IIPG-H problems: each solution
    equals the single-problem solve of the same scheme."""
    probs, data = [], []
    for k, (sch, code) in enumerate([("hdg", hdgmg.SCHEME_HDG), ("sipg", hdgmg.SCHEME_SIPG),
                                     ("nipg", hdgmg.SCHEME_NIPG), ("iipg", hdgmg.SCHEME_IIPG)]):
        wl = workload(16, 2 + k % 2, seed=30 + k)
        probs.append(dict(n=wl.n, p=wl.p, tau_mode=TAU[wl.tau_mode], tau_c=wl.tau_c, scheme=code))
        data.append((sch, wl))
    b = hdgmg.Batch(probs, krylov=hdgmg.KRYLOV_GMRES, coarsest_n=2, rtol=1e-12, max_it=300)
    b.setup([cuda(wl.log_kappa) for _, wl in data])
    lams, _, _, infos = b.solve([cuda(wl.f) for _, wl in data])
    for (sch, wl), lam, info in zip(data, lams, infos):
        assert info.converged == 1, sch
        if sch == "hdg":
            pr = hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau())
            lam_ref = pr.solve_direct(wl.f[0])
        else:
            lam_ref = oracle(wl, sch).solve_direct(wl.f[0])
        assert rel_l2(host(lam)[0], lam_ref) <= 1e-8, sch


def test_indefinite_penalty_is_reported():
    """SIPG-H with a penalty far below (p+1)(p+2)/h: the volume block
    kappa (Kst - N - N^T) + tau E is indefinite, the condensation finds a
    non-positive s_i = kappa g_i + tau e_i and set-up reports EBREAKDOWN."""
    wl = W.lognormal(8, 2, sigma=0.5, seed=2, tau_mode="const", tau_c=0.01)
    s = hdgmg.Solver(8, 2, tau_mode=hdgmg.TAU_CONST, tau_c=0.01, scheme=hdgmg.SCHEME_SIPG)
    with pytest.raises(hdgmg.HdgmgError) as ei:
        s.setup(cuda(wl.log_kappa))
    assert "EBREAKDOWN" in str(ei.value)
