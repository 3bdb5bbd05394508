"""GPU tests of blocked multi-right-hand-side solves (opts.rhs_block > 1): FP64
iterative refinement around k simultaneous FP32 PCGs that share every V-cycle,
matvec and vector pass.

Tolerances: every right-hand side's lambda, u and q within 1e-8 relative L2
of the oracle's direct solve and recovery (solved to 1e-12, as the
single-right-hand-side solution tests), and within 1e-8 of the same
right-hand side solved alone; the reported residual is the worst of the
block."""
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


def forcing(n, p, k, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, (p + 1) ** 2, n * n))


@pytest.mark.parametrize("precision,pcycle", [(hdgmg.PREC_FP32_IR, 1), (hdgmg.PREC_FP32, 1),
                                              (hdgmg.PREC_FP32_IR, 0)])
def test_blocked_solve_matches_direct_and_single(precision, pcycle):
    """5 right-hand sides in blocks of 4 (a block of 4, then a block of 1)."""
    n, p, k = 32, 3, 5
    wl = W.lognormal(n, p, seed=21)
    F = forcing(n, p, k, 22)
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-12, precision=precision, pcycle=pcycle,
              tau_mode=hdgmg.TAU_OVER_H)
    sb = hdgmg.Solver(n, p, rhs_block=4, **kw)
    sb.setup(cuda(wl.log_kappa))
    lam, u, q, info = sb.solve(cuda(F))
    assert info.converged == 1 and info.rel_res <= 1e-12, info.as_dict()
    s1 = hdgmg.Solver(n, p, **dict(kw, precision=hdgmg.PREC_FP32_IR))
    s1.setup(cuda(wl.log_kappa))
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau())
    for j in range(k):
        ref = pr.solve_direct(F[j])
        uo, qo = pr.recover(ref, F[j])
        assert rel(host(lam[j]), ref) <= 1e-8, j
        assert rel(host(u[j]), uo) <= 1e-8, j
        assert rel(host(q[j]), qo) <= 1e-8, j
        l1, _, _, i1 = s1.solve(cuda(F[j]), want_u=False, want_q=False)
        assert rel(host(lam[j]), host(l1)) <= 1e-8, j


def test_blocked_solve_with_a_zero_and_dirichlet_data():
    """A zero right-hand side inside a block (solved at once, lambda = 0) and
    Dirichlet data on another (Example I data)."""
    n, p = 16, 2
    wl = W.example1(n, p)
    F = np.stack([wl.f[0], np.zeros_like(wl.f[0]), forcing(n, p, 1, 3)[0]])
    G = np.stack([wl.gD[0], np.zeros_like(wl.gD[0]), np.zeros_like(wl.gD[0])])
    s = hdgmg.Solver(n, p, coarsest_n=2, rtol=1e-12, precision=hdgmg.PREC_FP32_IR, rhs_block=3,
                     tau_mode=hdgmg.TAU_OVER_H)
    s.setup(cuda(wl.log_kappa))
    lam, u, _, info = s.solve(cuda(F), cuda(G), want_q=False)
    assert info.converged == 1
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau())
    for j in (0, 2):
        ref = pr.solve_direct(F[j], G[j])
        assert rel(host(lam[j]), ref) <= 1e-8, j
    assert np.abs(host(lam[1])).max() == 0.0
    assert np.abs(host(u[1])).max() == 0.0


@pytest.mark.parametrize("k", [2, 16])
def test_blocked_cycle_equals_its_right_hand_sides_alone(k):
    """With the blocked layout, right-hand side j's iterate depends on its own
    data only: the first right-hand side solved in a block of k matches it
    solved in a block of one (same kernels, k-independent arithmetic)."""
    n, p = 64, 4
    wl = W.lognormal(n, p, seed=31)
    F = forcing(n, p, k, 32)
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-10, precision=hdgmg.PREC_FP32_IR,
              tau_mode=hdgmg.TAU_OVER_H, rhs_block=k)
    s = hdgmg.Solver(n, p, **kw)
    s.setup(cuda(wl.log_kappa))
    lam, _, _, info = s.solve(cuda(F), want_u=False, want_q=False)
    assert info.converged == 1
    t = hdgmg.Solver(n, p, **dict(kw, rhs_block=2))
    t.setup(cuda(wl.log_kappa))
    lam2, _, _, _ = t.solve(cuda(np.stack([F[0], F[0]])), want_u=False, want_q=False)
    assert rel(host(lam[0]), host(lam2[0])) <= 1e-8


def test_blocked_solve_rejections():
    with pytest.raises(hdgmg.HdgmgError):
        hdgmg.Solver(8, 2, rhs_block=17, precision=hdgmg.PREC_FP32)
    with pytest.raises(hdgmg.HdgmgError):
        hdgmg.Solver(8, 2, rhs_block=4, precision=hdgmg.PREC_FP64)
    with pytest.raises(hdgmg.HdgmgError):
        hdgmg.Solver(8, 2, rhs_block=4, precision=hdgmg.PREC_FP32, krylov=hdgmg.KRYLOV_GMRES)


def test_blocked_batch_problem_equals_alone():
    """A batch with rhs_block: each problem's block solve is the problem's
    own (bit-identical to the same problem solved alone with the cycle the
    batch's contexts run, the launched one)."""
    shapes = [(32, 2), (16, 4), (32, 3)]
    rng = np.random.default_rng(41)
    logks = [cuda(0.5 * rng.standard_normal(n * n)) for n, _ in shapes]
    fs = [cuda(rng.standard_normal((3, (p + 1) ** 2, n * n))) for n, p in shapes]
    opts = dict(coarsest_n=4, m_fine=1, m_max=2, rtol=1e-10, precision=hdgmg.PREC_FP32_IR,
                rhs_block=3)
    b = hdgmg.Batch([dict(n=n, p=p) for n, p in shapes], nthreads=3, **opts)
    b.setup(logks)
    lams, _, _, infos = b.solve(fs, want_u=False, want_q=False)
    for i, (n, p) in enumerate(shapes):
        assert infos[i].converged == 1
        s = hdgmg.Solver(n, p, pcycle=0, **opts)
        s.setup(logks[i])
        lam, _, _, _ = s.solve(fs[i], want_u=False, want_q=False)
        assert np.array_equal(host(lams[i]), host(lam)), i


def test_single_solve_after_blocked_solve_is_unchanged():
    """The blocked and the single-right-hand-side persistent cycles launch
    different grid sizes; each keeps its own barrier count, so a single solve
    after a blocked one in the same context repeats its earlier result bit for
    bit."""
    n, p = 64, 2
    wl = W.lognormal(n, p, seed=23)
    F = forcing(n, p, 4, 24)
    s = hdgmg.Solver(n, p, coarsest_n=4, m_fine=1, m_max=2, rtol=1e-10, precision=hdgmg.PREC_FP32,
                     pcycle=1, rhs_block=4, tau_mode=hdgmg.TAU_OVER_H)
    s.setup(cuda(wl.log_kappa))
    f0 = cuda(F[0])
    la, _, _, ia = s.solve(f0, want_u=False, want_q=False)
    la = host(la).copy()
    for _ in range(3):
        _, _, _, ib = s.solve(cuda(F[:3]), want_u=False, want_q=False)
        assert ib.converged == 1
        lc, _, _, ic = s.solve(f0, want_u=False, want_q=False)
        assert ic.iters == ia.iters
        assert np.array_equal(host(lc), la)
