"""GPU tests of the persistent V-cycle over the P1 levels (opts.pcycle = 2:
in the FP32 and the FP64 cycle; the default 1 keeps the FP64 cycle launched):
Algorithm 1 from the first P1 level to the coarsest and back in one
cooperative launch, the steps separated by grid barriers with bounded waits.

Tolerances:
  * against the oracle's V-cycle (FP64): 1e-10 relative, max norm -- the
    V-cycle tolerance of the suite;
  * against the launched form of the same cycle (pcycle = 0: one kernel per
    step plus the single-block tail): FP64 1e-12, FP32 1e-5 relative.  Both
    forms run the same item arithmetic except on the levels of the
    single-block tail, which forms A e element by element there, so the two
    differ by rounding only;
  * solutions: lambda within 1e-8 of the oracle's direct solve (solved to
    1e-13), the PCG count within one of the launched form's.
An expired wait must come back as HDGMG_ETIMEOUT with the context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg, mg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

LC = {"none": hdgmg.LC_NONE, "pre": hdgmg.LC_PRE, "both": hdgmg.LC_BOTH}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def workload(n, p, seed):
    rng = np.random.default_rng(seed)
    wl = W.lognormal(n, p, sigma=1.0, seed=seed, tau_mode="over_h")
    wl.f = rng.standard_normal(wl.f.shape)
    return wl


def make(wl, **opts):
    s = hdgmg.Solver(wl.n, wl.p, tau_mode=hdgmg.TAU_OVER_H, tau_c=wl.tau_c, **opts)
    s.setup(cuda(wl.log_kappa))
    return s


def rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# tail_n: 0 = every level on the whole grid; 4 / 8 = the levels with n <= 4 / 8
# on block 0; 1000 = the whole cycle on one block
@pytest.mark.parametrize("n,p,lc,m,tail_n", [(16, 2, "both", 1, 0), (16, 2, "both", 1, 4),
                                              (16, 2, "both", 1, 1000), (8, 1, "pre", 2, 16),
                                              (16, 4, "pre", 3, 8), (32, 3, "both", 1, 8),
                                              (8, 2, "none", 2, 0)])
def test_pcycle_vcycle_matches_oracle(n, p, lc, m, tail_n):
    wl = workload(n, p, 41 + p)
    s = make(wl, coarsest_n=2, m_fine=m, local_corr=LC[lc], pcycle=2, pcycle_tail_n=tail_n)
    H = mg.Hierarchy(hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau()), coarsest_n=2, m_fine=m,
                     local_corr=lc)
    rng = np.random.default_rng(9)
    for _ in range(2):                               # two cycles in a row: the barrier re-arms
        r = rng.standard_normal((p + 1, hdg.n_edges(n)))
        e = host(s.apply_vcycle(cuda(r)))
        ref = H.from_free(H.vcycle(H.to_free(r)))
        assert rel_max(e, ref) <= 1e-10


@pytest.mark.parametrize("precision,n,p,tol", [(hdgmg.PREC_FP64, 64, 2, 1e-12),
                                               (hdgmg.PREC_FP32, 64, 4, 1e-5),
                                               (hdgmg.PREC_FP32, 128, 1, 1e-5),
                                               (hdgmg.PREC_BF16, 32, 1, 1e-5),
                                               (hdgmg.PREC_BF16, 32, 3, 1e-5)])
def test_pcycle_matches_launched_cycle(precision, n, p, tol):
    """Same cycle, persistent vs launched; p = 1 with BF16 keeps level 0 (the
    BF16 finest operator) launched and starts the persistent part one level
    below from the restricted residual."""
    wl = workload(n, p, 60 + p)
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, precision=precision)
    a = make(wl, pcycle=2, **kw)
    b = make(wl, pcycle=0, **kw)
    rng = np.random.default_rng(10)
    r = cuda(rng.standard_normal((p + 1, hdg.n_edges(n))))
    ea, eb = host(a.apply_vcycle(r)), host(b.apply_vcycle(r))
    assert rel_max(ea, eb) <= tol


def test_pcycle_nonsymmetric_matches_launched_cycle():
    """Convection-diffusion (full storage, restriction from A_BI)."""
    n, p = 32, 3
    wl = W.convdiff(n, p, eps=1e-2)
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, krylov=hdgmg.KRYLOV_GMRES, local_corr=hdgmg.LC_PRE)
    r = cuda(np.random.default_rng(13).standard_normal((p + 1, hdg.n_edges(n))))
    out = []
    for pc in (2, 0):
        s = hdgmg.Solver(n, p, tau_mode=hdgmg.TAU_OVER_H, tau_c=wl.tau_c, beta=wl.beta, pcycle=pc, **kw)
        s.setup(cuda(wl.log_kappa))
        out.append(host(s.apply_vcycle(r)))
    assert rel_max(out[0], out[1]) <= 1e-12


@pytest.mark.parametrize("precision", [hdgmg.PREC_FP64, hdgmg.PREC_FP32])
def test_pcycle_pcg_solution(precision):
    n, p = 32, 3
    wl = workload(n, p, 70)
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, precision=precision, rtol=1e-13)
    a = make(wl, pcycle=2, **kw)
    b = make(wl, pcycle=0, **kw)
    f = cuda(wl.f[0])
    la, _, _, ia = a.solve(f, want_u=False, want_q=False)
    lb, _, _, ib = b.solve(f, want_u=False, want_q=False)
    assert ia.converged == 1 and abs(ia.iters - ib.iters) <= 1
    assert ia.kernel_launches < ib.kernel_launches
    pr = hdg.HDGProblem(n, p, np.exp(wl.log_kappa), wl.tau())
    ref = pr.solve_direct(wl.f[0])
    assert np.linalg.norm(host(la) - ref) / np.linalg.norm(ref) <= 1e-8


@pytest.mark.parametrize("precision", [hdgmg.PREC_FP64, hdgmg.PREC_FP32])
def test_pcycle_expired_wait_reports_timeout(precision):
    """Every block withholds its arrival at the first barrier: the bounded
    waits run out, the kernel returns, the call reports HDGMG_ETIMEOUT, and the
    next solve gives the same answer as before (barrier and flag reset)."""
    n, p = 64, 2
    wl = workload(n, p, 80)
    s = make(wl, coarsest_n=4, m_fine=1, m_max=2, precision=precision, pcycle=2)
    f = cuda(wl.f[0])
    lam0, _, _, i0 = s.solve(f, want_u=False, want_q=False)
    st = s.lib.hdgmg_check_cycle_timeout(s.ctx, 2000)
    assert st == -6, s.lib.hdgmg_last_error().decode()
    assert "ran out" in s.lib.hdgmg_last_error().decode()
    lam1, _, _, i1 = s.solve(f, want_u=False, want_q=False)
    assert i1.converged == 1 and i1.iters == i0.iters
    assert np.array_equal(host(lam0), host(lam1))
    # a context without the persistent cycle rejects the check
    t = make(wl, coarsest_n=4, pcycle=0)
    assert t.lib.hdgmg_check_cycle_timeout(t.ctx, 2000) == -1


def test_host_driven_pcg_equals_graph_pcg():
    """pcg_graph = 0 launches each PCG iteration from the host (for per-kernel
    profiling): the same kernels in the same order, so the same iterate."""
    n, p = 32, 3
    wl = workload(n, p, 90)
    kw = dict(coarsest_n=4, m_fine=1, m_max=2, precision=hdgmg.PREC_FP32)
    a = make(wl, pcg_graph=1, **kw)
    b = make(wl, pcg_graph=0, **kw)
    f = cuda(wl.f[0])
    la, _, _, ia = a.solve(f, want_u=False, want_q=False)
    lb, _, _, ib = b.solve(f, want_u=False, want_q=False)
    assert ia.iters == ib.iters and ib.converged == 1
    assert np.array_equal(host(la), host(lb))


def test_trace_vcycle_records_every_step():
    """hdgmg_trace_vcycle: the same correction as apply_vcycle, and one
    (time, tag) record per barrier in step order: kernel start first, kernel
    end last, times non-decreasing, one coarsest solve."""
    n, p = 64, 2
    wl = workload(n, p, 95)
    s = make(wl, coarsest_n=4, m_fine=1, m_max=2, precision=hdgmg.PREC_FP32, pcycle=1,
             local_corr=hdgmg.LC_BOTH)
    r = cuda(np.random.default_rng(14).standard_normal((p + 1, hdg.n_edges(n))))
    e0 = host(s.apply_vcycle(r))
    e1, rec = s.trace_vcycle(r)
    assert np.array_equal(e0, host(e1))
    tags = [t for _, t in rec]
    times = [t for t, _ in rec]
    assert tags[0] == 0 and tags[-1] == 11 and len(rec) > 4
    assert all(b >= a for a, b in zip(times, times[1:]))
    assert sum(1 for t in tags if t % 16 == 7) == 1
    # a context without the persistent cycle rejects the call
    t = make(wl, coarsest_n=4, pcycle=0)
    with pytest.raises(hdgmg.HdgmgError):
        t.trace_vcycle(r)
