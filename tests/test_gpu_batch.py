"""Batching layer: independent problems of different size and order, several
right-hand sides each, solved concurrently; every problem must equal the
single-problem path bit for bit and the oracle's direct solve within the
solution tolerance of the suite (1e-8 relative L2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import hdg  # noqa: E402
from paper_1811_09909_gb300 import hdgmg  # noqa: E402

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_batch_matches_single_and_oracle():
    rng = np.random.default_rng(4)
    shapes = [(8, 1), (16, 2), (32, 4), (16, 3), (8, 2), (32, 1)]
    nrhs = 2
    logks = [rng.normal(0.0, 0.5, size=n * n) for n, p in shapes]
    fs = [rng.standard_normal((nrhs, (p + 1) ** 2, n * n)) for n, p in shapes]
    opts = dict(rtol=1e-12, precision=hdgmg.PREC_FP32)
    b = hdgmg.Batch([dict(n=n, p=p) for n, p in shapes], nthreads=4, **opts)
    b.setup([cuda(lk) for lk in logks])
    lams, us, _, infos = b.solve([cuda(f) for f in fs])
    torch.cuda.synchronize()
    for i, (n, p) in enumerate(shapes):
        assert infos[i].converged == 1
        # the batch's contexts run the launched cycle (pcycle = 0): the same
        # problem alone with that cycle gives bit-identical results
        s = hdgmg.Solver(n, p, pcycle=0, **opts)
        s.setup(cuda(logks[i]))
        lam1, u1, _, _ = s.solve(cuda(fs[i]), want_q=False)
        assert torch.equal(lam1, lams[i]) and torch.equal(u1, us[i])
        pr = hdg.HDGProblem(n, p, np.exp(logks[i]), float(n))
        for k in range(nrhs):
            lam_ref = pr.solve_direct(fs[i][k])
            err = np.linalg.norm(lams[i][k].cpu().numpy() - lam_ref) / np.linalg.norm(lam_ref)
            assert err <= 1e-8, (i, k, err)


def test_batch_reports_the_failing_problem():
    b = hdgmg.Batch([dict(n=8, p=2), dict(n=8, p=2)], nthreads=2)
    good = cuda(np.zeros(64))
    bad = cuda(np.full(64, np.nan))
    with pytest.raises(hdgmg.HdgmgError) as ei:
        b.setup([good, bad])
    assert ei.value.status == -5 and "problem 1" in str(ei.value)
