"""Examples III and IV of Sec. 4 on quadrilateral meshes (robustness
workloads): the oracle's multigrid against the paper's Example IV tables
(tests/golden/paper_example1_iterations.txt) and the qualitative claims of
Example III.

Reading: kappa is constant per element (K = kappa_e I), sampled at the element
centre.  Example IV's jump line x, y = 0.56 then falls on the fine grid line
nearest to it: at levels 2 and 3 (4 x 4, 8 x 8) on x = 1/2, aligned with every
coarse mesh; from level 4 (x = 9/16, 18/32, 36/64) it cuts coarse
macro-elements, which the DtN coarse operators represent exactly but the P1
macro-edge traces do not.  Levels 2-3 are therefore compared tightly, finer
levels by bounds and by h-robustness of the GMRES counts."""
import numpy as np
import pytest

from oracle import hdg, mg
from paper_1811_09909_gb300 import workloads as W
from conftest import load_paper_table


def _counts(wl, scheme="hdg", gmres=True, solver=True):
    pr = hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau(), scheme=scheme)
    _, bf, *_ = pr.system(wl.f[0], wl.gD[0])
    Hh = mg.Hierarchy(pr, coarsest_n=2, m_fine=3, m_growth=2, local_corr="pre")
    it = it2 = None
    if solver:
        _, it, _, ok = Hh.solve_fixed_point(bf, tol=1e-9, max_it=300)
        it = it if ok else None
    if gmres:
        _, it2, _, ok2 = Hh.solve_gmres(bf, tol=1e-9, max_it=300, left=True)
        it2 = it2 if ok2 else None
    return it, it2


@pytest.mark.parametrize("scheme,section,c", [
    ("hdg", "ex4_hdg_tau_kappa_over_h", lambda p: 1.0),
    ("sipg", "ex4_sipg_tau_kappa", lambda p: float((p + 1) * (p + 2))),
])
def test_example4_counts(scheme, section, c):
    """Example IV, tau proportional to kappa (Tables tab:HDG_discont_k_tau1,
    tab:SIPG_discont_k): levels 2-3 within max(1, 15%) of the table as solver,
    and MG-GMRES no slower than printed (up to 1 iteration; the oracle's
    left-preconditioned GMRES needs up to 3 fewer here); levels 4-6: GMRES
    within 3 of the table and within 2 of each other (h-robust), the MG
    solver converging within 2.5 x the table."""
    table = load_paper_table(section)
    for p in (1, 2, 3):
        gm = []
        for L in (2, 3, 4, 5, 6):
            wl = W.checkerboard(2 ** L, p, tau_mode="kappa_over_h", tau_c=c(p))
            ours = _counts(wl, scheme)
            ref = (table[p][0][L - 2], table[p][1][L - 2])
            assert ours[0] is not None and ours[1] is not None, (p, L)
            if L <= 3:
                assert abs(ours[0] - ref[0]) <= max(1, 0.15 * ref[0]), (scheme, p, L, ours, ref)
                assert ours[1] <= ref[1] + 1, (scheme, p, L, ours, ref)
            else:
                assert ours[1] <= ref[1] + 3, (scheme, p, L, ours, ref)
                assert ours[0] <= 2.5 * ref[0], (scheme, p, L, ours, ref)
                gm.append(ours[1])
        assert max(gm) - min(gm) <= 2, (scheme, p, gm)


def test_example4_gmres_insensitive_to_tau():
    """Table tab:HDG_discont_k_tau23: MG-GMRES with tau = 1/h_min and tau = 1.
    Levels 2-3 within 1 of the table; for p >= 2 every level 2-6 within 3; at
    p = 1 the counts grow and fall with the level as the printed ones do
    (within 5)."""
    table = load_paper_table("ex4_hdg_gmres_tau_over_h_then_tau_one")
    for p in (1, 2, 3):
        for k, mode in enumerate(("over_h", "const")):
            for L in (2, 3, 4, 5, 6):
                wl = W.checkerboard(2 ** L, p, tau_mode=mode, tau_c=1.0)
                _, it = _counts(wl, solver=False)
                ref = table[p][k][L - 2]
                tol = 1 if L <= 3 else (3 if p >= 2 else 5)
                assert it is not None and abs(it - ref) <= tol, (mode, p, L, it, ref)


def test_example3_on_quads():
    """Example III (smooth kappa): IIPG-H with tau = kappa (p+1)(p+2)/h_min
    needs no more MG-solver iterations than HDG with tau = 1 (the paper finds
    slightly fewer) and its MG-GMRES counts are h-independent; HDG tau = 1/h
    and tau = kappa/h give h-independent GMRES counts too."""
    for p in (1, 2, 3):
        iipg, hdg1 = [], []
        for L in (3, 4, 5):
            n = 2 ** L
            iipg.append(_counts(W.example3(n, p, "kappa_over_h", (p + 1) * (p + 2)), "iipg"))
            hdg1.append(_counts(W.example3(n, p, "const", 1.0)))
        assert all(a[0] <= b[0] for a, b in zip(iipg, hdg1)), (p, iipg, hdg1)
        gm = [b for _, b in iipg]
        assert max(gm) - min(gm) <= 1, (p, iipg)
        for mode in ("over_h", "kappa_over_h"):
            gm = [_counts(W.example3(2 ** L, p, mode, 1.0), solver=False)[1] for L in (3, 4, 5)]
            assert max(gm) - min(gm) <= 1 and max(gm) <= 8, (p, mode, gm)


def test_example3_discretisation_error():
    """The smooth-kappa solution converges to u = x y exp(x^2 y^3): the
    element-centre kappa adds an O(h^2) coefficient error, so the L2 error of
    u falls by at least 3.5x per halving of h at p = 2."""
    errs = []
    for n in (8, 16):
        wl = W.example3(n, 2, "over_h", 1.0)
        pr = hdg.HDGProblem(n, 2, np.exp(wl.log_kappa), wl.tau())
        lam = pr.solve_direct(wl.f[0], wl.gD[0])
        u, _ = pr.recover(lam, wl.f[0])
        errs.append(pr.l2_error(u, W.ex1_u))
    assert errs[0] / errs[1] > 3.5, errs
