"""Accuracy of local condensation in FP32 followed by FP64 iterative
refinement (the precision layer's reading of Sec. 2's local solves), on the
oracle's element forms:

  * the convection-diffusion element of the 512 x 512, p = 6 workload
    (eps = 1e-3, beta = (1, 0.5), tau_f = eps / h + max(beta.n_f, 0));
  * the diffusion element of the 256 x 256, p = 4 workload (kappa = 1,
    tau = 1 / h).

The local block L (3 nv x 3 nv, unknowns q_x, q_y, u) is solved by LU in
FP32, then refined once: the residual R - L X in FP64, the correction solved
in FP32.  A_e = C X - T is compared with the FP64 solve.  FP32 alone is off
by a few times the FP32 rounding unit (L is well conditioned once the
element size is scaled out); one refinement step brings A_e to the FP64
level, far inside the 1e-11 operator parity.  So accuracy does not rule the
FP32-plus-refinement route out; its cost does: the FP64 residual is a
dense nv x nv by nv x nt product per element on the FP64 pipe."""
import numpy as np

from oracle import hdg


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def refine_once(L, R, C, T):
    A64 = C @ np.linalg.solve(L, R) - T
    L32 = L.astype(np.float32)
    X = np.linalg.solve(L32, R.astype(np.float32)).astype(np.float64)
    e0 = rel(C @ X - T, A64)
    res = R - L @ X                                        # FP64 residual
    X = X + np.linalg.solve(L32, res.astype(np.float32)).astype(np.float64)
    return e0, rel(C @ X - T, A64)


def test_convdiff_element_fp32_then_one_refinement():
    p, n, eps = 6, 512, 1e-3
    h = 1.0 / n
    fr = hdg.ElementForms(p, h, h)
    beta = np.array((1.0, 0.5))
    tau_f = eps / h + np.maximum(fr.normals @ beta, 0.0)
    L, R, C, T = fr.local_cd(eps, tau_f, beta)
    e0, e1 = refine_once(L, R, C, T)
    assert 1e-9 < e0 < 1e-6          # FP32: a few units of 6e-8
    assert e1 < 1e-13                # one FP64 refinement: FP64 level


def test_diffusion_element_fp32_then_one_refinement():
    p, n = 4, 256
    h = 1.0 / n
    fr = hdg.ElementForms(p, h, h)
    tau = 1.0 / h
    L, R, C = fr.local(1.0, tau)
    e0, e1 = refine_once(L, R, C, -tau * fr.El)
    assert 1e-9 < e0 < 1e-6
    assert e1 < 1e-13
