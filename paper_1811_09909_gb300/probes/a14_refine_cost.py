"""Cost of local condensation in FP32 with one FP64 refinement step, against
the FP64 condensation the library runs, on the convection-diffusion workload
(512 x 512 quads, p = 6: nv = 49 volume modes, nt = 28 trace modes,
262,144 elements).

Per element the condensation forms A_e = eps K + diag - V^T S^-1 W with S
(nv x nv) = eps G + S0.  Times, with CUDA events after warm-up:
  * fp64_basis_ms: the library's FP64 condensation (pencil basis, one
    kernel), from hdgmg's own timing of the set-up;
  * fp32_product_ms: the FP32 route's dominant product V^T X (nt x nv by
    nv x nt per element) as a batched cuBLAS SGEMM -- a lower bound for the
    whole FP32 condensation;
  * fp64_residual_ms: one refinement step's FP64 residual W - S X, i.e. the
    product S X (nv x nv by nv x nt per element) with S the same for every
    element here (eps constant), as ONE cuBLAS DGEMM of 49 x 49 by
    49 x (28 x 262,144) -- a lower bound for the refinement step (the
    correction's FP32 solve and the FP64 update of A_e come on top).
The FP32-plus-refinement route costs at least fp32_product_ms +
fp64_residual_ms.

  python -m paper_1811_09909_gb300.probes.a14_refine_cost"""
import json
import statistics

import torch

from paper_1811_09909_gb300 import hdgmg
from paper_1811_09909_gb300 import workloads as W


def timed(fn, reps=5, warmup=2):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def main():
    n, p, eps, beta = 512, 6, 1e-3, (1.0, 0.5)
    nv, nt, E = (p + 1) ** 2, 4 * (p + 1), n * n
    dev = torch.device("cuda", 0)
    wl = W.convdiff(n, p, eps=eps, beta=beta)
    s = hdgmg.Solver(n, p, precision=hdgmg.PREC_FP64, coarsest_n=4, krylov=hdgmg.KRYLOV_GMRES,
                     local_corr=hdgmg.LC_PRE, tau_mode=hdgmg.TAU_OVER_H, tau_c=eps, beta=beta)
    logk = torch.as_tensor(wl.log_kappa, device=dev)
    f = torch.as_tensor(wl.f[0], device=dev)
    cond = []
    for it in range(4):
        s.setup(logk)
        _, _, _, info = s.solve(f, want_u=False, want_q=False)
        if it >= 1:
            cond.append(info.t_condense_ms)
    s.close()
    del s
    torch.cuda.empty_cache()
    g = torch.Generator(device=dev).manual_seed(5)
    # FP32 route's product V^T X per element (batched SGEMM)
    V = torch.randn((E, nt, nv), device=dev, generator=g)
    X = torch.randn((E, nv, nt), device=dev, generator=g)
    torch.backends.cuda.matmul.allow_tf32 = False
    fp32_ms = timed(lambda: torch.bmm(V, X))
    torch.backends.cuda.matmul.allow_tf32 = True
    tf32_ms = timed(lambda: torch.bmm(V, X))
    torch.backends.cuda.matmul.allow_tf32 = False
    del V, X
    torch.cuda.empty_cache()
    # one refinement step's FP64 residual product S X over all elements
    S = torch.randn((nv, nv), dtype=torch.float64, device=dev, generator=g)
    X64 = torch.randn((nv, nt * E), dtype=torch.float64, device=dev, generator=g)
    fp64_ms = timed(lambda: S @ X64)
    flop = 2.0 * nv * nv * nt * E
    print(json.dumps({
        "workload": "convection-diffusion 512x512, p=6 (nv=49, nt=28, 262144 elements)",
        "fp64_basis_ms": round(statistics.mean(cond), 3),
        "fp32_product_ms": round(fp32_ms, 3), "tf32_product_ms": round(tf32_ms, 3),
        "fp64_residual_ms": round(fp64_ms, 3),
        "fp64_residual_tflops": round(flop / (fp64_ms * 1e-3) / 1e12, 3),
        "fp32_plus_refinement_lower_bound_ms": round(fp32_ms + fp64_ms, 3)}))


if __name__ == "__main__":
    main()
