"""Profiling driver: set-up and solve of the lognormal-coefficient problem on
an n x n mesh of order p (the bench step) a given number of times, with the
solver options named on the command line, so that a profiler sees every
kernel of the step.  With pcg_graph=0 each PCG iteration is launched from the
host, so that the kernel nodes of the iteration appear as separate launches.

  python -m paper_1811_09909_gb300.probes.pcg_step --n 256 --p 4 --reps 2 pcg_graph=0

Prints one line per repetition: the PCG iteration count and the step time
(CUDA events, the step only)."""
import argparse
import json

import torch

from paper_1811_09909_gb300 import hdgmg
from paper_1811_09909_gb300 import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("opts", nargs="*", help="solver options as name=value (integers or floats)")
    a = ap.parse_args()
    kw = dict(coarsest_n=4, m_fine=1, m_growth=2, m_max=2, rtol=1e-10, tau_mode=hdgmg.TAU_OVER_H, tau_c=1.0,
              precision=hdgmg.PREC_FP32)
    for o in a.opts:
        k, v = o.split("=", 1)
        kw[k] = float(v) if "." in v or "e" in v else int(v)
    wl = W.lognormal(a.n, a.p, seed=a.seed)
    dev = torch.device("cuda", 0)
    logk = torch.as_tensor(wl.log_kappa, device=dev)
    f = torch.as_tensor(wl.f[0], device=dev)
    s = hdgmg.Solver(a.n, a.p, **kw)
    lam = torch.empty((1, a.p + 1, 2 * a.n * (a.n + 1)), dtype=torch.float64, device=dev)
    u = torch.empty((1, (a.p + 1) ** 2, a.n * a.n), dtype=torch.float64, device=dev)
    q = torch.empty((1, 2, (a.p + 1) ** 2, a.n * a.n), dtype=torch.float64, device=dev)
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.setup(logk)
        st, info = s.solve_status(f, None, lam, u, q)
        e1.record()
        e1.synchronize()
        if st != 0:
            raise SystemExit(f"solve failed with status {st}")
        print(json.dumps({"iters": info.iters, "step_ms": round(e0.elapsed_time(e1), 3),
                          "launches": info.kernel_launches}), flush=True)
    s.close()


if __name__ == "__main__":
    main()
