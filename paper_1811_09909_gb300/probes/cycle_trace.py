"""Profiling driver: per-step times of the persistent V-cycle kernel
(hdgmg_trace_vcycle) on the lognormal-coefficient problem, n x n mesh of
order p, FP32 cycle.  Prints, for each barrier of the kernel, the level
(0 = the first P1 level), the step kind and the median time since the
previous barrier over `reps` traced cycles (block 0's global timer).

  python -m paper_1811_09909_gb300.probes.cycle_trace --n 256 --p 4 [name=value ...]"""
import argparse

import numpy as np
import torch

from paper_1811_09909_gb300 import hdgmg
from paper_1811_09909_gb300 import workloads as W

KINDS = ["start", "first sweep", "down sweep", "local corr.", "resid.+restr.", "residual", "restriction",
         "coarsest solve", "prolongation", "up sweep", "tail done", "end"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--reps", type=int, default=9)
    ap.add_argument("opts", nargs="*", help="solver options as name=value (integers)")
    a = ap.parse_args()
    kw = dict(coarsest_n=4, m_fine=1, m_growth=2, m_max=2, rtol=1e-10, tau_mode=hdgmg.TAU_OVER_H, tau_c=1.0,
              precision=hdgmg.PREC_FP32, pcycle=1)
    for o in a.opts:
        k, v = o.split("=", 1)
        kw[k] = int(v)
    wl = W.lognormal(a.n, a.p, seed=2)
    dev = torch.device("cuda", 0)
    s = hdgmg.Solver(a.n, a.p, **kw)
    s.setup(torch.as_tensor(wl.log_kappa, device=dev))
    r = torch.randn((a.p + 1, 2 * a.n * (a.n + 1)), dtype=torch.float64, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(3))
    for _ in range(5):
        s.apply_vcycle(r)
    runs = [s.trace_vcycle(r)[1] for _ in range(a.reps)]
    tags = [t for _, t in runs[0]]
    if any([t for _, t in rec] != tags for rec in runs):
        raise SystemExit("the traced step sequence changed between cycles")
    d = np.median(np.array([[b[0] - c[0] for c, b in zip(rec, rec[1:])] for rec in runs]), axis=0) / 1e3
    total = float(np.median([rec[-1][0] - rec[0][0] for rec in runs])) / 1e3
    print(f"# n={a.n} p={a.p} opts={kw}")
    print(f"# {len(tags) - 1} steps, {total:.2f} us from kernel start to block 0's end (median of {a.reps})")
    print("level,step,us")
    for t, us in zip(tags[1:], d):
        print(f"{t // 16},{KINDS[t % 16]},{us:.2f}")
    s.close()


if __name__ == "__main__":
    main()
