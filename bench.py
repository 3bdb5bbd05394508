"""Benchmark: HDG trace DOFs solved per second to 1e-10 relative residual.

One step = the whole hot path on one synthetic problem: element condensation,
block-Jacobi blocks, p-coarsening and every 2x2 agglomeration level, coarsest
factorisation, condensed right-hand side, V-cycle-preconditioned CG to
||g - A lambda|| / ||g|| <= 1e-10 (checked in FP64), and recovery of u and q.

Workload: 256 x 256 quads on [0,1]^2, p = 4, per-element log kappa iid N(0,1)
(seed 2), f = 1, g_D = 0, tau = 1/h (652,800 interior trace DOFs).  Two arms are
timed: the mixed form (FP32 V-cycle inside FP64 CG, FP64 condensation and
outer residual) -- the headline -- and the plain FP64 form.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch under torch.distributed.run: every rank solves its own
instance (replicas, weak scaling); value = all ranks' DOFs / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HDG trace DOFs solved/s to 1e-10 rel res, mixed vs FP64; V-cycle HBM GB/s"
UNIT = "trace DOFs/s"
N_MESH, P_ORDER, SEED = 256, 4, 2
SAMPLE_N = 128          # oracle sample: same recipe on a 128 x 128 mesh
L2_FLUSH_BYTES = 512 << 20
# symmetric V(1,1): m_N = 1 doubling per level up to 4, local correction in
# steps 3 and 5, coarsest level 4 x 4 macro-elements (48 DOFs, dense Cholesky)
SOLVER_OPTS = dict(coarsest_n=4, m_fine=1, m_growth=2, m_max=4, rtol=1e-10)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--arm", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def workload_config(n=N_MESH):
    return {"workload": f"variable-coefficient diffusion {n}x{n} quads, p={P_ORDER}, "
                        f"log kappa iid N(0,1) seed {SEED}, f=1, g_D=0, tau=1/h",
            "mesh": n, "p": P_ORDER, "interior_trace_dofs": 2 * n * (n - 1) * (P_ORDER + 1),
            "rtol": 1e-10, "krylov": "PCG with the symmetric V-cycle (m_N=1, m doubling per level "
                                     "capped at 4, local correction steps 3+5, coarsest 4x4 dense)",
            "l2": "flushed between steps (512 MiB write)"}


# ---------------------------------------------------------------- oracle leg
def oracle_sample_run():
    """One oracle pass over the sample problem; prints seconds and DOFs."""
    import numpy as np
    from oracle import hdg, mg
    from paper_1811_09909_gb300 import workloads as W
    wl = W.lognormal(SAMPLE_N, P_ORDER, seed=SEED)
    t0 = time.perf_counter()
    pr = hdg.HDGProblem(wl.n, wl.p, np.exp(wl.log_kappa), wl.tau())
    Ae, ge = pr.condense(wl.f[0])
    A = pr.assemble(Ae)
    g = pr.assemble_rhs(ge)
    fd = pr.free_dofs()
    bf = g[fd]
    H = mg.Hierarchy(pr, Ae=Ae, coarsest_n=2, m_fine=1, local_corr="both")
    x, it, _, ok = H.solve_pcg(bf, tol=1e-10)
    lam = np.zeros(pr.ne * pr.nd)
    lam[fd] = x
    pr.recover(hdg.edge_major_to_api(lam, wl.n, wl.p + 1), wl.f[0])
    dt = time.perf_counter() - t0
    res = float(np.linalg.norm(bf - A[fd][:, fd] @ x) / np.linalg.norm(bf))
    print(json.dumps({"seconds": dt, "dofs": wl.interior_trace_dofs, "iters": it, "ok": bool(ok),
                      "rel_res": res}))


def run_oracle_subprocess():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_obj(runs):
    v = statistics.mean(r["dofs"] / r["seconds"] for r in runs)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"full pipeline (condensation, hierarchy, PCG to 1e-10, recovery) of the "
                      f"oracle on the same recipe at {SAMPLE_N}x{SAMPLE_N}, p={P_ORDER} "
                      f"({2 * SAMPLE_N * (SAMPLE_N - 1) * (P_ORDER + 1)} DOFs), single thread, "
                      f"{len(runs)} run(s), mean {statistics.mean(r['seconds'] for r in runs):.2f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        run_oracle_subprocess()
    runs = [run_oracle_subprocess() for _ in range(args.steps)]
    ms = statistics.mean(r["seconds"] for r in runs) * 1e3
    cb = cpu_baseline_obj(runs)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(SAMPLE_N), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# -------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.proc = None
        self.dev = dev_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={dev_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            tok = [t.strip() for t in line.split(",")]
            if len(tok) < 9:
                continue
            try:
                sm.append(float(tok[1]))
                smax.append(float(tok[2]))
            except ValueError:
                continue
            for nm, val in zip(names, tok[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- GPU leg
def run_ours(args):
    import numpy as np
    import torch
    from paper_1811_09909_gb300 import hdgmg
    from paper_1811_09909_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    wl = W.lognormal(N_MESH, P_ORDER, seed=SEED + 1000 * rank)
    logk = torch.as_tensor(wl.log_kappa, device=dev)
    f = torch.as_tensor(wl.f[0], device=dev)
    nd, ne, nv, E = P_ORDER + 1, 2 * N_MESH * (N_MESH + 1), (P_ORDER + 1) ** 2, N_MESH * N_MESH
    lam = torch.empty((1, nd, ne), dtype=torch.float64, device=dev)
    u = torch.empty((1, nv, E), dtype=torch.float64, device=dev)
    q = torch.empty((1, 2, nv, E), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    common = dict(tau_mode=hdgmg.TAU_OVER_H, tau_c=1.0, stream=stream, **SOLVER_OPTS)
    arms = {"mixed": hdgmg.Solver(N_MESH, P_ORDER, precision=hdgmg.PREC_FP32, **common),
            "fp64": hdgmg.Solver(N_MESH, P_ORDER, precision=hdgmg.PREC_FP64, **common)}
    if args.arm != "both":
        arms = {args.arm: arms[args.arm]}

    def step(solver):
        solver.setup(logk)
        st, info = solver.solve_status(f, None, lam, u, q)
        if st != 0:
            raise RuntimeError(f"solve failed with status {st}: {info.as_dict()}")
        return info

    results = {}
    for name, s in arms.items():
        for _ in range(args.warmup):
            step(s)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        times, infos = [], []
        clocks = ClockSampler(dev.index) if name == "mixed" else None
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step(s)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall0
        if dist:
            dist.barrier()
        ck = clocks.stop() if clocks else None
        tot = torch.tensor([sum(times)], device=dev, dtype=torch.float64)
        if dist:
            dist.all_reduce(tot, op=dist.ReduceOp.MAX)
        ms = float(tot.item()) / args.steps
        worst = max(i.rel_res for i in infos)
        assert all(i.converged for i in infos) and worst <= 1e-10, worst
        results[name] = {"ms": ms, "iters": infos[-1].iters, "rel_res": worst,
                         "setup_ms": infos[-1].t_setup_ms, "solve_ms": infos[-1].t_solve_ms,
                         "clocks": ck, "wall_s": wall,
                         "launches": sum(i.kernel_launches for i in infos)}

    dofs = wl.interior_trace_dofs
    if args.arm != "both":
        r = results[args.arm]
        if rank == 0:
            return {"arm": args.arm, "ms_per_step": r["ms"], "iters": r["iters"],
                    "rel_res": r["rel_res"], "gpu_launches": r["launches"]}
        return None
    mixed, fp64 = results["mixed"], results["fp64"]
    value = dofs * world / (mixed["ms"] * 1e-3)

    # end to end through the C ABI on pinned host buffers (mixed arm)
    s = arms["mixed"]
    if args.no_e2e:
        args.warmup, args.steps = 0, 1
    h_logk = torch.as_tensor(wl.log_kappa).pin_memory()
    h_f = torch.as_tensor(wl.f[0]).pin_memory()
    h_lam = torch.empty((nd, ne), dtype=torch.float64).pin_memory()
    h_u = torch.empty((nv, E), dtype=torch.float64).pin_memory()
    h_q = torch.empty((2, nv, E), dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        s.run_host(h_logk, h_f, None, h_lam, h_u, h_q)
    e2e_t = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = s.run_host(h_logk, h_f, None, h_lam, h_u, h_q)
        e2e_t.append(time.perf_counter() - t0)
        assert st == 0 and info.rel_res <= 1e-10
    h2d = 8 * (E + nv * E)
    d2h = 8 * (nd * ne + nv * E + 2 * nv * E)
    e2e = {"value": dofs * world / statistics.mean(e2e_t), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 condensation+outer CG, f32 V-cycle", "data": "synthetic",
                "config": workload_config(),
                "fp64": {"value": dofs * world / (fp64["ms"] * 1e-3), "ms_per_step": fp64["ms"],
                         "iters": fp64["iters"], "rel_res": fp64["rel_res"],
                         "setup_ms": fp64["setup_ms"], "solve_ms": fp64["solve_ms"]},
                "mixed": {"iters": mixed["iters"], "rel_res": mixed["rel_res"],
                          "setup_ms": mixed["setup_ms"], "solve_ms": mixed["solve_ms"]},
                "clocks": mixed["clocks"], "e2e": e2e, "gpu_launches": mixed["launches"]}
    return line


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_run()
        return
    if args.impl == "reference":
        run_reference(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    line = run_ours(args)
    if rank == 0:
        if (not args.no_cpu_baseline and args.arm == "both"
                and int(os.environ.get("WORLD_SIZE", "1")) == 1):
            line["cpu_baseline"] = cpu_baseline_obj([run_oracle_subprocess()])
        print(json.dumps(line))


if __name__ == "__main__":
    main()
