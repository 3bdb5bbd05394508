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
# symmetric V(1,1): m_N = 1 doubling per level up to 2, local correction in
# steps 3 and 5, coarsest level 4 x 4 macro-elements (48 DOFs, dense inverse)
SOLVER_OPTS = dict(coarsest_n=4, m_fine=1, m_growth=2, m_max=2, rtol=1e-10)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--arm", default="both", choices=["both", "mixed", "fp64", "mixed_matrix_free"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (64 problems x 16 RHS), adjoint (1024^2) and "
                         "convection-diffusion (512^2, p=6) lines")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def workload_config(n=N_MESH):
    return {"workload": f"variable-coefficient diffusion {n}x{n} quads, p={P_ORDER}, "
                        f"log kappa iid N(0,1) seed {SEED}, f=1, g_D=0, tau=1/h",
            "mesh": n, "p": P_ORDER, "interior_trace_dofs": 2 * n * (n - 1) * (P_ORDER + 1),
            "rtol": 1e-10, "krylov": "PCG with the symmetric V-cycle (m_N=1, m doubling per level "
                                     "capped at 2, local correction steps 3+5, coarsest 4x4 dense)",
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
        """Start nvidia-smi sampling every 100 ms and return once its first
        sample has arrived, so that the timed region that follows is covered."""
        import threading
        self.proc = None
        self.dev = dev_index
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={dev_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line)
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
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
    from paper_1811_09909_gb300 import hdgmg, replicas
    from paper_1811_09909_gb300 import workloads as W

    rank, world, local = replicas.rank_info()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    wl = W.lognormal(N_MESH, P_ORDER, seed=replicas.replica_seed(SEED, rank))
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
            "fp64": hdgmg.Solver(N_MESH, P_ORDER, precision=hdgmg.PREC_FP64, **common),
            "mixed_matrix_free": hdgmg.Solver(N_MESH, P_ORDER, precision=hdgmg.PREC_FP32,
                                              matrix_free=1, **common)}
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
        ms = replicas.max_over_ranks(sum(times), dist, device=dev) / args.steps
        worst = max(i.rel_res for i in infos)
        assert all(i.converged for i in infos) and worst <= 1e-10, worst
        results[name] = {"ms": ms, "iters": infos[-1].iters, "rel_res": worst,
                         "setup_ms": infos[-1].t_setup_ms, "solve_ms": infos[-1].t_solve_ms,
                         "clocks": ck, "wall_s": wall,
                         "launches": sum(i.kernel_launches for i in infos),
                         "condense_ms": statistics.mean(i.t_condense_ms for i in infos)}

    dofs = wl.interior_trace_dofs
    if args.arm != "both":
        r = results[args.arm]
        if rank == 0:
            return {"arm": args.arm, "ms_per_step": r["ms"], "iters": r["iters"],
                    "rel_res": r["rel_res"], "gpu_launches": r["launches"]}
        return None
    mixed, fp64, mfree = results["mixed"], results["fp64"], results["mixed_matrix_free"]
    value = replicas.whole_job_rate(dofs, world, mixed["ms"])

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
    e2e_s = replicas.max_over_ranks(statistics.mean(e2e_t), dist, device=dev)
    e2e = {"value": dofs * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": mixed["ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 condensation+outer CG, f32 V-cycle", "data": "synthetic",
                "config": workload_config(),
                "fp64": {"value": replicas.whole_job_rate(dofs, world, fp64["ms"]),
                         "ms_per_step": fp64["ms"],
                         "iters": fp64["iters"], "rel_res": fp64["rel_res"],
                         "setup_ms": fp64["setup_ms"], "solve_ms": fp64["solve_ms"]},
                "mixed_matrix_free": {
                    "value": replicas.whole_job_rate(dofs, world, mfree["ms"]),
                    "ms_per_step": mfree["ms"], "iters": mfree["iters"], "rel_res": mfree["rel_res"],
                    "note": "the mixed arm with the V-cycle's FP32 finest-level matvecs applied "
                            "matrix-free through the eigenbasis (opts.matrix_free)"},
                "mixed": {"iters": mixed["iters"], "rel_res": mixed["rel_res"],
                          "setup_ms": mixed["setup_ms"], "solve_ms": mixed["solve_ms"],
                          "solve_only_value": replicas.whole_job_rate(dofs, world,
                                                                      mixed["solve_ms"])},
                "clocks": mixed["clocks"], "e2e": e2e, "gpu_launches": mixed["launches"],
                "roofline": roofline_pcg(arms["mixed"], mixed),
                "roofline_condense": roofline_condense(mixed["condense_ms"]),
                "vcycle": vcycle_bandwidth(arms["mixed"], dev)}
    return line


# ------------------------------------------------------------- roofline
def hbm_peak():
    """HBM copy bandwidth measured on this machine's GPUs (the driver writes it
    next to this file); the recipe's earlier single measurement otherwise."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk
# x 2 flop x 2.07 GHz; a throughput probe on the box measured 1.20 TFLOP/s
# for FP64 FMA and 1.06 for FP64 MMA (mma.sync m8n8k4), so the FP64 set-up
# runs on the FMA pipe (paper_1811_09909_gb300/probes/mma_rate.cu).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM traffic of one condensation launch at 256^2, p = 4: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of the current kernel
# (576 KB read, 54.0 MB written); None until captured for this kernel.
CONDENSE_TRAFFIC_BYTES = 576512 + 54012416
# DRAM traffic of one PCG iteration at 256^2, p = 4, mixed form: ncu
# dram__bytes_read.sum + dram__bytes_write.sum summed over the kernels of one
# iteration (host-driven loop, warm L2, average of 56 iterations of the
# 256 x 256, p = 4 step): persistent cycle 51.2 MB, fused FP64 matvec 131.9,
# two FP32 finest matvecs 121.2, update 15.8, the two block-Jacobi steps
# 19.6 + 7.9.  Below the algorithmic bytes because the persistent cycle's
# steps re-read their level operators from L2.
PCG_ITER_TRAFFIC_BYTES = 347.69e6


def condense_flops(p, nE):
    """Algorithmic flops of K1 per launch in the basis that diagonalises every
    volume block: s_i = kappa g_i + tau e_i (n_v FMAs), U = s^-1/2 (kappa P +
    tau Q) (n_v n_t entries, 3 flops each), A_e = kappa K + tau I - U^T U
    (n_t (n_t + 1) / 2 packed entries, n_v FMAs each, plus the kappa K term).
    At p = 4 this is 12.5 kflop per element, 3.2x fewer than the block
    elimination count n_v^3/3 + 2 n_v^2 n_t + n_t^2 n_v = 40.2 kflop that the
    per-element factorisation route needs."""
    nv, nt = (p + 1) ** 2, 4 * (p + 1)
    nsa = nt * (nt + 1) // 2
    return (2.0 * nv + 3.0 * nv * nt + 2.0 * nsa * (nv + 1)) * nE


def roofline_condense(ms):
    flops = condense_flops(P_ORDER, N_MESH * N_MESH)
    achieved = flops / (ms * 1e-3) / 1e12
    nv, nt = (P_ORDER + 1) ** 2, 4 * (P_ORDER + 1)
    elim = (nv ** 3 / 3 + 2 * nv * nv * nt + nt * nt * nv) * N_MESH * N_MESH
    return {"kernel": "condense_eig_kernel (element condensation, FP64)", "bound": "alu",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": CONDENSE_TRAFFIC_BYTES,
            "algorithmic_flops_per_launch": flops, "launch_ms": ms,
            "flop_count": "eigenbasis route, 12.5 kflop per element at p=4; the block-elimination "
                          "count of the factorisation route (40.2 kflop per element) would read "
                          f"{elim / (ms * 1e-3) / 1e12:.2f} TFLOP/s for the same launch",
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (probe on the box: "
                           "1.20 TFLOP/s FP64 FMA, 1.06 FP64 MMA)"}


def pcg_iteration_bytes(solver):
    """Algorithmic HBM bytes of one mixed PCG iteration: the FP32 V-cycle
    (vcycle_bytes), the FP64 outer matvec (packed operator once, p read, A p
    read and written) and the CG vector passes of the fused kernels (r.z,
    p = z + beta p, p.Ap, x += alpha p with r -= alpha Ap and the FP32 copy of r):
    108 bytes per trace value."""
    n, nd = solver.level_shape(0)
    nE, ned = n * n, 2 * n * (n + 1)
    nsym = 4 * nd * (4 * nd + 1) // 2
    vals = nd * ned
    matvec64 = nsym * nE * 8 + 3 * vals * 8
    cg = 108 * vals
    return vcycle_bytes(solver) + matvec64 + cg, matvec64, cg


def roofline_pcg(solver, info):
    peak, src = hbm_peak()
    b, mv, cg = pcg_iteration_bytes(solver)
    it_ms = info["solve_ms"] / max(info["iters"], 1)
    achieved = b / (it_ms * 1e-3) / 1e9
    return {"kernel": "PCG iteration: FP32 V-cycle (pcycle_kernel over the P1 levels, fine-level "
                      "matvec and block-Jacobi kernels) + FP64 outer matvec + fused CG updates",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": PCG_ITER_TRAFFIC_BYTES,
            "algorithmic_bytes_per_iteration": b, "fp64_matvec_bytes": mv, "cg_vector_bytes": cg,
            "iteration_ms": it_ms,
            "peak_source": f"{src} HBM copy bandwidth",
            "note": "iteration time = CUDA-event solve time of the library / iterations (the solve "
                    "also holds the right-hand side, the final FP64 residual and the recovery)"}


def vcycle_bytes(solver):
    """Algorithmic HBM bytes of one FP32 V-cycle application: every operator,
    block-Jacobi inverse and transfer block read once per use, every trace
    vector read/written once per kernel that touches it."""
    nl = solver.num_levels()
    o = solver.opts
    total = 0.0
    m = o.m_fine
    for k in range(nl - 1):
        n, nd = solver.level_shape(k)
        nE, ned = n * n, 2 * n * (n + 1)
        nsym = 4 * nd * (4 * nd + 1) // 2
        vec = nd * ned * 4
        matvecs = (m - 1) + 1 + m
        sweeps = 2 * m
        total += matvecs * (nsym * nE * 4 + 3 * vec)
        total += sweeps * (nd * (nd + 1) // 2 * ned * 4 + 3 * vec)
        if nd == 2 and k + 1 < nl:
            nC = nE // 4
            lcs = 2 if o.local_corr == 2 else (1 if o.local_corr == 1 else 0)
            total += lcs * (164 * nC * 4 + 2 * vec)
            total += 2 * (64 * nC * 4 + 2 * vec)
        else:
            total += 4 * vec
        m = min(m * o.m_growth, o.m_max) if o.m_max else m * o.m_growth
    return total


def vcycle_bandwidth(solver, dev, reps=20):
    import torch
    r = torch.randn((P_ORDER + 1, 2 * N_MESH * (N_MESH + 1)), dtype=torch.float64, device=dev)
    for _ in range(3):
        solver.apply_vcycle(r)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        solver.apply_vcycle(r)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    b = vcycle_bytes(solver)
    gbs = b / (ms * 1e-3) / 1e9
    peak, src = hbm_peak()
    return {"ms": ms, "algorithmic_bytes": b, "achieved_gbs": gbs,
            "hbm_peak_gbs": peak, "peak_source": src, "frac": gbs / peak,
            "note": "one FP32 V-cycle through hdgmg_apply_vcycle (fine level launched, the P1 levels "
                    "in one persistent cooperative launch; FP64<->FP32 conversions of r and e "
                    "included); the L2-resident coarse levels keep it latency-bound"}


# ------------------------------------------------------- extra workloads
def run_batched(dev, steps, warmup):
    """64 independent problems, n in {32,64,128,256}, p in {2,4,8}, log kappa
    iid N(0, 0.5^2), 16 N(0,1) forcing right-hand sides each, one batch call
    for set-up and one for all solves.  Three arms: the 16 right-hand sides of
    a problem solved together (rhs_block = 16: FP64 refinement around 16
    simultaneous FP32 PCGs), the mixed form one right-hand side at a time, and
    the plain FP64 form one at a time."""
    import numpy as np
    import torch
    from paper_1811_09909_gb300 import hdgmg
    rng = np.random.default_rng(4)
    shapes = [(int(rng.choice((32, 64, 128, 256))), int(rng.choice((2, 4, 8)))) for _ in range(64)]
    gen = torch.Generator(device=dev).manual_seed(4)
    logks = [torch.randn(n * n, generator=gen, device=dev, dtype=torch.float64) * 0.5 for n, p in shapes]
    fs = [torch.randn((16, (p + 1) ** 2, n * n), generator=gen, device=dev, dtype=torch.float64)
          for n, p in shapes]
    dofs = sum(2 * n * (n - 1) * (p + 1) for n, p in shapes) * 16
    stream = torch.cuda.current_stream(dev)
    arms = {"mixed_blocked16": dict(precision=hdgmg.PREC_FP32, rhs_block=16),
            "mixed_one_at_a_time": dict(precision=hdgmg.PREC_FP32),
            "fp64_one_at_a_time": dict(precision=hdgmg.PREC_FP64)}
    out = {}
    for name, kw in arms.items():
        b = hdgmg.Batch([dict(n=n, p=p) for n, p in shapes], nthreads=16, **kw, **SOLVER_OPTS)
        times, worst = [], 0.0
        for it in range(warmup + steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.setup(logks)
            lams, us, _, infos = b.solve(fs, want_u=True, want_q=False)
            e1.record(stream)
            e1.synchronize()
            if it >= warmup:
                times.append(e0.elapsed_time(e1))
                worst = max(worst, max(i.rel_res for i in infos))
        del lams, us
        b.close()
        ms = statistics.mean(times)
        out[name] = {"value": dofs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "worst_rel_res": worst}
    return {"value": out["mixed_blocked16"]["value"], "unit": UNIT,
            "ms_per_step": out["mixed_blocked16"]["ms_per_step"], "problems": 64,
            "rhs_per_problem": 16, "trace_dofs_x_rhs": dofs, "arms": out,
            "workload": "64 problems, n in {32,64,128,256}, p in {2,4,8}, log kappa iid N(0,0.25), "
                        "16 N(0,1) right-hand sides each; one batch set-up + solve of all right-hand "
                        "sides to 1e-10 (value: the blocked mixed arm)"}


def condense_cd_flops(p, nE, basis=False):
    """Algorithmic FP64 flops of the convection-diffusion condensation per
    launch.  Local LU: LU of S (2 n_v^3 / 3), X = S^-1 W (2 n_v^2 n_t), V^T X
    (2 n_t^2 n_v) per element.  Pencil basis: Vt = eps Pv1 + Pv0 and
    W~ = eps Pw1 + Pw0 (2 n_v n_t each), the 1 x 1 / 2 x 2 blocks on W~
    (3 n_v n_t), Vt^T Y plus eps K (2 n_t^2 (n_v + 1))."""
    nv, nt = (p + 1) ** 2, 4 * (p + 1)
    if basis:
        return nE * (7.0 * nv * nt + 2.0 * nt * nt * (nv + 1))
    return nE * (2.0 * nv ** 3 / 3.0 + 2.0 * nv * nv * nt + 2.0 * nt * nt * nv)


def run_convdiff(dev, steps, warmup):
    """Convection-diffusion, eps = 1e-3, beta = (1, 0.5), 512 x 512 quads,
    p = 6, manufactured u = sin(pi x) sin(pi y): FP64 condensation, FGMRES(30)
    right-preconditioned by the step-3 V-cycle in FP32 with the BF16 finest
    operator (mixed) or in FP64; the error of the mixed solution against the
    FP64 one and against the manufactured solution is reported."""
    import math
    import numpy as np
    import torch
    from paper_1811_09909_gb300 import hdgmg
    from paper_1811_09909_gb300 import workloads as W
    n, p, eps, beta = 512, 6, 1e-3, (1.0, 0.5)
    wl = W.convdiff(n, p, eps=eps, beta=beta)
    logk = torch.as_tensor(wl.log_kappa, device=dev)
    f = torch.as_tensor(wl.f[0], device=dev)
    opts = dict(coarsest_n=4, m_fine=1, m_growth=2, m_max=4, rtol=1e-10,
                krylov=hdgmg.KRYLOV_GMRES, gmres_restart=30, local_corr=hdgmg.LC_PRE,
                tau_mode=hdgmg.TAU_OVER_H, tau_c=eps, beta=beta)
    stream = torch.cuda.current_stream(dev)
    out = {}
    sols = {}
    for name, prec in (("mixed_bf16", hdgmg.PREC_BF16), ("mixed_fp32", hdgmg.PREC_FP32),
                       ("fp64", hdgmg.PREC_FP64)):
        s = hdgmg.Solver(n, p, precision=prec, stream=stream, **opts)
        times, infos = [], []
        for it in range(warmup + steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.setup(logk)
            lam, u, _, info = s.solve(f, want_q=False)
            e1.record(stream)
            e1.synchronize()
            if it >= warmup:
                times.append(e0.elapsed_time(e1))
                infos.append(info)
        assert all(i.converged for i in infos)
        ms = statistics.mean(times)
        sols[name] = (lam, u)
        cms = statistics.mean(i.t_condense_ms for i in infos)
        out[name] = {"value": wl.interior_trace_dofs / (ms * 1e-3), "ms_per_step": ms,
                     "setup_ms": infos[-1].t_setup_ms, "condense_ms": cms,
                     "solve_ms": infos[-1].t_solve_ms, "iters": infos[-1].iters,
                     "rel_res": max(i.rel_res for i in infos),
                     "condense_route": ("basis" if infos[-1].condense_kind == hdgmg.CONDENSE_BASIS
                                        else "factor")}
        s.close()
    # the same condensation by local LU (the factor route), for comparison
    s = hdgmg.Solver(n, p, precision=hdgmg.PREC_FP64, stream=stream,
                     condensation=hdgmg.CONDENSE_FACTOR, **opts)
    fms = []
    for it in range(2):
        s.setup(logk)
        _, _, _, info = s.solve(f, want_u=False, want_q=False)
        fms.append(info.t_condense_ms)
    s.close()
    lam64, u64 = sols["fp64"]
    for name in ("mixed_bf16", "mixed_fp32"):
        lam, u = sols[name]
        out[name]["lambda_rel_err_vs_fp64"] = float(torch.linalg.norm(lam - lam64) /
                                                    torch.linalg.norm(lam64))
    xi, _ = np.polynomial.legendre.leggauss(p + 1)
    e = np.arange(n * n)
    jj, ii = np.divmod(e, n)
    a = np.arange((p + 1) ** 2)
    Xn = (ii[None, :] + 0.5) / n + 0.5 / n * xi[a % (p + 1)][:, None]
    Yn = (jj[None, :] + 0.5) / n + 0.5 / n * xi[a // (p + 1)][:, None]
    u_ex = torch.as_tensor(np.sin(math.pi * Xn) * np.sin(math.pi * Yn), device=dev)
    err = float((sols["mixed_bf16"][1] - u_ex).abs().max())
    flops = condense_cd_flops(p, n * n, basis=out["fp64"]["condense_route"] == "basis")
    lu_flops = condense_cd_flops(p, n * n)
    return {"workload": "convection-diffusion eps=1e-3, beta=(1,0.5), 512x512 quads, p=6, "
                        "u=sin(pi x)sin(pi y); FGMRES(30) + step-3 V-cycle (m_N=1 doubling to 4, "
                        "coarsest 4x4); FP64 condensation",
            "interior_trace_dofs": wl.interior_trace_dofs, "unit": UNIT, **out,
            "u_nodal_max_err_vs_exact": err,
            "condense_fp64_tflops": flops / (out["fp64"]["condense_ms"] * 1e-3) / 1e12,
            "condense_fp64_frac": flops / (out["fp64"]["condense_ms"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
            "condense_factor_route_ms": fms[-1],
            "condense_factor_route_frac": lu_flops / (fms[-1] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}


def run_unstructured(dev, steps, warmup, n=96, p=3):
    """Unstructured meshes (seed-point agglomeration, Sec. 3.1.2): the
    Example II stand-in -- a 2 x 1 box with eight holes, 2n x n jittered cells
    cut into triangles and split into quadrilaterals (about 97k elements at
    n = 96), kappa = 1, f = 1, zero Dirichlet data, seven seed points;
    set-up (geometric condensation, Schur complements of every
    macro-element) + MG-preconditioned CG to 1e-10 + recovery, all FP64.
    The roofline line is the finest-level operator application (element
    gather-multiply + edge sum), timed alone."""
    import numpy as np
    import torch
    from paper_1811_09909_gb300 import umesh as um
    from paper_1811_09909_gb300 import workloads as W
    v, q, sp, logk, f = W.example2(n, p)
    s = um.USolver(v, q, p, 1.0, sp, rtol=1e-10)
    lk = torch.as_tensor(logk, device=dev)
    fd = torch.as_tensor(f, device=dev)
    stream = torch.cuda.current_stream(dev)
    times, infos = [], []
    for it in range(warmup + steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.setup(lk)
        lam, u, qq, info = s.solve(fd)
        e1.record(stream)
        e1.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
            infos.append(info)
    assert all(i.converged for i in infos)
    ms = statistics.mean(times)
    # the same step with the FP32 V-cycle inside the FP64 PCG
    from paper_1811_09909_gb300 import hdgmg
    s32 = um.USolver(v, q, p, 1.0, sp, rtol=1e-10, precision=hdgmg.PREC_FP32)
    t32, i32 = [], []
    for it in range(warmup + steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s32.setup(lk)
        _, _, _, info32 = s32.solve(fd)
        e1.record(stream)
        e1.synchronize()
        if it >= warmup:
            t32.append(e0.elapsed_time(e1))
            i32.append(info32)
    assert all(i.converged for i in i32)
    ms32 = statistics.mean(t32)
    s32.close()
    n0, nel, nd, ndm = s.level_sizes(0)
    x = torch.randn(n0, dtype=torch.float64, device=dev)
    for _ in range(3):
        s.apply(0, x)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        s.apply(0, x)
    e1.record(stream)
    e1.synchronize()
    ams = e0.elapsed_time(e1) / reps
    abytes = nel * ndm * ndm * 8.0 + 2 * n0 * 8.0       # A_e once, x and y once
    gbs = abytes / (ams * 1e-3) / 1e9
    last = infos[-1]
    out = {"workload": f"Example II stand-in: 2x1 box, 8 holes, {nel} quads (bilinear), p={p}, "
                       f"{len(sp)} seeds, kappa=1, f=1; set-up + PCG (V-cycle, damped edge "
                       "block-Jacobi 0.8, m=2 doubling to 4) to 1e-10 + recovery, FP64",
           "elements": nel, "trace_dofs": s.trace_dofs, "levels": s.n_levels,
           "value": s.trace_dofs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "setup_ms": last.t_setup_ms, "condense_ms": last.t_condense_ms,
           "solve_ms": last.t_solve_ms, "iters": last.iters, "rel_res": max(i.rel_res for i in infos),
           "gpu_launches_per_step": last.kernel_launches,
           "fp32_cycle": {"value": s.trace_dofs / (ms32 * 1e-3), "ms_per_step": ms32,
                          "solve_ms": i32[-1].t_solve_ms, "iters": i32[-1].iters,
                          "rel_res": max(i.rel_res for i in i32)},
           "apply_roofline": {"bound": "hbm", "kernel": "u_elem_matvec_mesh_kernel + u_edge_kernel",
                              "achieved": gbs, "peak": hbm_peak()[0], "unit": "GB/s",
                              "frac": gbs / hbm_peak()[0],
                              "ms": ams, "algorithmic_bytes": abytes}}
    s.close()
    return out


def run_adjoint(dev, steps, warmup):
    """Misfit gradient at 1024 x 1024, p = 4: set-up, forward solve, misfit,
    transposed multigrid solve and per-element contraction."""
    import torch
    from paper_1811_09909_gb300 import hdgmg
    n, p = 1024, 4
    gen = torch.Generator(device=dev).manual_seed(52)
    logk = torch.randn(n * n, generator=gen, device=dev, dtype=torch.float64)
    f = torch.ones(((p + 1) ** 2, n * n), device=dev, dtype=torch.float64)
    s = hdgmg.Solver(n, p, precision=hdgmg.PREC_FP32, **SOLVER_OPTS)
    s.setup(logk)
    _, u_ref, _, _ = s.solve(f, want_q=False)
    u_obs = u_ref * (1.0 + 0.01 * torch.randn(u_ref.shape, generator=gen, device=dev,
                                              dtype=torch.float64))
    stream = torch.cuda.current_stream(dev)
    times = []
    for it in range(warmup + steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.setup(logk)
        J, gk, gf, info = s.gradient(f, u_obs)
        e1.record(stream)
        e1.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    ms = statistics.mean(times)
    dofs = 2 * n * (n - 1) * (p + 1)
    s.close()
    return {"ms_per_gradient": ms, "trace_dofs": dofs, "parameters": n * n,
            "adjoint_iters": info.iters, "adjoint_rel_res": info.rel_res,
            "workload": "1024x1024 quads, p=4, log kappa iid N(0,1), J = 1/2 |u - u_obs|_M^2 with "
                        "1% noise; set-up + forward + adjoint solve + contraction, mixed precision"}


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
    if rank == 0 and line is not None and args.arm == "both" and not args.no_extra:
        import torch
        dev = torch.device("cuda", 0)
        line["batched"] = run_batched(dev, steps=2, warmup=1)
        line["adjoint"] = run_adjoint(dev, steps=2, warmup=1)
        line["convdiff"] = run_convdiff(dev, steps=2, warmup=1)
        line["unstructured"] = run_unstructured(dev, steps=2, warmup=1)
    if rank == 0:
        if (not args.no_cpu_baseline and args.arm == "both"
                and int(os.environ.get("WORLD_SIZE", "1")) == 1):
            line["cpu_baseline"] = cpu_baseline_obj([run_oracle_subprocess()])
        print(json.dumps(line))


if __name__ == "__main__":
    main()
