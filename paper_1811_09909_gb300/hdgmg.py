"""Thin ctypes binding of the hdgmg C ABI (include/hdgmg.h).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libhdgmg.so``.  Device buffers are torch tensors (float64, CUDA,
contiguous); the library runs on torch's current CUDA stream.  If the library
has not been built, loading raises -- there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhdgmg.so")

TAU_CONST, TAU_OVER_H, TAU_KAPPA_OVER_H = 0, 1, 2
LC_NONE, LC_PRE, LC_BOTH = 0, 1, 2
KRYLOV_NONE, KRYLOV_CG, KRYLOV_GMRES = 0, 1, 2
PREC_FP64, PREC_FP32, PREC_FP32_IR, PREC_BF16 = 0, 1, 2, 3
PDE_DIFFUSION, PDE_CONVDIFF = 0, 1
SCHEME_HDG, SCHEME_SIPG, SCHEME_NIPG, SCHEME_IIPG = 0, 1, 2, 3
SMOOTH_BLOCK_JACOBI, SMOOTH_POINT_JACOBI, SMOOTH_CHEBYSHEV, SMOOTH_LU_SGS = 0, 1, 2, 3
CONDENSE_AUTO, CONDENSE_BASIS, CONDENSE_FACTOR = 0, 1, 2

STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOCONV",
          -5: "EBREAKDOWN", -6: "ETIMEOUT"}

EXPORTED = ["hdgmg_default_opts", "hdgmg_create", "hdgmg_setup", "hdgmg_solve",
            "hdgmg_run_host", "hdgmg_num_levels", "hdgmg_level_shape",
            "hdgmg_copy_element_matrices", "hdgmg_apply_operator", "hdgmg_apply_vcycle",
            "hdgmg_condensed_rhs", "hdgmg_last_error", "hdgmg_destroy",
            "hdgmg_apply_operator_noalloc", "hdgmg_gradient", "hdgmg_adjoint",
            "hdgmg_batch_create", "hdgmg_batch_setup", "hdgmg_batch_solve",
            "hdgmg_batch_context", "hdgmg_batch_destroy", "hdgmg_check_cycle_timeout",
            "hdgmg_trace_vcycle"]


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("tau_mode", ctypes.c_int32), ("tau_c", ctypes.c_double),
                ("pde", ctypes.c_int32), ("beta_x", ctypes.c_double), ("beta_y", ctypes.c_double),
                ("scheme", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("coarsest_n", ctypes.c_int32), ("m_fine", ctypes.c_int32),
                ("m_growth", ctypes.c_int32), ("m_max", ctypes.c_int32),
                ("local_corr", ctypes.c_int32), ("omega", ctypes.c_double),
                ("krylov", ctypes.c_int32), ("max_it", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("inner_rtol", ctypes.c_double), ("cluster_tail_n", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("smoother", ctypes.c_int32),
                ("condensation", ctypes.c_int32), ("l2_persist_mb", ctypes.c_int32),
                ("pcycle", ctypes.c_int32), ("pcycle_tail_n", ctypes.c_int32),
                ("pcg_graph", ctypes.c_int32), ("rhs_block", ctypes.c_int32),
                ("pcg_fuse", ctypes.c_int32), ("matrix_free", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rel_res", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("n_levels", ctypes.c_int32),
                ("trace_dofs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("refinements", ctypes.c_int32), ("t_condense_ms", ctypes.c_double),
                ("condense_threads", ctypes.c_int32),
                ("condense_elements_per_block", ctypes.c_int32),
                ("condense_kind", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HdgmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hdgmg {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "paper_1811_09909_gb300.build.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.hdgmg_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.hdgmg_default_opts.restype = None
    lib.hdgmg_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Problem), ctypes.POINTER(Opts), P]
    lib.hdgmg_setup.argtypes = [P, P]
    lib.hdgmg_solve.argtypes = [P, I32, P, P, P, P, P, ctypes.POINTER(Info)]
    lib.hdgmg_run_host.argtypes = [P, P, P, P, P, P, P, ctypes.POINTER(Info)]
    lib.hdgmg_num_levels.argtypes = [P, ctypes.POINTER(I32)]
    lib.hdgmg_level_shape.argtypes = [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32)]
    lib.hdgmg_copy_element_matrices.argtypes = [P, I32, P]
    lib.hdgmg_apply_operator.argtypes = [P, I32, P, P]
    lib.hdgmg_apply_operator_noalloc.argtypes = [P, I32, P, P]
    lib.hdgmg_gradient.argtypes = [P, P, P, P, ctypes.POINTER(D), P, P, ctypes.POINTER(Info)]
    lib.hdgmg_adjoint.argtypes = [P, P, P, P, P, P, ctypes.POINTER(Info)]
    PP = ctypes.POINTER(P)
    lib.hdgmg_batch_create.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(Problem),
                                       ctypes.POINTER(Opts), I32, P]
    lib.hdgmg_batch_setup.argtypes = [P, PP]
    lib.hdgmg_batch_solve.argtypes = [P, I32, PP, PP, PP, PP, PP, ctypes.POINTER(Info)]
    lib.hdgmg_batch_context.argtypes = [P, I32, ctypes.POINTER(P)]
    lib.hdgmg_batch_destroy.argtypes = [P]
    lib.hdgmg_batch_destroy.restype = None
    lib.hdgmg_apply_vcycle.argtypes = [P, P, P]
    lib.hdgmg_check_cycle_timeout.argtypes = [P, I32]
    lib.hdgmg_trace_vcycle.argtypes = [P, P, P, P, I32, P]
    lib.hdgmg_condensed_rhs.argtypes = [P, P, P, P]
    lib.hdgmg_last_error.argtypes = []
    lib.hdgmg_last_error.restype = ctypes.c_char_p
    lib.hdgmg_destroy.argtypes = [P]
    lib.hdgmg_destroy.restype = None
    for name in EXPORTED:
        if name not in ("hdgmg_default_opts", "hdgmg_last_error", "hdgmg_destroy",
                        "hdgmg_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise HdgmgError(status, _lib.hdgmg_last_error().decode())


def default_opts(**kw):
    lib = load()
    o = Opts()
    lib.hdgmg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expects contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    """numpy array (float64, C-contiguous) or pinned torch CPU tensor -> pointer."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class Solver:
    """One HDG trace problem on the GPU.

    n, p, domain, tau, beta (convection velocity or None) and scheme
    (SCHEME_*) as in hdgmg_problem; options as keyword arguments of
    hdgmg_opts (coarsest_n, m_fine, m_growth, m_max, local_corr, omega,
    krylov, max_it, rtol, precision)."""

    def __init__(self, n, p, tau_mode=TAU_OVER_H, tau_c=1.0, domain=(0.0, 1.0, 0.0, 1.0),
                 stream=None, beta=None, scheme=SCHEME_HDG, **opts):
        import torch
        lib = load()
        self.torch = torch
        self.n, self.p = n, p
        self.nd = p + 1
        self.nv = (p + 1) ** 2
        self.n_edges = 2 * n * (n + 1)
        pde = PDE_DIFFUSION if beta is None else PDE_CONVDIFF
        bx, by = (0.0, 0.0) if beta is None else (float(beta[0]), float(beta[1]))
        prob = Problem(n, p, domain[0], domain[1], domain[2], domain[3], tau_mode, tau_c, pde, bx, by,
                       scheme)
        self.opts = default_opts(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        ctx = ctypes.c_void_p()
        _check(lib.hdgmg_create(ctypes.byref(ctx), ctypes.byref(prob), ctypes.byref(self.opts),
                                ctypes.c_void_p(stream.cuda_stream)))
        self.ctx = ctx
        self.lib = lib

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.hdgmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- main calls -------------------------------------------------------
    def setup(self, log_kappa):
        _check(self.lib.hdgmg_setup(self.ctx, _ptr(log_kappa)))

    def solve(self, f, gD=None, want_u=True, want_q=True):
        """f [nrhs][nv][E] (or [nv][E]); returns (lam, u, q, info)."""
        torch = self.torch
        single = f.dim() == 2
        if single:
            f = f.unsqueeze(0)
            if gD is not None:
                gD = gD.unsqueeze(0)
        nrhs = f.shape[0]
        dev = f.device
        lam = torch.empty((nrhs, self.nd, self.n_edges), dtype=torch.float64, device=dev)
        u = torch.empty((nrhs, self.nv, self.n * self.n), dtype=torch.float64, device=dev) if want_u else None
        q = torch.empty((nrhs, 2, self.nv, self.n * self.n), dtype=torch.float64, device=dev) if want_q else None
        info = Info()
        st = self.lib.hdgmg_solve(self.ctx, nrhs, _ptr(f), _ptr(gD), _ptr(lam), _ptr(u), _ptr(q),
                                  ctypes.byref(info))
        if st not in (0, -4):
            _check(st)
        if single:
            lam = lam[0]
            u = u[0] if u is not None else None
            q = q[0] if q is not None else None
        return lam, u, q, info

    def solve_status(self, f, gD, lam, u, q):
        """Raw call on preallocated outputs; returns (status, info)."""
        info = Info()
        nrhs = 1 if f.dim() == 2 else f.shape[0]
        st = self.lib.hdgmg_solve(self.ctx, nrhs, _ptr(f), _ptr(gD), _ptr(lam), _ptr(u), _ptr(q),
                                  ctypes.byref(info))
        return st, info

    def run_host(self, log_kappa, f, gD, lam, u, q):
        """End-to-end call on host buffers (numpy arrays or pinned tensors)."""
        info = Info()
        st = self.lib.hdgmg_run_host(self.ctx, _hptr(log_kappa), _hptr(f), _hptr(gD), _hptr(lam),
                                     _hptr(u), _hptr(q), ctypes.byref(info))
        if st not in (0, -4):
            _check(st)
        return st, info

    # -- adjoint ------------------------------------------------------------
    def gradient(self, f, u_obs, gD=None):
        """(J, dJ/dlog kappa [E], dJ/df [nv][E], info) of J = 1/2 |u - u_obs|_M^2."""
        torch = self.torch
        E = self.n * self.n
        gk = torch.empty(E, dtype=torch.float64, device=f.device)
        gf = torch.empty((self.nv, E), dtype=torch.float64, device=f.device)
        J = ctypes.c_double()
        info = Info()
        st = self.lib.hdgmg_gradient(self.ctx, _ptr(f), _ptr(gD), _ptr(u_obs), ctypes.byref(J),
                                     _ptr(gk), _ptr(gf), ctypes.byref(info))
        if st not in (0, -4):
            _check(st)
        return J.value, gk, gf, info

    def adjoint(self, lam, u, g_u):
        """(dL/dlog kappa, dL/df) for the nodal sensitivity g_u = dL/du."""
        torch = self.torch
        E = self.n * self.n
        gk = torch.empty(E, dtype=torch.float64, device=u.device)
        gf = torch.empty((self.nv, E), dtype=torch.float64, device=u.device)
        info = Info()
        st = self.lib.hdgmg_adjoint(self.ctx, _ptr(lam), _ptr(u), _ptr(g_u), _ptr(gk), _ptr(gf),
                                    ctypes.byref(info))
        if st not in (0, -4):
            _check(st)
        return gk, gf

    # -- inspection ---------------------------------------------------------
    def num_levels(self):
        k = ctypes.c_int32()
        _check(self.lib.hdgmg_num_levels(self.ctx, ctypes.byref(k)))
        return k.value

    def level_shape(self, level):
        n, nd = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.hdgmg_level_shape(self.ctx, level, ctypes.byref(n), ctypes.byref(nd)))
        return n.value, nd.value

    def element_matrices(self, level=0):
        n, nd = self.level_shape(level)
        nl = 4 * nd
        out = self.torch.empty((nl, nl, n * n), dtype=self.torch.float64, device="cuda")
        _check(self.lib.hdgmg_copy_element_matrices(self.ctx, level, _ptr(out)))
        return out

    def apply_operator(self, level, x):
        y = self.torch.empty_like(x)
        _check(self.lib.hdgmg_apply_operator(self.ctx, level, _ptr(x), _ptr(y)))
        return y

    def apply_vcycle(self, r):
        e = self.torch.empty_like(r)
        _check(self.lib.hdgmg_apply_vcycle(self.ctx, _ptr(r), _ptr(e)))
        return e

    def trace_vcycle(self, r, cap=512):
        """One V-cycle as apply_vcycle, with the persistent kernel's step
        trace: returns (e, [(time_ns, tag), ...]) (see hdgmg_trace_vcycle)."""
        import numpy as np
        e = self.torch.empty_like(r)
        stamps = np.zeros(2 * cap, dtype=np.int64)
        count = ctypes.c_int32(0)
        _check(self.lib.hdgmg_trace_vcycle(self.ctx, _ptr(r), _ptr(e), _hptr(stamps), cap,
                                           ctypes.byref(count)))
        return e, [(int(stamps[2 * i]), int(stamps[2 * i + 1])) for i in range(count.value)]

    def condensed_rhs(self, f, gD=None):
        b = self.torch.empty((self.nd, self.n_edges), dtype=self.torch.float64, device="cuda")
        _check(self.lib.hdgmg_condensed_rhs(self.ctx, _ptr(f), _ptr(gD), _ptr(b)))
        return b


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class Batch:
    """Many independent problems solved concurrently on one GPU.

    problems: list of dicts with n, p and optionally tau_mode, tau_c, domain,
    beta, scheme; options as keyword arguments (one set for all problems)."""

    def __init__(self, problems, nthreads=8, stream=None, **opts):
        import torch
        lib = load()
        self.torch = torch
        self.lib = lib
        self.problems = []
        arr = (Problem * len(problems))()
        for i, pr in enumerate(problems):
            dom = pr.get("domain", (0.0, 1.0, 0.0, 1.0))
            beta = pr.get("beta")
            arr[i] = Problem(pr["n"], pr["p"], dom[0], dom[1], dom[2], dom[3],
                             pr.get("tau_mode", TAU_OVER_H), pr.get("tau_c", 1.0),
                             PDE_DIFFUSION if beta is None else PDE_CONVDIFF,
                             *((0.0, 0.0) if beta is None else (float(beta[0]), float(beta[1]))),
                             pr.get("scheme", SCHEME_HDG))
            self.problems.append((pr["n"], pr["p"]))
        self.opts = default_opts(**opts)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        b = ctypes.c_void_p()
        _check(lib.hdgmg_batch_create(ctypes.byref(b), len(problems), arr, ctypes.byref(self.opts),
                                      nthreads, ctypes.c_void_p(stream.cuda_stream)))
        self.b = b

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            self.lib.hdgmg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, log_kappas):
        _check(self.lib.hdgmg_batch_setup(self.b, _ptr_array(log_kappas)))

    def solve(self, fs, gDs=None, want_u=True, want_q=False):
        """fs: list of [nrhs][nv][E] tensors; returns (lams, us, qs, infos)."""
        torch = self.torch
        nrhs = fs[0].shape[0]
        lams, us, qs = [], [], []
        for (n, p), f in zip(self.problems, fs):
            assert f.shape[0] == nrhs
            E, nv, ne = n * n, (p + 1) ** 2, 2 * n * (n + 1)
            lams.append(torch.empty((nrhs, p + 1, ne), dtype=torch.float64, device=f.device))
            us.append(torch.empty((nrhs, nv, E), dtype=torch.float64, device=f.device) if want_u else None)
            qs.append(torch.empty((nrhs, 2, nv, E), dtype=torch.float64, device=f.device) if want_q else None)
        infos = (Info * len(fs))()
        st = self.lib.hdgmg_batch_solve(self.b, nrhs, _ptr_array(fs),
                                        _ptr_array(gDs) if gDs is not None else None,
                                        _ptr_array(lams), _ptr_array(us) if want_u else None,
                                        _ptr_array(qs) if want_q else None, infos)
        if st not in (0, -4):
            _check(st)
        return lams, us, qs, list(infos)


def _autograd_function():
    import torch

    class HDGSolve(torch.autograd.Function):
        """u = HDGSolve.apply(solver, log_kappa, f): set-up and solve on the GPU;
        the backward pass is the library's adjoint (one transposed multigrid
        solve plus per-element contractions).  The solver must not be set up
        again between forward and backward."""

        @staticmethod
        def forward(ctx, solver, log_kappa, f):
            solver.setup(log_kappa.detach().contiguous())
            lam, u, _, info = solver.solve(f.detach().contiguous(), want_q=False)
            ctx.solver = solver
            ctx.save_for_backward(lam, u)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            lam, u = ctx.saved_tensors
            gk, gf = ctx.solver.adjoint(lam, u, grad_u.contiguous())
            return None, gk, gf

    return HDGSolve


def hdg_solve(solver, log_kappa, f):
    """Differentiable solve: u(log kappa, f) for one right-hand side."""
    global _HDGSolve
    try:
        fn = _HDGSolve
    except NameError:
        fn = _HDGSolve = _autograd_function()
    return fn.apply(solver, log_kappa, f)
