"""Thin ctypes binding of the unstructured-mesh C ABI (include/hdgmg_umesh.h).

Argument marshalling only; the plan is built by the library's host code and
every numerical step runs in its CUDA kernels.  Device buffers are torch
tensors (float64, CUDA, contiguous) on torch's current stream.
"""
import ctypes

import numpy as np

from . import hdgmg as _h

EXPORTED = ["hdgmg_umesh_default_opts", "hdgmg_umesh_plan_create", "hdgmg_umesh_plan_destroy", "hdgmg_umesh_plan_sizes",
            "hdgmg_umesh_plan_edges", "hdgmg_umesh_plan_partition", "hdgmg_umesh_plan_macro_edges",
            "hdgmg_umesh_create", "hdgmg_umesh_setup", "hdgmg_umesh_solve",
            "hdgmg_umesh_level_sizes", "hdgmg_umesh_element_matrices", "hdgmg_umesh_apply",
            "hdgmg_umesh_vcycle", "hdgmg_umesh_destroy"]


class UProblem(ctypes.Structure):
    _fields_ = [("n_vert", ctypes.c_int32), ("xy", ctypes.c_void_p),
                ("n_elem", ctypes.c_int32), ("quads", ctypes.c_void_p),
                ("p", ctypes.c_int32), ("tau", ctypes.c_double),
                ("n_seeds", ctypes.c_int32), ("seeds", ctypes.c_void_p)]


_ready = False


def load():
    global _ready
    lib = _h.load()
    if _ready:
        return lib
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    PP = ctypes.POINTER(P)
    lib.hdgmg_umesh_plan_create.argtypes = [PP, ctypes.POINTER(UProblem)]
    lib.hdgmg_umesh_plan_destroy.argtypes = [P]
    lib.hdgmg_umesh_plan_destroy.restype = None
    lib.hdgmg_umesh_plan_sizes.argtypes = [P, P]
    lib.hdgmg_umesh_plan_edges.argtypes = [P, P]
    lib.hdgmg_umesh_plan_partition.argtypes = [P, I32, P]
    lib.hdgmg_umesh_plan_macro_edges.argtypes = [P, I32, P, P, P]
    lib.hdgmg_umesh_default_opts.argtypes = [ctypes.POINTER(_h.Opts)]
    lib.hdgmg_umesh_default_opts.restype = None
    lib.hdgmg_umesh_create.argtypes = [PP, ctypes.POINTER(UProblem), ctypes.POINTER(_h.Opts), P]
    lib.hdgmg_umesh_setup.argtypes = [P, P]
    lib.hdgmg_umesh_solve.argtypes = [P, P, P, P, P, ctypes.POINTER(_h.Info)]
    lib.hdgmg_umesh_level_sizes.argtypes = [P, I32, P]
    lib.hdgmg_umesh_element_matrices.argtypes = [P, I32, P, P]
    lib.hdgmg_umesh_apply.argtypes = [P, I32, P, P]
    lib.hdgmg_umesh_vcycle.argtypes = [P, P, P]
    lib.hdgmg_umesh_destroy.argtypes = [P]
    lib.hdgmg_umesh_destroy.restype = None
    for name in EXPORTED:
        if name not in ("hdgmg_umesh_plan_destroy", "hdgmg_umesh_destroy", "hdgmg_umesh_default_opts"):
            getattr(lib, name).restype = ctypes.c_int
    _ready = True
    return lib


def _check(st):
    if st != 0:
        raise _h.HdgmgError(st, _h.load().hdgmg_last_error().decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class _Problem:
    """Keeps the host arrays of a UProblem alive."""

    def __init__(self, verts, quads, p, tau, seeds):
        self.xy = np.ascontiguousarray(verts, dtype=np.float64)
        self.quads = np.ascontiguousarray(quads, dtype=np.int32)
        self.seeds = np.ascontiguousarray(seeds, dtype=np.float64)
        self.s = UProblem(len(self.xy), _ptr(self.xy), len(self.quads), _ptr(self.quads),
                          int(p), float(tau), len(self.seeds), _ptr(self.seeds))


class Plan:
    """Host-only plan (hdgmg_umesh_plan_*): partitions and macro-edges."""

    def __init__(self, verts, quads, p, tau, seeds):
        lib = load()
        self._pr = _Problem(verts, quads, p, tau, seeds)
        self._h = ctypes.c_void_p()
        _check(lib.hdgmg_umesh_plan_create(ctypes.byref(self._h), ctypes.byref(self._pr.s)))
        out = np.zeros(4, dtype=np.int64)
        _check(lib.hdgmg_umesh_plan_sizes(self._h, _ptr(out)))
        self.n_edges, self.n_parts, self.n_levels, self.trace_dofs = (int(x) for x in out)

    def edges(self):
        ev = np.zeros((self.n_edges, 2), dtype=np.int32)
        _check(load().hdgmg_umesh_plan_edges(self._h, _ptr(ev)))
        return ev

    def partition(self, r):
        out = np.zeros(len(self._pr.quads), dtype=np.int32)
        _check(load().hdgmg_umesh_plan_partition(self._h, int(r), _ptr(out)))
        return out

    def macro_edges(self, t):
        """(info [n, 6]: side0, side1, start, end, closed, offset; items [m, 2])."""
        lib = load()
        counts = np.zeros(2, dtype=np.int64)
        _check(lib.hdgmg_umesh_plan_macro_edges(self._h, int(t), _ptr(counts), None, None))
        info = np.zeros((int(counts[0]), 6), dtype=np.int32)
        items = np.zeros((int(counts[1]), 2), dtype=np.int32)
        _check(lib.hdgmg_umesh_plan_macro_edges(self._h, int(t), _ptr(counts), _ptr(info), _ptr(items)))
        return info, items

    def close(self):
        if self._h:
            load().hdgmg_umesh_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dptr(t):
    import torch
    if t is None:
        return None
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


class USolver:
    """One unstructured-mesh problem on the current CUDA device."""

    def __init__(self, verts, quads, p, tau, seeds, **opts):
        import torch
        lib = load()
        self.p = int(p)
        self._pr = _Problem(verts, quads, p, tau, seeds)
        o = _h.Opts()
        lib.hdgmg_umesh_default_opts(ctypes.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        self.opts = o
        self._h = ctypes.c_void_p()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _check(lib.hdgmg_umesh_create(ctypes.byref(self._h), ctypes.byref(self._pr.s),
                                      ctypes.byref(o), stream))
        self.E = len(self._pr.quads)
        self.nv = (self.p + 1) ** 2
        plan = Plan(verts, quads, p, tau, seeds)
        self.n_edges, self.n_levels = plan.n_edges, plan.n_levels
        self.trace_dofs = plan.trace_dofs
        plan.close()

    def setup(self, log_kappa):
        _check(load().hdgmg_umesh_setup(self._h, _dptr(log_kappa)))

    def solve(self, f, want_u=True, want_q=True):
        import torch
        dev = f.device
        lam = torch.empty(self.n_edges, self.p + 1, dtype=torch.float64, device=dev)
        u = torch.empty(self.E, self.nv, dtype=torch.float64, device=dev) if want_u else None
        q = torch.empty(self.E, 2, self.nv, dtype=torch.float64, device=dev) if want_q else None
        info = _h.Info()
        st = load().hdgmg_umesh_solve(self._h, _dptr(f), _dptr(lam), _dptr(u), _dptr(q),
                                      ctypes.byref(info))
        if st not in (0, -4):
            _check(st)
        return lam, u, q, info

    def level_sizes(self, level):
        out = np.zeros(4, dtype=np.int64)
        _check(load().hdgmg_umesh_level_sizes(self._h, int(level), _ptr(out)))
        return tuple(int(x) for x in out)

    def element_matrices(self, level):
        import torch
        n, nel, nd, ndm = self.level_sizes(level)
        A = torch.zeros(nel, ndm, ndm, dtype=torch.float64, device="cuda")
        dofs = np.zeros((nel, ndm), dtype=np.int32)
        _check(load().hdgmg_umesh_element_matrices(self._h, int(level), _dptr(A), _ptr(dofs)))
        return A, dofs

    def apply(self, level, x):
        import torch
        y = torch.empty_like(x)
        _check(load().hdgmg_umesh_apply(self._h, int(level), _dptr(x), _dptr(y)))
        return y

    def vcycle(self, r):
        import torch
        z = torch.empty_like(r)
        _check(load().hdgmg_umesh_vcycle(self._h, _dptr(r), _dptr(z)))
        return z

    def close(self):
        if self._h:
            load().hdgmg_umesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
