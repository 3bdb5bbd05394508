"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/hdgmg.h declares, and rejects bad arguments before
touching the GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdgmg.h")


def _declared(header=HEADER):
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hdgmg_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1811_09909_gb300 import build, hdgmg
    if not os.path.exists(hdgmg.LIB_PATH):
        build.build()
    return hdgmg.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hdgmg_create", "hdgmg_setup", "hdgmg_solve", "hdgmg_destroy",
                     "hdgmg_last_error", "hdgmg_run_host", "hdgmg_apply_vcycle"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1811_09909_gb300 import hdgmg
    assert sorted(hdgmg.EXPORTED) == sorted(n for n in _declared())


def test_library_exports_every_unstructured_symbol(lib):
    from paper_1811_09909_gb300 import umesh
    names = _declared(os.path.join(ROOT, "include", "hdgmg_umesh.h"))
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(umesh.EXPORTED) == names


def test_default_options(lib):
    from paper_1811_09909_gb300 import hdgmg
    o = hdgmg.default_opts()
    assert (o.coarsest_n, o.m_fine, o.m_growth, o.m_max) == (2, 1, 2, 0)
    assert o.local_corr == hdgmg.LC_BOTH and o.krylov == hdgmg.KRYLOV_CG
    assert o.omega == 1.0 and o.rtol == 1e-10 and o.max_it == 200
    assert o.precision == hdgmg.PREC_FP64 and o.inner_rtol == 1e-5
    assert o.cluster_tail_n == 0 and o.gmres_restart == 30
    assert o.smoother == hdgmg.SMOOTH_BLOCK_JACOBI
    assert o.condensation == hdgmg.CONDENSE_AUTO and o.l2_persist_mb == 64


@pytest.mark.parametrize("kw,msg", [
    (dict(p=0), "p must"), (dict(p=9), "p must"), (dict(n=1), "n must"),
    (dict(n=12, coarsest=2), "halve"), (dict(tau_c=-1.0), "tau_c"),
    (dict(krylov=2, restart=0), "gmres_restart"), (dict(krylov=2, restart=257), "gmres_restart"),
    (dict(krylov=3), "krylov"),
    (dict(pde=1, krylov=1), "symmetric"), (dict(pde=5), "unknown pde"),
    (dict(smoother=4), "unknown smoother"),
    (dict(scheme=4), "unknown scheme"), (dict(scheme=-1), "unknown scheme"),
    (dict(scheme=2, pde=1, krylov=2), "diffusion only"),
    (dict(scheme=2, krylov=1), "symmetric"), (dict(scheme=3, krylov=1), "symmetric"),
    (dict(tau_mode=3), "tau_mode"),
    (dict(condensation=3), "unknown condensation"),
])
def test_create_rejects_bad_arguments(lib, kw, msg):
    from paper_1811_09909_gb300 import hdgmg
    n = kw.get("n", 16)
    p = kw.get("p", 2)
    prob = hdgmg.Problem(n, p, 0.0, 1.0, 0.0, 1.0, kw.get("tau_mode", hdgmg.TAU_CONST),
                         kw.get("tau_c", 1.0), kw.get("pde", 0), 1.0, 0.5, kw.get("scheme", 0))
    o = hdgmg.default_opts(coarsest_n=kw.get("coarsest", 2), krylov=kw.get("krylov", 1),
                           gmres_restart=kw.get("restart", 30), smoother=kw.get("smoother", 0),
                           condensation=kw.get("condensation", 0))
    ctx = ctypes.c_void_p()
    st = lib.hdgmg_create(ctypes.byref(ctx), ctypes.byref(prob), ctypes.byref(o), None)
    assert st == -1
    assert ctx.value is None
    assert msg in lib.hdgmg_last_error().decode()


def test_null_arguments(lib):
    assert lib.hdgmg_create(None, None, None, None) == -1
    assert lib.hdgmg_setup(None, None) == -1
    assert lib.hdgmg_solve(None, 1, None, None, None, None, None, None) == -1
    lib.hdgmg_destroy(None)
