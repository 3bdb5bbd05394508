"""hdgmg_apply_operator_noalloc: the allocation-free variant of
hdgmg_apply_operator for callers that cannot allocate device memory when they
apply the operator (their device memory belongs to another allocator, or their
loop must not pay for cudaMalloc/cudaFree, which can synchronise the device).
It keeps its temporaries in one static device array of 2^20 doubles instead of
cudaMalloc'd buffers.

Checked through the C ABI against hdgmg_apply_operator, on two calls in a row
(the array keeps the previous call's contents), on an FP64 level and on an
FP32 level, plus the size limit.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_09909_gb300 import hdgmg  # noqa: E402
from paper_1811_09909_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-11          # relative, max norm: the operator-parity tolerance of the suite


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _both(s, level, x):
    lib = s.lib
    y_ref = torch.empty_like(x)
    y_new = torch.empty_like(x)
    assert lib.hdgmg_apply_operator(s.ctx, level, _ptr(x), _ptr(y_ref)) == 0
    st = lib.hdgmg_apply_operator_noalloc(s.ctx, level, _ptr(x), _ptr(y_new))
    assert st == 0, lib.hdgmg_last_error().decode()
    return y_ref.cpu().numpy(), y_new.cpu().numpy()


@pytest.mark.parametrize("precision", [hdgmg.PREC_FP64, hdgmg.PREC_FP32])
def test_noalloc_matches_apply_operator_twice(precision):
    wl = W.lognormal(32, 3, seed=8)
    s = hdgmg.Solver(32, 3, precision=precision)
    s.setup(torch.as_tensor(wl.log_kappa, device="cuda"))
    rng = np.random.default_rng(1)
    for level in (0, 2):
        n, nd = s.level_shape(level)
        for _ in range(2):                       # two calls in a row
            x = torch.as_tensor(rng.standard_normal((nd, 2 * n * (n + 1))), device="cuda")
            ref, new = _both(s, level, x)
            assert np.abs(new - ref).max() <= TOL * np.abs(ref).max()


def test_noalloc_rejects_levels_beyond_the_scratch():
    s = hdgmg.Solver(512, 1, coarsest_n=4)        # level 0: 2 * 2*512*513 > 2^20 values
    x = torch.zeros((2, 2 * 512 * 513), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    st = s.lib.hdgmg_apply_operator_noalloc(s.ctx, 0, _ptr(x), _ptr(y))
    assert st == -1
    assert "static scratch" in s.lib.hdgmg_last_error().decode()
