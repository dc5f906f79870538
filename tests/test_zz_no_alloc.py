"""The allocation-free approximate inverse overlap entry point.

paw_apply_Sinv_approx_noalloc serves callers that cannot call cudaMalloc where
they need Shat^-1 X: real-time loops that must not wait on the allocator, hosts
that give the library a fixed memory budget.  Its scratch is a static device array inside the
library.  This test calls it through the C ABI twice in a row and checks both
results against paw_apply_Sinv_approx within the operator-test tolerances, and
checks that a request beyond the static scratch is refused before any device
work.  It is collected last on purpose (file name), and passes both alone in a
fresh process and after the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import gpu_fe, rel_err, to_dev

pytestmark = pytest.mark.gpu

# fp64 / fp32: the same SIMT arithmetic as the allocating call.  tf32 / bf16: the allocating call
# runs the projector contractions on the tensor cores (TF32 operands), this one in FP32 FMA, so
# the two differ by TF32 operand rounding (the operator tests' TF32 bound).
TOL = {"fp64": 1e-11, "fp32": 2e-5, "tf32": 4e-3, "bf16": 4e-3}


def _noalloc(fe, prec, X, Y):
    import torch
    from paper_2604_26037_gb300 import _lib as L
    code = fe._lib.paw_apply_Sinv_approx_noalloc(
        fe._h, L.Precision.of(prec), C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
        X.shape[1], X.stride(0), Y.stride(0), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code


@pytest.mark.parametrize("name", ["tiny", "p6"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_noalloc_matches_allocating_entry_point(name, prec):
    import torch
    fe = gpu_fe(name)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(31)
    for call in range(2):   # two calls in a row share the static scratch
        X = to_dev(rng.standard_normal((fe.ndof, 24 + 8 * call)), dt)
        ref = fe.apply_Sinv_approx(X, prec=prec).double().cpu().numpy()
        Y = torch.full_like(X, float("nan"))
        assert _noalloc(fe, prec, X, Y) == 0, fe._lib.paw_last_error()
        torch.cuda.synchronize()
        assert rel_err(Y.double().cpu().numpy(), ref) < TOL[prec]
    fe.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_strided_blocks(prec):
    """X and Y as column blocks of wider arrays (ld > ncols): only their own columns are
    read and written."""
    import torch
    fe = gpu_fe("p6")
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(32)
    Xw = to_dev(rng.standard_normal((fe.ndof, 40)), dt)
    Yw = torch.full((fe.ndof, 48), 7.0, dtype=dt, device="cuda")
    X, Y = Xw[:, 5:25], Yw[:, 11:31]
    ref = fe.apply_Sinv_approx(X.contiguous(), prec=prec).double().cpu().numpy()
    assert _noalloc(fe, prec, X, Y) == 0, fe._lib.paw_last_error()
    torch.cuda.synchronize()
    assert rel_err(Y.double().cpu().numpy(), ref) < TOL[prec]
    untouched = torch.cat([Yw[:, :11], Yw[:, 31:]], 1)
    assert bool((untouched == 7.0).all())
    fe.close()


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    import torch
    fe = gpu_fe("p6")
    X = torch.zeros((fe.ndof, 4), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    from paper_2604_26037_gb300 import _lib as L
    huge = 1 << 22   # columns; refused by the size check before any device access
    code = fe._lib.paw_apply_Sinv_approx_noalloc(fe._h, L.Precision.FP64, C.c_void_p(X.data_ptr()),
                                                 C.c_void_p(Y.data_ptr()), huge, huge, huge, None)
    assert code == 1
    assert b"scratch" in fe._lib.paw_last_error()
    fe.close()
