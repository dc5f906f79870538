"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point include/paw_fe.h declares, and rejects bad arguments
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2604_26037_gb300 as P
from paper_2604_26037_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:paw_status|const char \*)\s*(paw_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    P.build_library()
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, f"{n} has no binding"


def test_version(lib):
    assert b"sm_103a" in lib.paw_version()


def _create(lib, **kw):
    args = dict(L=10.0, n=2, degree=3, periodic=1, natoms=0, D=None, dS=None, shells=())
    args.update(kw)
    mesh = L._Mesh((C.c_double * 3)(args["L"], args["L"], args["L"]),
                   (C.c_int32 * 3)(args["n"], args["n"], args["n"]),
                   (C.c_int32 * 3)(args["periodic"], 1, 1))
    pos = np.zeros((max(args["natoms"], 1), 3))
    atoms = L._Atoms(args["natoms"], pos.ctypes.data_as(L._DP))
    ls = np.array([l for l, _ in args["shells"]] or [0], dtype=np.int32)
    ws = np.array([w for _, w in args["shells"]] or [1.0])
    proj = L._Proj(len(args["shells"]), ls.ctypes.data_as(C.POINTER(C.c_int32)), ws.ctypes.data_as(L._DP))
    D = args["D"] if args["D"] is not None else np.zeros(1)
    dS = args["dS"] if args["dS"] is not None else np.zeros(1)
    h = C.c_void_p()
    opts = None
    if "kpoint" in args:
        opts = C.byref(L._Opts(0, 0, 0, 0, (C.c_double * 3)(*args["kpoint"]), int(args.get("y0_pair32", 0)), 0))
    code = lib.paw_fe_create(C.byref(mesh), args["degree"], C.byref(atoms), C.byref(proj),
                             D.ctypes.data_as(L._DP), dS.ctypes.data_as(L._DP), None, opts, C.byref(h))
    return code, lib.paw_last_error().decode()


def test_rejects_bad_arguments_before_device_work(lib):
    assert _create(lib, periodic=0)[0] == 2
    assert _create(lib, degree=9)[0] == 2
    assert _create(lib, degree=0)[0] == 2
    assert _create(lib, L=-1.0)[0] == 1
    # asymmetric coupling matrix
    D = np.zeros((1, 1, 1))
    Da = np.zeros((1, 4, 4))
    Da[0, 0, 1] = 1.0
    code, msg = _create(lib, natoms=1, shells=((0, 0.5), (1, 0.5)), D=Da, dS=np.zeros((1, 4, 4)))
    assert code == 1 and "symmetric" in msg
    # l = 3 is not supported
    assert _create(lib, natoms=1, shells=((3, 0.5),), D=D, dS=D)[0] == 2
    # cutoff reaching half the box
    assert _create(lib, natoms=1, shells=((0, 1.0),), D=D, dS=D)[0] == 2


def test_rejects_bad_kpoint_arguments_before_device_work(lib):
    # a Bloch wavevector stores 2 nproj real projectors: at most 16 projectors per atom
    shells = ((2, 0.5), (2, 0.5), (2, 0.5), (2, 0.5))
    D = np.zeros((1, 20, 20))
    code, msg = _create(lib, natoms=1, shells=shells, D=D, dS=D, kpoint=(0.1, 0.0, 0.0))
    assert code == 2 and "16 projectors" in msg
    code, msg = _create(lib, kpoint=(float("nan"), 0.0, 0.0))
    assert code == 1 and "kpoint" in msg
    # pair-of-FP32 step 2 is implemented for real vectors only
    code, msg = _create(lib, kpoint=(0.1, 0.0, 0.0), y0_pair32=1)
    assert code == 2 and "y0_pair32" in msg


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.paw_apply_H(None, 0, None, None, 4, 4, 4, None) == 1
    assert lib.paw_sync_status(None) == 1
    assert lib.paw_set_wait_limit(None, 1.0, 0) == 1
    assert lib.paw_destroy(None) == 0
    b = L._Bounds(1.0, 0.5, 2.0)
    lam = np.zeros(1)
    assert lib.paw_cheb_filter(None, 0, None, 1, lam.ctypes.data_as(L._DP), 1, 3, b, None, 1, None) == 1


def test_precision_names():
    assert L.Precision.of("tf32") == 2 and L.Precision.of("FP64") == 0
    assert L.Precision.of("f32x2") == L.Precision.F32X2 == 4


def _header():
    return open(os.path.join(ROOT, "include", "paw_fe.h")).read()


def test_options_struct_matches_header():
    """paw_options field order in the header is the binding's ctypes layout."""
    body = re.search(r"typedef struct \{([^{}]*)\} paw_options;", _header()).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)(?:\[\d+\])?;", body)
    assert fields == [f for f, _ in L._Opts._fields_]


def test_precision_enum_matches_header():
    vals = dict((k, int(v)) for k, v in re.findall(r"PAW_(FP64|FP32|TF32|BF16|F32X2) = (\d+)", _header()))
    assert vals == {k: getattr(L.Precision, k) for k in vals} and len(vals) == 5


def test_sinv_entry_points_reject_the_same_requests(lib):
    """paw_apply_Sinv_approx and its allocation-free variant share their argument checks:
    the same request gets the same status code from both (checked before the handle)."""
    for prec, code in ((L.Precision.F32X2, 2), (17, 1)):
        a = lib.paw_apply_Sinv_approx(None, prec, None, None, 4, 4, 4, None)
        b = lib.paw_apply_Sinv_approx_noalloc(None, prec, None, None, 4, 4, 4, None)
        assert a == b == code, (prec, a, b)
    for args in ((4, 4, 4), (-1, 4, 4)):   # NULL handle, then a bad column count
        assert lib.paw_apply_Sinv_approx(None, 0, None, None, *args, None) == \
            lib.paw_apply_Sinv_approx_noalloc(None, 0, None, None, *args, None) == 1
