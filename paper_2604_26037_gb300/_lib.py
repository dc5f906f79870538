"""ctypes binding of libpawfe (names follow include/paw_fe.h)."""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpawfe.so")
_lib = None
_lock = threading.Lock()


class Precision:
    FP64 = 0
    FP32 = 1
    TF32 = 2
    BF16 = 3
    F32X2 = 4   # FP64 data, pair-of-FP32 arithmetic (apply_H / apply_S)
    names = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "f32x2": 4}

    @classmethod
    def of(cls, p) -> int:
        if isinstance(p, str):
            return cls.names[p.lower()]
        return int(p)


STATUS = {0: "PAW_OK", 1: "PAW_ERR_INVALID_ARG", 2: "PAW_ERR_UNSUPPORTED", 3: "PAW_ERR_NOT_SPD",
          4: "PAW_ERR_CUDA", 5: "PAW_ERR_NO_MEMORY", 6: "PAW_ERR_TIMEOUT", 7: "PAW_ERR_NONFINITE",
          8: "PAW_ERR_LIBRARY"}


class PawError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class _Mesh(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("n_cells", C.c_int32 * 3), ("periodic", C.c_int32 * 3)]


class _Atoms(C.Structure):
    _fields_ = [("natoms", C.c_int32), ("positions", C.POINTER(C.c_double))]


class _Proj(C.Structure):
    _fields_ = [("nshells", C.c_int32), ("l", C.POINTER(C.c_int32)), ("width", C.POINTER(C.c_double))]


class _Vloc(C.Structure):
    _fields_ = [("ngauss", C.c_int32), ("centers", C.POINTER(C.c_double)),
                ("depth", C.POINTER(C.c_double)), ("width", C.POINTER(C.c_double))]


class _Opts(C.Structure):
    _fields_ = [("block", C.c_int32), ("pp_overlap", C.c_int32), ("y0_fp32", C.c_int32),
                ("rr_mixed", C.c_int32), ("kpoint", C.c_double * 3), ("y0_pair32", C.c_int32),
                ("no_overlap", C.c_int32)]


class _Bounds(C.Structure):
    _fields_ = [("a0", C.c_double), ("bW", C.c_double), ("bU", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("ndof", C.c_int64), ("ncells", C.c_int32), ("nodes_per_cell", C.c_int32),
                ("quad_per_cell", C.c_int32), ("natoms", C.c_int32), ("nproj", C.c_int32),
                ("degree", C.c_int32), ("support_pairs", C.c_int64), ("device_bytes", C.c_int64),
                ("owner_pairs", C.c_int64), ("nproj_padded", C.c_int32), ("complex_vectors", C.c_int32),
                ("proj_nnz", C.c_int64)]


class _Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("intervals", C.c_int64 * 6), ("launches", C.c_int64 * 6),
                ("total_launches", C.c_int64)]


class _BatchProblem(C.Structure):
    _fields_ = [("X_in", C.c_void_p), ("ldx", C.c_int32), ("lambda_in", C.POINTER(C.c_double)),
                ("ncols", C.c_int32), ("degree", C.c_int32), ("bounds", _Bounds),
                ("X_out", C.c_void_p), ("ldo", C.c_int32)]


class _BatchOpts(C.Structure):
    _fields_ = [("streams", C.c_int32), ("autotune", C.c_int32), ("reserved", C.c_int32 * 6)]


class _BatchTuning(C.Structure):
    _fields_ = [("tc_variant", C.c_int32), ("grid_cap", C.c_int32), ("branch", C.c_int32),
                ("branches", C.c_int32), ("graph_nodes", C.c_int32), ("kernel_nodes", C.c_int32),
                ("captures", C.c_int32), ("tuned_ms", C.c_double * 2)]


_VP, _I, _D, _DP = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)
SIGNATURES = {
    "paw_fe_create": [C.POINTER(_Mesh), _I, C.POINTER(_Atoms), C.POINTER(_Proj), _DP, _DP,
                      C.POINTER(_Vloc), C.POINTER(_Opts), C.POINTER(_VP)],
    "paw_set_veff": [_VP, _VP],
    "paw_set_dij": [_VP, _DP],
    "paw_get_info": [_VP, C.POINTER(_Info)],
    "paw_apply_H": [_VP, _I, _VP, _VP, _I, _I, _I, _VP],
    "paw_apply_S": [_VP, _I, _VP, _VP, _I, _I, _I, _VP],
    "paw_apply_Sinv_approx": [_VP, _I, _VP, _VP, _I, _I, _I, _VP],
    "paw_apply_Sinv_approx_noalloc": [_VP, _I, _VP, _VP, _I, _I, _I, _VP],
    "paw_cheb_filter": [_VP, _I, _VP, _I, _DP, _I, _I, _Bounds, _VP, _I, _VP],
    "paw_batch_create": [C.POINTER(_VP), _I, C.POINTER(_BatchOpts), C.POINTER(_VP)],
    "paw_batch_cheb_filter": [_VP, _I, C.POINTER(_BatchProblem), C.POINTER(C.c_int), _VP],
    "paw_batch_tuning_get": [_VP, _I, C.POINTER(_BatchTuning)],
    "paw_batch_destroy": [_VP],
    "paw_rayleigh_ritz": [_VP, _VP, _I, _I, _DP, _VP],
    "paw_residuals": [_VP, _VP, _I, _DP, _I, _DP, _VP],
    "paw_lanczos_bounds": [_VP, _I, C.c_uint64, _DP, _DP, _VP],
    "paw_energy": [_VP, _I, _VP, _I, _I, _DP, _VP],
    "paw_energy_grad": [_VP, _I, _VP, _I, _I, _VP, _VP, _VP],
    "paw_density": [_VP, _I, _VP, _I, _I, _DP, _VP, _VP, _VP],
    "paw_profile_enable": [_VP, _I],
    "paw_profile_read": [_VP, C.c_void_p],
    "paw_sync_status": [_VP],
    "paw_set_wait_limit": [_VP, _D, _I],
    "paw_destroy": [_VP],
    "paw_last_error": [],
    "paw_version": [],
}


def lib_path() -> str:
    return _LIB_PATH


def build_library(force: bool = False) -> str:
    from . import build as _b
    return _b.build(force=force)


def load_library():
    """Load libpawfe.so; raises ImportError if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with "
                              "paper_2604_26037_gb300.build_library() (nvcc, sm_103a)")
        lib = C.CDLL(_LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_char_p if name in ("paw_last_error", "paw_version") else C.c_int
        _lib = lib
        return lib


def _check(code):
    if code != 0:
        msg = load_library().paw_last_error()
        raise PawError(code, msg.decode() if msg else "")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _stream(t=None):
    import torch
    dev = t.device if t is not None else torch.device("cuda")
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _mat(t, dtype=None):
    """(pointer, rows, cols, ld) of a 2D CUDA tensor with unit column stride."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dim() != 2:
        raise ValueError("expected a 2D (ndof x ncols) tensor")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError("the vector index must be the fastest (stride(1) == 1)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    ld = t.stride(0) if t.shape[1] > 0 else 1
    return C.c_void_p(t.data_ptr()), t.shape[0], t.shape[1], max(ld, t.shape[1])


class PawFE:
    """One PAW finite-element problem on the current CUDA device."""

    def __init__(self, L, ncell, degree, positions=(), shells=(), D=None, dS=None,
                 vloc=None, block=256, pp_overlap=False, y0_fp32=False, rr_mixed=False, kpoint=None,
                 y0_pair32=False, overlap=True):
        self._lib = load_library()
        pos = np.ascontiguousarray(np.asarray(positions, float).reshape(-1, 3))
        na = pos.shape[0]
        ls = np.ascontiguousarray([int(l) for l, _ in shells], dtype=np.int32)
        ws = np.ascontiguousarray([float(w) for _, w in shells], dtype=np.float64)
        npj = int(sum(2 * l + 1 for l, _ in shells))
        self.natoms, self.nproj = na, npj
        mesh = _Mesh((C.c_double * 3)(L, L, L), (C.c_int32 * 3)(ncell, ncell, ncell),
                     (C.c_int32 * 3)(1, 1, 1))
        atoms = _Atoms(na, _dptr(pos))
        proj = _Proj(len(ls), ls.ctypes.data_as(C.POINTER(C.c_int32)), _dptr(ws))
        Dh = np.ascontiguousarray(np.zeros((na, npj, npj)) if D is None else np.asarray(D, float))
        dSh = np.ascontiguousarray(np.zeros((na, npj, npj)) if dS is None else np.asarray(dS, float))
        keep = [pos, ls, ws, Dh, dSh]
        vp = None
        if vloc is not None:
            cen = np.ascontiguousarray(np.asarray(vloc["centers"], float).reshape(-1, 3))
            dep = np.ascontiguousarray(np.asarray(vloc["depth"], float))
            wid = np.ascontiguousarray(np.asarray(vloc["width"], float))
            keep += [cen, dep, wid]
            vp = C.pointer(_Vloc(cen.shape[0], _dptr(cen), _dptr(dep), _dptr(wid)))
        kp = (0.0, 0.0, 0.0) if kpoint is None else tuple(float(x) for x in kpoint)
        opts = _Opts(int(block), int(bool(pp_overlap)), int(bool(y0_fp32)), int(bool(rr_mixed)),
                     (C.c_double * 3)(*kp), int(bool(y0_pair32)), int(not overlap))
        h = C.c_void_p()
        _check(self._lib.paw_fe_create(C.byref(mesh), int(degree), C.byref(atoms), C.byref(proj),
                                       _dptr(Dh), _dptr(dSh), vp, C.byref(opts), C.byref(h)))
        self._h = h
        del keep
        info = _Info()
        _check(self._lib.paw_get_info(self._h, C.byref(info)))
        self.ndof = int(info.ndof)
        self.ncells = int(info.ncells)
        self.nodes_per_cell = int(info.nodes_per_cell)
        self.quad_per_cell = int(info.quad_per_cell)
        self.support_pairs = int(info.support_pairs)
        self.owner_pairs = int(info.owner_pairs)
        self.nproj_padded = int(info.nproj_padded)
        self.proj_nnz = int(info.proj_nnz)
        self.complex = bool(info.complex_vectors)   # k != 0: complex multivectors
        self.block = int(block)

    @classmethod
    def from_system(cls, sysd: dict, **kw):
        vloc = dict(centers=sysd["vloc_centers"], depth=sysd["vloc_depth"], width=sysd["vloc_width"])
        return cls(sysd["L"], sysd["ncell"], sysd["p"], sysd["positions"], sysd["shells"],
                   sysd["D"], sysd["dS"], vloc=vloc, **kw)

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self._lib.paw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        info = _Info()
        _check(self._lib.paw_get_info(self._h, C.byref(info)))
        return {k: getattr(info, k) for k, _ in _Info._fields_}

    def sync_status(self):
        """Raise PawError (PAW_ERR_TIMEOUT) if a kernel of an earlier, asynchronous call
        (cheb_filter) gave up on a bounded wait; synchronises the handle's stream."""
        _check(self._lib.paw_sync_status(self._h))

    def set_wait_limit(self, seconds=2.0, probe=False):
        """Give-up bound of the tensor-core pipelines' waits; probe=True makes their
        launches wait on a word nothing sets, so they give up (failure-path check)."""
        _check(self._lib.paw_set_wait_limit(self._h, float(seconds), int(bool(probe))))

    PHASES = ("residual_local", "recurrence", "projection", "cell_products", "residual_nonlocal", "recovery")

    def profile_enable(self, on=True):
        _check(self._lib.paw_profile_enable(self._h, int(bool(on))))

    def profile_read(self) -> dict:
        prof = _Profile()
        _check(self._lib.paw_profile_read(self._h, C.byref(prof)))
        out = {name: dict(ms=prof.ms[i], intervals=prof.intervals[i], launches=prof.launches[i])
               for i, name in enumerate(self.PHASES)}
        out["total_launches"] = prof.total_launches
        return out

    # ------------------------------------------------------------------ operators
    def _apply(self, fn, X, Y, prec):
        import torch
        prec = Precision.of(prec)
        if self.complex:
            dt = torch.complex128 if prec in (Precision.FP64, Precision.F32X2) else torch.complex64
        else:
            dt = torch.float64 if prec in (Precision.FP64, Precision.F32X2) else torch.float32
        xp, rows, n, ldx = _mat(X, dt)
        if rows != self.ndof:
            raise ValueError(f"X has {rows} rows, expected {self.ndof}")
        if Y is None:
            Y = torch.empty((self.ndof, n), dtype=dt, device=X.device)
        yp, _, ny, ldy = _mat(Y, dt)
        if ny != n:
            raise ValueError("X and Y column counts differ")
        _check(fn(self._h, prec, xp, yp, n, ldx, ldy, _stream(X)))
        return Y

    def apply_H(self, X, Y=None, prec="fp64"):
        return self._apply(self._lib.paw_apply_H, X, Y, prec)

    def apply_S(self, X, Y=None, prec="fp64"):
        return self._apply(self._lib.paw_apply_S, X, Y, prec)

    def apply_Sinv_approx(self, X, Y=None, prec="fp64"):
        return self._apply(self._lib.paw_apply_Sinv_approx, X, Y, prec)

    # ------------------------------------------------------------------ filter
    def _fp64(self):
        import torch
        return torch.complex128 if self.complex else torch.float64

    def cheb_filter(self, X, lam, degree, bounds, prec="tf32", out=None):
        """Algorithm 2 on the columns of X (stream-ordered: returns once enqueued;
        sync_status() reports a kernel that gave up on a bounded wait)."""
        import torch
        xp, rows, n, ldx = _mat(X, self._fp64())
        if out is None:
            out = torch.empty((self.ndof, n), dtype=self._fp64(), device=X.device)
        op, _, n2, ldo = _mat(out, self._fp64())
        lam = np.ascontiguousarray(np.asarray(lam, float).reshape(-1))
        if n2 != n or lam.size != n:
            raise ValueError("column counts of X, out and lambda differ")
        a0, bW, bU = bounds
        _check(self._lib.paw_cheb_filter(self._h, Precision.of(prec), xp, ldx, _dptr(lam), n, int(degree),
                                         _Bounds(a0, bW, bU), op, ldo, _stream(X)))
        return out

    def rayleigh_ritz(self, X):
        xp, rows, n, ld = _mat(X, self._fp64())
        lam = np.zeros(n)
        _check(self._lib.paw_rayleigh_ritz(self._h, xp, ld, n, _dptr(lam), _stream(X)))
        return lam

    def residuals(self, X, lam):
        xp, rows, n, ld = _mat(X, self._fp64())
        lam = np.ascontiguousarray(np.asarray(lam, float))
        out = np.zeros(n)
        _check(self._lib.paw_residuals(self._h, xp, ld, _dptr(lam), n, _dptr(out), _stream(X)))
        return out

    def lanczos_bounds(self, k=20, seed=7):
        tmin, up = C.c_double(), C.c_double()
        _check(self._lib.paw_lanczos_bounds(self._h, int(k), C.c_uint64(seed), C.byref(tmin), C.byref(up),
                                            _stream()))
        return tmin.value, up.value

    # ------------------------------------------------------------------ gradient
    def set_veff(self, Vq):
        import torch
        if not (isinstance(Vq, torch.Tensor) and Vq.is_cuda and Vq.dtype == torch.float64
                and Vq.is_contiguous() and Vq.numel() == self.ncells * self.quad_per_cell):
            raise ValueError("Vq must be a contiguous CUDA float64 tensor (ncells x nq)")
        _check(self._lib.paw_set_veff(self._h, C.c_void_p(Vq.data_ptr())))

    def set_dij(self, D):
        D = np.ascontiguousarray(np.asarray(D, float))
        _check(self._lib.paw_set_dij(self._h, _dptr(D)))

    def energy(self, X, prec="fp64"):
        import torch
        prec = Precision.of(prec)
        xp, rows, n, ld = _mat(X, torch.float64 if prec == Precision.FP64 else torch.float32)
        E = C.c_double()
        _check(self._lib.paw_energy(self._h, prec, xp, ld, n, C.byref(E), _stream(X)))
        return E.value

    def energy_grad(self, X, prec="fp64"):
        import torch
        prec = Precision.of(prec)
        xp, rows, n, ld = _mat(X, torch.float64 if prec == Precision.FP64 else torch.float32)
        dV = torch.empty((self.ncells, self.quad_per_cell), dtype=torch.float64, device=X.device)
        dD = torch.zeros((max(self.natoms, 1), self.nproj, self.nproj), dtype=torch.float64, device=X.device)
        _check(self._lib.paw_energy_grad(self._h, prec, xp, ld, n, C.c_void_p(dV.data_ptr()),
                                         C.c_void_p(dD.data_ptr()), _stream(X)))
        return dV, dD[: self.natoms]

    def density(self, X, occ=None, prec="fp64"):
        """(rho at the Gauss points of every cell, occupation matrices D^a) of the block X."""
        import torch
        prec = Precision.of(prec)
        xp, rows, n, ld = _mat(X, torch.float64 if prec == Precision.FP64 else torch.float32)
        rho = torch.empty((self.ncells, self.quad_per_cell), dtype=torch.float64, device=X.device)
        Dm = torch.zeros((max(self.natoms, 1), self.nproj, self.nproj), dtype=torch.float64, device=X.device)
        f = None if occ is None else np.ascontiguousarray(np.asarray(occ, float).reshape(-1))
        if f is not None and f.size != n:
            raise ValueError("one occupation per column")
        _check(self._lib.paw_density(self._h, prec, xp, ld, n, _dptr(f) if f is not None else None,
                                     C.c_void_p(rho.data_ptr()), C.c_void_p(Dm.data_ptr()), _stream(X)))
        return rho, Dm[: self.natoms]


class PawBatch:
    """Many PawFE instances filtered by one CUDA-graph launch per call
    (paw_batch_create / paw_batch_cheb_filter).  The instances stay owned by
    the caller and must outlive the batch."""

    def __init__(self, instances, streams=4, autotune=True):
        self._lib = load_library()
        self.instances = list(instances)
        hs = (_VP * len(self.instances))(*[fe._h for fe in self.instances])
        opts = _BatchOpts(int(streams), 1 if autotune else 0)
        h = _VP()
        _check(self._lib.paw_batch_create(hs, len(self.instances), C.byref(opts), C.byref(h)))
        self._h = h
        self._keep = ()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.paw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cheb_filter(self, problems, prec="tf32", raise_on_error=True):
        """problems: one (X, lam, degree, (a0, bW, bU), out) tuple per instance,
        or None to skip it.  Returns the list of per-instance status codes."""
        import torch
        n = len(self.instances)
        if len(problems) != n:
            raise ValueError("one problem per instance")
        arr = (_BatchProblem * n)()
        keep = []
        stream = None
        for i, q in enumerate(problems):
            if q is None:
                arr[i].ncols = 0
                continue
            X, lam, degree, bounds, out = q
            xp, _, nc, ldx = _mat(X, torch.float64)
            op, _, nc2, ldo = _mat(out, torch.float64)
            lam = np.ascontiguousarray(np.asarray(lam, float).reshape(-1))
            keep.append(lam)
            arr[i].X_in, arr[i].ldx = xp.value, ldx
            arr[i].lambda_in = _dptr(lam)
            arr[i].ncols, arr[i].degree = nc, int(degree)
            arr[i].bounds = _Bounds(*bounds)
            arr[i].X_out, arr[i].ldo = op.value, ldo
            stream = stream or _stream(X)
        st = (C.c_int * n)()
        code = self._lib.paw_batch_cheb_filter(self._h, Precision.of(prec), arr, st,
                                               stream if stream is not None else C.c_void_p(0))
        if code != 0 and raise_on_error:
            _check(code)
        return list(st)

    def tuning(self, i) -> dict:
        t = _BatchTuning()
        _check(self._lib.paw_batch_tuning_get(self._h, int(i), C.byref(t)))
        d = {k: getattr(t, k) for k, _ in _BatchTuning._fields_ if k != "tuned_ms"}
        d["tuned_ms"] = list(t.tuned_ms)
        return d


def _subspace_energy_cls():
    import torch

    class SubspaceEnergy(torch.autograd.Function):
        """E = tr(X^T H(V, Delta_H) X) with X fixed; backward by the adjoint kernels.

        forward(Vq, D, X, fe, prec): Vq (ncells x nq, float64 CUDA) and D
        (natoms x npj x npj, float64) define H; returns a 0-d tensor.
        """

        @staticmethod
        def forward(ctx, Vq, D, X, fe, prec="fp64"):
            fe.set_veff(Vq.detach().contiguous())
            fe.set_dij(D.detach().cpu().numpy())
            E = fe.energy(X, prec)
            ctx.fe, ctx.prec, ctx.d_device = fe, prec, D.device
            ctx.save_for_backward(X)
            return torch.tensor(E, dtype=torch.float64, device=Vq.device)

        @staticmethod
        def backward(ctx, gE):
            (X,) = ctx.saved_tensors
            dV, dD = ctx.fe.energy_grad(X, ctx.prec)
            return gE * dV, (gE * dD).to(ctx.d_device), None, None, None

    return SubspaceEnergy


class _LazyEnergy:
    _cls = None

    def __getattr__(self, name):
        if _LazyEnergy._cls is None:
            _LazyEnergy._cls = _subspace_energy_cls()
        return getattr(_LazyEnergy._cls, name)


SubspaceEnergy = _LazyEnergy()
