"""GB300 (sm_103a) FP64 stiffness assembly for 3D laminated solids.

Thin Python binding of the C ABI in ``include/lam.h`` (liblam.so, built in-tree
by ``paper_1905_05417_gb300.build``). Every step of the assembly runs in the
library's CUDA kernels; this module only marshals arguments. PyTorch supplies
device memory and streams. There is no CPU fallback: when the library is not
built or no GPU is present, the device calls raise.

Method: Antolin (2019), split assembly of K = sum_m sum_ab P_{m,ab} (x) Q_{m,ab}
(Section 3, Eq. Km_2) and the standard 3D quadrature (Section 2.4).

Module-level functions mirror the C entry points (``plan_create``,
``plan_get_info``, ``pattern``, ``assemble_split``, ``assemble_standard``,
``assemble_split_host``, ``plan_update``, ``plan_destroy``, ``last_error``,
``version``, ``adjoint``); ``Plan`` wraps them for convenience, and
``StiffnessFunction`` exposes the assembly and its adjoint to torch.autograd.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "LamError", "Plan", "load", "plan_create", "plan_destroy", "plan_get_info", "pattern", "assemble_split",
    "assemble_standard", "assemble_split_host", "assemble_split_noalloc", "plan_update", "profile_enable", "profile_get", "last_error",
    "version", "adjoint", "inplane_operators", "StiffnessFunction", "Batch", "batch_create", "batch_assemble", "batch_get_info",
    "batch_destroy", "SYMBOLS", "KERNEL_KINDS", "BSPLINE", "LAGRANGE", "ARITH_FP64", "ARITH_DOUBLE_FLOAT",
]

BSPLINE = 0
LAGRANGE = 1
ARITH_FP64 = 0
ARITH_DOUBLE_FLOAT = 1
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblam.so")

# every symbol include/lam.h declares
SYMBOLS = ("lam_plan_create", "lam_plan_destroy", "lam_plan_get_info", "lam_pattern", "lam_assemble_split",
           "lam_assemble_standard", "lam_assemble_split_host", "lam_assemble_split_noalloc", "lam_plan_update",
           "lam_adjoint", "lam_inplane_operators", "lam_batch_create", "lam_batch_assemble", "lam_batch_get_info", "lam_batch_destroy",
           "lam_profile_enable",
           "lam_profile_get", "lam_last_error", "lam_version")
KERNEL_KINDS = ("pattern", "thickness", "inplane", "combine", "standard", "adjoint", "adjoint_aux")
P_FROM_GRAM = 0
P_VOIGT_FREE = 1
COTANGENT_CSR = 0
COTANGENT_LOWRANK = 1
ADJOINT_FP64 = 1
ADJOINT_DOUBLE_FLOAT = 2

_STATUS = {0: "LAM_OK", 1: "LAM_ERR_INVALID_ARG", 2: "LAM_ERR_UNSUPPORTED", 3: "LAM_ERR_OOM", 4: "LAM_ERR_CUDA",
           5: "LAM_ERR_TIMEOUT"}


class LamError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {message}")
        self.status = status


class _Basis1d(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("degree", ctypes.c_int32), ("n_knots", ctypes.c_int32),
                ("knots", ctypes.POINTER(ctypes.c_double))]


class _Inplane(ctypes.Structure):
    _fields_ = [("u", _Basis1d), ("v", _Basis1d), ("ctrl", ctypes.POINTER(ctypes.c_double)),
                ("weights", ctypes.POINTER(ctypes.c_double)), ("ctrl_dim", ctypes.c_int32),
                ("extrusion", ctypes.c_double * 3)]


class _Ply(ctypes.Structure):
    _fields_ = [("thickness", ctypes.c_double), ("material", ctypes.c_int32), ("angle_rad", ctypes.c_double)]


class _Material(ctypes.Structure):
    _fields_ = [("C", ctypes.c_double * 21)]


class _Options(ctypes.Structure):
    _fields_ = [("nq_u", ctypes.c_int32), ("nq_v", ctypes.c_int32), ("nq_t", ctypes.c_int32),
                ("class_tol", ctypes.c_double), ("arith", ctypes.c_int32)]


class _Profile(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("launches", ctypes.c_int64 * 7), ("ms", ctypes.c_double * 7),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64)]


class _Cotangent(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rank", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("values", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("n_plans", ctypes.c_int32), ("n_meshes", ctypes.c_int32), ("nnz_total", ctypes.c_int64),
                ("n_persistent", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("rows_per_item", ctypes.c_int32), ("chunk_ctas", ctypes.c_int32), ("tuned_ms", ctypes.c_double * 36)]


class _Info(ctypes.Structure):
    _fields_ = [("n_dof", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_s", ctypes.c_int64), ("n_t", ctypes.c_int64),
                ("nnz_inplane", ctypes.c_int64), ("nnz_thickness", ctypes.c_int64), ("n_configs", ctypes.c_int32),
                ("n_classes", ctypes.c_int32), ("monoclinic", ctypes.c_int32), ("n_pieces", ctypes.c_int32),
                ("combine_streaming", ctypes.c_int32), ("combine_chunks", ctypes.c_int32), ("shell", ctypes.c_int32),
                ("arith", ctypes.c_int32), ("combine_terms", ctypes.c_int32),
                ("combine_source_terms", ctypes.c_int32), ("combine_block_terms", ctypes.c_int32)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def load() -> ctypes.CDLL:
    """Load liblam.so (built by ``paper_1905_05417_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1905_05417_gb300.build` "
                          "(the CUDA library is required; there is no fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    L.lam_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Inplane), ctypes.POINTER(_Basis1d),
                                  ctypes.POINTER(_Ply), ctypes.c_int32, ctypes.POINTER(_Material), ctypes.c_int32,
                                  ctypes.POINTER(_Options)]
    L.lam_plan_destroy.argtypes = [vp]
    L.lam_plan_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    L.lam_pattern.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), vp, vp, vp]
    L.lam_assemble_split.argtypes = [vp, vp, vp]
    L.lam_assemble_standard.argtypes = [vp, vp, vp]
    L.lam_assemble_split_host.argtypes = [vp, vp, vp]
    L.lam_assemble_split_noalloc.argtypes = [vp, vp, vp]
    L.lam_plan_update.argtypes = [vp, _D, ctypes.c_int32, ctypes.POINTER(_Material), ctypes.c_int32]
    L.lam_adjoint.argtypes = [vp, ctypes.POINTER(_Cotangent), vp, vp, vp, vp]
    L.lam_inplane_operators.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
    L.lam_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int32]
    L.lam_batch_assemble.argtypes = [vp, ctypes.POINTER(vp), vp]
    L.lam_batch_get_info.argtypes = [vp, ctypes.POINTER(_BatchInfo)]
    L.lam_batch_destroy.argtypes = [vp]
    L.lam_profile_enable.argtypes = [vp, ctypes.c_int32]
    L.lam_profile_get.argtypes = [vp, ctypes.POINTER(_Profile)]
    L.lam_last_error.restype = ctypes.c_char_p
    L.lam_version.restype = ctypes.c_char_p
    for name in SYMBOLS:
        if name not in ("lam_last_error", "lam_version"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def last_error() -> str:
    return load().lam_last_error().decode()


def version() -> str:
    return load().lam_version().decode()


def _check(status: int, where: str):
    if status != 0:
        raise LamError(status, where, last_error())


def _as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    """Device address of a torch tensor (or an int address; None for NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def plan_create(u, v, ctrl, t, ply_thickness, ply_material, ply_angle, C21, weights=None,
                nq: Sequence[int] = (0, 0, 0), class_tol: float = -1.0, extrusion=None,
                arith: int = 0) -> ctypes.c_void_p:
    """lam_plan_create. u, v, t are (kind, degree, knots); C21 is (n_materials, 21);
    ctrl is (n_s, 2) for a planar map or (n_s, 3) for a surface in R^3;
    extrusion is the direction a of F = S + xi^3 a (None: e_z); arith is
    ARITH_FP64 (default) or ARITH_DOUBLE_FLOAT."""
    L = load()
    keep = []

    def basis(b):
        kind, degree, knots = b
        k = _as_f64(knots)
        keep.append(k)
        return _Basis1d(int(kind), int(degree), len(k), k.ctypes.data_as(_D))

    ctrl = _as_f64(ctrl)
    keep.append(ctrl)
    cdim = ctrl.shape[1] if ctrl.ndim == 2 else 2
    if cdim not in (2, 3):
        raise ValueError("ctrl must have 2 or 3 columns")
    w = None if weights is None else _as_f64(weights)
    keep.append(w)
    a = (0.0, 0.0, 0.0) if extrusion is None else tuple(float(x) for x in extrusion)
    if len(a) != 3:
        raise ValueError("extrusion must have 3 components")
    ip = _Inplane(basis(u), basis(v), ctrl.ctypes.data_as(_D), w.ctypes.data_as(_D) if w is not None else _D(),
                  cdim, (ctypes.c_double * 3)(*a))
    tb = basis(t)
    h = _as_f64(ply_thickness)
    pm = np.ascontiguousarray(ply_material, dtype=np.int32)
    pa = _as_f64(ply_angle)
    n = len(h)
    if len(pm) != n or len(pa) != n:
        raise ValueError("ply arrays differ in length")
    plies = (_Ply * n)(*[_Ply(float(h[k]), int(pm[k]), float(pa[k])) for k in range(n)])
    C = np.atleast_2d(_as_f64(C21))
    if C.shape[1] != 21:
        raise ValueError("C21 must have 21 columns")
    mats = (_Material * C.shape[0])()
    for k in range(C.shape[0]):
        mats[k].C[:] = C[k].tolist()
    opt = _Options(int(nq[0]), int(nq[1]), int(nq[2]), float(class_tol), int(arith))
    handle = ctypes.c_void_p()
    _check(L.lam_plan_create(ctypes.byref(handle), ctypes.byref(ip), ctypes.byref(tb), plies, n, mats, C.shape[0],
                             ctypes.byref(opt)), "lam_plan_create")
    return handle


def plan_destroy(handle) -> None:
    _check(load().lam_plan_destroy(handle), "lam_plan_destroy")


def plan_get_info(handle) -> dict:
    info = _Info()
    _check(load().lam_plan_get_info(handle, ctypes.byref(info)), "lam_plan_get_info")
    return {name: getattr(info, name) for name, _ in _Info._fields_}


def pattern(handle, d_row_ptr=None, d_col_ind=None, stream=None) -> int:
    """lam_pattern. With no buffers, returns nnz only (host)."""
    nnz = ctypes.c_int64()
    if d_row_ptr is None and d_col_ind is None:
        _check(load().lam_pattern(handle, ctypes.byref(nnz), None, None, None), "lam_pattern")
        return nnz.value
    _check(load().lam_pattern(handle, ctypes.byref(nnz), _ptr(d_row_ptr), _ptr(d_col_ind), _stream_handle(stream)),
           "lam_pattern")
    return nnz.value


def assemble_split(handle, d_values, stream=None) -> None:
    _check(load().lam_assemble_split(handle, _ptr(d_values), _stream_handle(stream)), "lam_assemble_split")


def assemble_split_noalloc(handle, d_values, stream=None) -> None:
    """lam_assemble_split_noalloc: the split assembly with its tables and
    workspace in the library's fixed static device array (no allocation)."""
    _check(load().lam_assemble_split_noalloc(handle, _ptr(d_values), _stream_handle(stream)),
           "lam_assemble_split_noalloc")


def assemble_standard(handle, d_values, stream=None) -> None:
    _check(load().lam_assemble_standard(handle, _ptr(d_values), _stream_handle(stream)), "lam_assemble_standard")


def assemble_split_host(handle, h_values, stream=None) -> None:
    """h_values: a host buffer (numpy float64 array or pinned torch CPU tensor)."""
    if isinstance(h_values, np.ndarray):
        if h_values.dtype != np.float64 or not h_values.flags.c_contiguous:
            raise ValueError("h_values must be a contiguous float64 array")
        addr = h_values.ctypes.data
    else:
        addr = h_values.data_ptr()
    _check(load().lam_assemble_split_host(handle, addr, _stream_handle(stream)), "lam_assemble_split_host")


def plan_update(handle, ply_angle=None, C21=None) -> None:
    pa = None if ply_angle is None else _as_f64(ply_angle)
    mats, nm = None, 0
    if C21 is not None:
        C = np.atleast_2d(_as_f64(C21))
        mats = (_Material * C.shape[0])()
        for k in range(C.shape[0]):
            mats[k].C[:] = C[k].tolist()
        nm = C.shape[0]
    _check(load().lam_plan_update(handle, pa.ctypes.data_as(_D) if pa is not None else _D(),
                                  0 if pa is None else len(pa), mats, nm), "lam_plan_update")


def adjoint(handle, d_dC=None, d_dtheta=None, d_dD=None, values=None, u=None, v=None, rank=1, fp64=False,
            stream=None, double_float=False) -> None:
    """lam_adjoint: gradients of L = sum(values * K) (values on the pattern) or
    of L = sum_q u_q^T K v_q (u, v: rank x n_dof) into the given device buffers.
    fp64: LAM_ADJOINT_FP64 (low rank through the generic pass); double_float:
    LAM_ADJOINT_DOUBLE_FLOAT (CSR cotangents, opt-in)."""
    c = _Cotangent()
    if values is not None:
        c.kind, c.values = COTANGENT_CSR, _ptr(values)
    else:
        c.kind, c.rank, c.u, c.v = COTANGENT_LOWRANK, int(rank), _ptr(u), _ptr(v)
    c.flags = (ADJOINT_FP64 if fp64 else 0) | (ADJOINT_DOUBLE_FLOAT if double_float else 0)
    _check(load().lam_adjoint(handle, ctypes.byref(c), _ptr(d_dC), _ptr(d_dtheta), _ptr(d_dD), _stream_handle(stream)),
           "lam_adjoint")


def inplane_operators(handle, ply: int, method: int, d_P, stream=None) -> None:
    """lam_inplane_operators: Eq. P for ply `ply`'s material into d_P (nnz_inplane x 4 x 3 x 3)."""
    _check(load().lam_inplane_operators(handle, int(ply), int(method), _ptr(d_P), _stream_handle(stream)),
           "lam_inplane_operators")


def batch_create(plan_handles) -> ctypes.c_void_p:
    """lam_batch_create over plan handles (the plans must outlive the batch)."""
    arr = (ctypes.c_void_p * len(plan_handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                                    for h in plan_handles])
    out = ctypes.c_void_p()
    _check(load().lam_batch_create(ctypes.byref(out), arr, len(plan_handles)), "lam_batch_create")
    return out


def batch_assemble(handle, d_values, stream=None) -> None:
    """d_values: one device tensor (or address) per plan, in the plans' order."""
    arr = (ctypes.c_void_p * len(d_values))(*[_ptr(v) for v in d_values])
    _check(load().lam_batch_assemble(handle, arr, _stream_handle(stream)), "lam_batch_assemble")


def batch_get_info(handle) -> dict:
    info = _BatchInfo()
    _check(load().lam_batch_get_info(handle, ctypes.byref(info)), "lam_batch_get_info")
    out = {name: getattr(info, name) for name, _ in _BatchInfo._fields_ if name != "tuned_ms"}
    out["tuned_ms"] = list(info.tuned_ms)
    return out


def batch_destroy(handle) -> None:
    _check(load().lam_batch_destroy(handle), "lam_batch_destroy")


def profile_enable(handle, enable: bool = True) -> None:
    """lam_profile_enable: start (or stop) timing every launch; counters restart."""
    _check(load().lam_profile_enable(handle, 1 if enable else 0), "lam_profile_enable")


def profile_get(handle) -> dict:
    """lam_profile_get: per kernel kind, launches and device milliseconds; bytes moved."""
    pr = _Profile()
    _check(load().lam_profile_get(handle, ctypes.byref(pr)), "lam_profile_get")
    out = {"enabled": bool(pr.enabled), "h2d_bytes": pr.h2d_bytes, "d2h_bytes": pr.d2h_bytes}
    for k, name in enumerate(KERNEL_KINDS):
        out[name] = {"launches": pr.launches[k], "ms": pr.ms[k]}
    return out


class Plan:
    """Convenience owner of a lam_plan handle; outputs are torch tensors."""

    def __init__(self, u, v, ctrl, t, ply_thickness, ply_material, ply_angle, C21, weights=None,
                 nq=(0, 0, 0), class_tol=-1.0, extrusion=None, arith=0):
        self.handle = plan_create(u, v, ctrl, t, ply_thickness, ply_material, ply_angle, C21, weights=weights,
                                  nq=nq, class_tol=class_tol, extrusion=extrusion, arith=arith)
        self.info = plan_get_info(self.handle)
        self.n_plies = len(ply_thickness)
        self.n_materials = int(np.atleast_2d(np.asarray(C21)).shape[0])

    @classmethod
    def from_laminate(cls, lam, class_tol=-1.0, arith=0) -> "Plan":
        """Build from any object with the fields u, v, t (kind, degree, knots),
        ctrl, weights, ply_thickness, ply_material, ply_angle, C21, nq."""
        b = lambda x: (x.kind, x.degree, x.knots)
        return cls(b(lam.u), b(lam.v), lam.ctrl, b(lam.t), lam.ply_thickness, lam.ply_material, lam.ply_angle,
                   lam.C21, weights=lam.weights, nq=tuple(lam.nq), class_tol=class_tol,
                   extrusion=getattr(lam, "extrusion", None), arith=arith)

    @property
    def nnz(self) -> int:
        return self.info["nnz"]

    @property
    def n_dof(self) -> int:
        return self.info["n_dof"]

    def pattern(self, stream=None):
        import torch
        row_ptr = torch.empty(self.n_dof + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(self.nnz, dtype=torch.int32, device="cuda")
        pattern(self.handle, row_ptr, col, stream)
        return row_ptr, col

    def assemble_split(self, values=None, stream=None):
        import torch
        if values is None:
            values = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        assemble_split(self.handle, values, stream)
        return values

    def assemble_standard(self, values=None, stream=None):
        import torch
        if values is None:
            values = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        assemble_standard(self.handle, values, stream)
        return values

    def assemble_split_host(self, values=None, stream=None):
        if values is None:
            values = np.empty(self.nnz, dtype=np.float64)
        assemble_split_host(self.handle, values, stream)
        return values

    def update(self, ply_angle=None, C21=None):
        plan_update(self.handle, ply_angle, C21)
        self.info = plan_get_info(self.handle)

    def inplane_operators(self, ply: int, method: int = P_FROM_GRAM, stream=None):
        """Eq. P of every in-plane pair for ply `ply`'s material: (nnz_inplane, 4, 3, 3) device tensor."""
        import torch
        P = torch.empty(self.info["nnz_inplane"], 4, 3, 3, dtype=torch.float64, device="cuda")
        inplane_operators(self.handle, ply, method, P, stream)
        return P

    def adjoint(self, values=None, u=None, v=None, fp64=False, want_dD=True, stream=None, double_float=False):
        """(dL/dC: n_materials x 21, dL/dtheta: n_plies, dL/dD: n_plies x 6 x 6 or None)
        for L = sum(values * K) or L = sum_q u_q^T K v_q; device tensors."""
        import torch
        dC = torch.empty(self.n_materials, 21, dtype=torch.float64, device="cuda")
        dth = torch.empty(self.n_plies, dtype=torch.float64, device="cuda")
        dD = torch.empty(self.n_plies, 6, 6, dtype=torch.float64, device="cuda") if want_dD else None
        rank = 1
        if values is None:
            u, v = u.reshape(-1, self.n_dof).contiguous(), v.reshape(-1, self.n_dof).contiguous()
            rank = u.shape[0]
            if v.shape[0] != rank:
                raise ValueError("u and v must have the same number of rows")
        adjoint(self.handle, dC, dth, dD, values=values, u=u, v=v, rank=rank, fp64=fp64, stream=stream,
                double_float=double_float)
        return dC, dth, dD

    def profile_enable(self, enable=True):
        profile_enable(self.handle, enable)

    def profile(self) -> dict:
        return profile_get(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many plans assembled together (lam_batch_*); keeps the plans alive."""

    def __init__(self, plans):
        self.plans = list(plans)
        self.handle = batch_create([p.handle for p in self.plans])

    @property
    def info(self) -> dict:
        return batch_get_info(self.handle)

    def assemble(self, values=None, stream=None):
        import torch
        if values is None:
            values = [torch.empty(p.nnz, dtype=torch.float64, device="cuda") for p in self.plans]
        batch_assemble(self.handle, values, stream)
        return values

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stiffness_function():
    import torch

    class StiffnessFunction(torch.autograd.Function):
        """values = K(C21, ply_angle) on the plan's pattern (lam_assemble_split),
        differentiable in the constants and the angles through lam_adjoint.
        The plan is updated to the given constants and angles (host copies)."""

        @staticmethod
        def forward(ctx, plan, C21, ply_angle):
            plan.update(ply_angle=ply_angle.detach().cpu().numpy(), C21=C21.detach().cpu().numpy())
            ctx.plan = plan
            ctx.devices = (C21.device, ply_angle.device)
            return plan.assemble_split()

        @staticmethod
        def backward(ctx, grad_values):
            dC, dth, _ = ctx.plan.adjoint(values=grad_values.contiguous(), want_dD=False)
            return None, dC.to(ctx.devices[0]), dth.to(ctx.devices[1])

    return StiffnessFunction


def __getattr__(name):
    if name == "StiffnessFunction":
        fn = _stiffness_function()
        globals()["StiffnessFunction"] = fn
        return fn
    raise AttributeError(name)
