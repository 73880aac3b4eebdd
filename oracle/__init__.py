"""Python access to the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference legs use it. The product package never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain C, -O2, no OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Basis(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("degree", ctypes.c_int32), ("n_knots", ctypes.c_int32),
                ("knots", ctypes.POINTER(ctypes.c_double))]


class _Problem(ctypes.Structure):
    _fields_ = [("u", _Basis), ("v", _Basis), ("ctrl", ctypes.POINTER(ctypes.c_double)),
                ("weights", ctypes.POINTER(ctypes.c_double)), ("t", _Basis), ("n_plies", ctypes.c_int32),
                ("ply_thickness", ctypes.POINTER(ctypes.c_double)),
                ("ply_material", ctypes.POINTER(ctypes.c_int32)),
                ("ply_angle", ctypes.POINTER(ctypes.c_double)), ("n_materials", ctypes.c_int32),
                ("C21", ctypes.POINTER(ctypes.c_double)), ("nq_u", ctypes.c_int32), ("nq_v", ctypes.c_int32),
                ("nq_t", ctypes.c_int32), ("ctrl_dim", ctypes.c_int32),
                ("extrusion", ctypes.POINTER(ctypes.c_double))]


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def configure(L):
    """Declare the argument types of an oracle library handle."""
    if True:
        L.ora_gauss.argtypes = [ctypes.c_int32, _D, _D]
        L.ora_nfun.argtypes = [ctypes.POINTER(_Basis)]
        L.ora_nfun.restype = ctypes.c_int32
        L.ora_nel.argtypes = [ctypes.POINTER(_Basis)]
        L.ora_nel.restype = ctypes.c_int32
        L.ora_basis1d_eval.argtypes = [ctypes.POINTER(_Basis), ctypes.c_int32, ctypes.c_double, _D, _D, _I32]
        L.ora_rotated_D.argtypes = [_D, ctypes.c_double, _D]
        L.ora_rotated_D.restype = None
        L.ora_sizes.argtypes = [ctypes.POINTER(_Problem), _I64, _I64]
        for f in (L.ora_assemble, L.ora_assemble_split):
            f.argtypes = [ctypes.POINTER(_Problem), _I64, _I32, _D]
        L.ora_pattern.argtypes = [ctypes.POINTER(_Problem), _I64, _I32]
        L.ora_adjoint_D.argtypes = [ctypes.POINTER(_Problem), _I64, _I32, _D, _D]
        L.ora_adjoint.argtypes = [ctypes.POINTER(_Problem), _I64, _I32, _D, _D, _D, _D]
        L.ora_inplane_P.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int, ctypes.c_int64, ctypes.c_int64, _D]
        L.ora_rotated_D_dtheta.argtypes = [_D, ctypes.c_double, _D]
        L.ora_rotated_D_dtheta.restype = None
        L.ora_block.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int64, ctypes.c_int64, _D]
        L.ora_element_stiffness.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _D]
        L.ora_assemble_elements.argtypes = [ctypes.POINTER(_Problem), _I64, _I32, _I32, ctypes.c_int32, _D]
        L.ora_inplane_row_blocks.argtypes = [ctypes.POINTER(_Problem), ctypes.c_int64, _I32, _D]
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = configure(ctypes.CDLL(_SO))
    return _lib


def _ptr(a, t=_D):
    return a.ctypes.data_as(t)


class Problem:
    """Marshals a ``workloads.Laminate`` into the oracle's problem struct and
    keeps the arrays alive."""

    def __init__(self, lam):
        self._keep = []

        def arr(x, dt=np.float64):
            a = np.ascontiguousarray(x, dtype=dt)
            self._keep.append(a)
            return a

        def basis(b):
            k = arr(b.knots)
            return _Basis(b.kind, b.degree, len(k), _ptr(k))

        ctrl = arr(lam.ctrl)
        w = arr(lam.weights) if lam.weights is not None else None
        h = arr(lam.ply_thickness)
        pm = arr(lam.ply_material, np.int32)
        pa = arr(lam.ply_angle)
        C = arr(lam.C21)
        nq = tuple(lam.nq) + (0,) * (3 - len(lam.nq))
        ext = getattr(lam, "extrusion", None)
        ext = arr(ext) if ext is not None else None
        self.s = _Problem(basis(lam.u), basis(lam.v), _ptr(ctrl), _ptr(w) if w is not None else _D(),
                          basis(lam.t), len(h), _ptr(h), _ptr(pm, _I32), _ptr(pa), C.shape[0], _ptr(C),
                          nq[0], nq[1], nq[2], int(ctrl.shape[1]) if ctrl.ndim == 2 else 2,
                          _ptr(ext) if ext is not None else _D())
        self.lam = lam

    def ref(self):
        return ctypes.byref(self.s)


def gauss(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().ora_gauss(n, _ptr(x), _ptr(w)) != 0:
        raise ValueError("bad Gauss order")
    return x, w


def basis1d_eval(kind: int, degree: int, knots, e: int, x: float):
    k = np.ascontiguousarray(knots, dtype=np.float64)
    b = _Basis(kind, degree, len(k), _ptr(k))
    val = np.zeros(degree + 1)
    der = np.zeros(degree + 1)
    first = ctypes.c_int32()
    if lib().ora_basis1d_eval(ctypes.byref(b), e, x, _ptr(val), _ptr(der), ctypes.byref(first)) != 0:
        raise ValueError("bad element")
    return first.value, val, der


def n_functions(kind: int, degree: int, knots) -> int:
    k = np.ascontiguousarray(knots, dtype=np.float64)
    b = _Basis(kind, degree, len(k), _ptr(k))
    return lib().ora_nfun(ctypes.byref(b))


def n_elements(kind: int, degree: int, knots) -> int:
    k = np.ascontiguousarray(knots, dtype=np.float64)
    b = _Basis(kind, degree, len(k), _ptr(k))
    return lib().ora_nel(ctypes.byref(b))


def rotated_D(C21, theta: float) -> np.ndarray:
    C = np.ascontiguousarray(C21, dtype=np.float64)
    D = np.zeros(36)
    lib().ora_rotated_D(_ptr(C), float(theta), _ptr(D))
    return D.reshape(6, 6)


def sizes(lam):
    p = Problem(lam)
    n = ctypes.c_int64()
    z = ctypes.c_int64()
    if lib().ora_sizes(p.ref(), ctypes.byref(n), ctypes.byref(z)) != 0:
        raise ValueError("oracle rejected the problem")
    return n.value, z.value


def _assemble(lam, fn):
    p = Problem(lam)
    n_dof, nnz = sizes(lam)
    row_ptr = np.zeros(n_dof + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    if fn(p.ref(), _ptr(row_ptr, _I64), _ptr(col, _I32), _ptr(val)) != 0:
        raise ValueError("oracle assembly failed")
    return row_ptr, col, val


def pattern(lam):
    """Sparsity pattern only: (row_ptr int64, col int32)."""
    p = Problem(lam)
    n_dof, nnz = sizes(lam)
    row_ptr = np.zeros(n_dof + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    if lib().ora_pattern(p.ref(), _ptr(row_ptr, _I64), _ptr(col, _I32)) != 0:
        raise ValueError("oracle pattern failed")
    return row_ptr, col


def assemble(lam):
    """Standard element-by-element assembly: (row_ptr int64, col int32, val f64)."""
    return _assemble(lam, lib().ora_assemble)


def assemble_split(lam):
    """Split assembly with one P per ply (small problems only)."""
    return _assemble(lam, lib().ora_assemble_split)


def adjoint_D(lam, row_ptr, col, gbar) -> np.ndarray:
    """dL/dD_l (n_plies x 6 x 6) for L = sum(gbar * K) on the oracle's pattern."""
    p = Problem(lam)
    out = np.zeros(36 * len(lam.ply_thickness))
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    g = np.ascontiguousarray(gbar, dtype=np.float64)
    if lib().ora_adjoint_D(p.ref(), _ptr(rp, _I64), _ptr(cl, _I32), _ptr(g), _ptr(out)) != 0:
        raise ValueError("oracle adjoint failed")
    return out.reshape(-1, 6, 6)


def adjoint(lam, row_ptr, col, gbar):
    """(dL/dC: n_materials x 21, dL/dtheta: n_plies, dL/dD: n_plies x 6 x 6)
    for L = sum(gbar * K) on the oracle's pattern."""
    p = Problem(lam)
    n_pl, n_mat = len(lam.ply_thickness), lam.C21.shape[0]
    dD = np.zeros(36 * n_pl)
    dC = np.zeros(21 * n_mat)
    dth = np.zeros(n_pl)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    g = np.ascontiguousarray(gbar, dtype=np.float64)
    if lib().ora_adjoint(p.ref(), _ptr(rp, _I64), _ptr(cl, _I32), _ptr(g), _ptr(dD), _ptr(dC), _ptr(dth)) != 0:
        raise ValueError("oracle adjoint failed")
    return dC.reshape(n_mat, 21), dth, dD.reshape(n_pl, 6, 6)


def lowrank_cotangent(row_ptr, col, u, v) -> np.ndarray:
    """Values of sum_r u_r v_r^T on the pattern (row-major CSR order): the
    cotangent of L = sum_r u_r^T K v_r."""
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    out = np.zeros(len(col))
    for r in range(u.shape[0]):
        out += u[r][rows] * v[r][col]
    return out


def inplane_P(lam, ply: int, i_s: int, j_s: int, problem: "Problem | None" = None) -> np.ndarray:
    """Eq. P for in-plane functions (i_s, j_s) and the material of `ply`:
    array (4, 3, 3) of the blocks 11, 12, 21, 22."""
    p = problem if problem is not None else Problem(lam)
    out = np.zeros(36)
    if lib().ora_inplane_P(p.ref(), int(ply), int(i_s), int(j_s), _ptr(out)) != 0:
        raise ValueError("oracle inplane_P failed")
    return out.reshape(4, 3, 3)


def rotated_D_dtheta(C21, theta: float) -> np.ndarray:
    out = np.zeros(36)
    c = np.ascontiguousarray(C21, dtype=np.float64)
    lib().ora_rotated_D_dtheta(_ptr(c), float(theta), _ptr(out))
    return out.reshape(6, 6)


def block(lam, i: int, j: int, problem: Problem | None = None) -> np.ndarray:
    p = problem if problem is not None else Problem(lam)
    out = np.zeros(9)
    if lib().ora_block(p.ref(), int(i), int(j), _ptr(out)) != 0:
        raise ValueError("bad block index")
    return out.reshape(3, 3)


def element_stiffness(lam, ex: int, ey: int, et: int, problem: Problem | None = None) -> np.ndarray:
    p = problem if problem is not None else Problem(lam)
    nl = (lam.u.degree + 1) * (lam.v.degree + 1) * (lam.t.degree + 1)
    out = np.zeros(nl * nl * 9)
    if lib().ora_element_stiffness(p.ref(), ex, ey, et, _ptr(out)) < 0:
        raise ValueError("element stiffness failed")
    return out.reshape(nl, nl, 3, 3)


def element_colours(lam):
    """The 3D elements (ex, ey, et) grouped so that no two elements of a group
    share a basis function: colour (ex mod (p_u + 1), ey mod (p_v + 1),
    et mod (q + 1)), each group an int32 array of triples."""
    nex, ney = n_elements(lam.u.kind, lam.u.degree, lam.u.knots), n_elements(lam.v.kind, lam.v.degree, lam.v.knots)
    net = n_elements(lam.t.kind, lam.t.degree, lam.t.knots)
    cu, cv, ct = lam.u.degree + 1, lam.v.degree + 1, lam.t.degree + 1
    groups = []
    for kt in range(ct):
        for ky in range(cv):
            for kx in range(cu):
                ex, ey, et = np.meshgrid(np.arange(kx, nex, cu), np.arange(ky, ney, cv), np.arange(kt, net, ct),
                                         indexing="ij")
                g = np.stack([ex.ravel(), ey.ravel(), et.ravel()], axis=1).astype(np.int32)
                if len(g):
                    groups.append(np.ascontiguousarray(g))
    return groups


def assemble_elements(lam, row_ptr, col, elems, val, problem: Problem | None = None) -> None:
    """Adds the element stiffness of the listed elements (int32 triples) into
    val on the CSR pattern (row_ptr, col) of pattern(lam). The C call releases
    the GIL, so lists of one colour may run on several threads at once."""
    p = problem if problem is not None else Problem(lam)
    e = np.ascontiguousarray(elems, dtype=np.int32)
    if lib().ora_assemble_elements(p.ref(), _ptr(row_ptr, _I64), _ptr(col, _I32), _ptr(e, _I32), len(e),
                                   _ptr(val)) != 0:
        raise ValueError("oracle element-list assembly failed")


def inplane_row_blocks(lam, i_s: int, problem: Problem | None = None):
    """Every 3x3 block of the rows (i_t, i_s) for all i_t: returns (bx0, by0,
    blocks[it, jt, jy - by0, jx - bx0, 3, 3]). The C call releases the GIL."""
    p = problem if problem is not None else Problem(lam)
    nt = n_functions(lam.t.kind, lam.t.degree, lam.t.knots)
    nbmax = (2 * lam.u.degree + 1) * (2 * lam.v.degree + 1)
    out = np.zeros(9 * nt * nt * nbmax)
    box = np.zeros(4, np.int32)
    if lib().ora_inplane_row_blocks(p.ref(), int(i_s), _ptr(box, _I32), _ptr(out)) != 0:
        raise ValueError("oracle row blocks failed")
    bx0, nbx, by0, nby = (int(x) for x in box)
    return bx0, by0, out[:9 * nt * nt * nbx * nby].reshape(nt, nt, nby, nbx, 3, 3)


def to_dense(row_ptr, col, val, n):
    K = np.zeros((n, n))
    for r in range(n):
        s, e = row_ptr[r], row_ptr[r + 1]
        K[r, col[s:e]] = val[s:e]
    return K
