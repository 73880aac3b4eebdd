"""The oracle's pins catch plausible mistakes.

Each case copies oracle.c, plants one mistake (a transposed operand, a wrong
index or sign, a dropped term, the paper's misprints taken literally), builds
the copy on the CPU, and runs a battery of quick pins against it. Every planted
mistake must make at least one pin fail, and the unmodified oracle must pass
them all.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle as O
import workloads as W
from tests import exact_rational as X

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

MUTATIONS = {
    # the misprint of the third row of B^T (gamma_23 from the third gradient component twice)
    "gamma23_misprint": ("B[5][1] = g[2]; B[5][2] = g[1];", "B[5][1] = g[2]; B[5][2] = g[2];"),
    # pull-back with DF^{-1} instead of DF^{-T}
    "jacobian_transposed": ("ip->g1[k][0] = Ji[0][0] * R1[k] + Ji[1][0] * R2[k];",
                            "ip->g1[k][0] = Ji[0][0] * R1[k] + Ji[0][1] * R2[k];"),
    # Cox-de Boor with its second term dropped
    "coxdeboor_dropped_term": ("  if (d2 > 0.0) v += (t[i + p + 1] - x) / d2 * bs_value(t, i + 1, p - 1, span, x);\n",
                               "\n"),
    # rotation by -theta
    "rotation_sign": ("double R[3][3] = {{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}};\n  static const int pairs",
                      "double R[3][3] = {{c, s, 0.0}, {-s, c, 0.0}, {0.0, 0.0, 1.0}};\n  static const int pairs"),
    # tensor (1/2) instead of engineering shear in gamma_12
    "half_shear": ("B[3][0] = g[1]; B[3][1] = g[0];", "B[3][0] = 0.5 * g[1]; B[3][1] = 0.5 * g[0];"),
    # Jacobian determinant dropped from the weight
    "no_jacobian": ("    ip->detJ = fabs(det);\n    return 0;", "    ip->detJ = 1.0;\n    return 0;"),
    # general extrusion: pull-back with DF^{-1} instead of DF^{-T} (columns of the inverse)
    "shell_dual_transposed": ("ip->g1[k][c] = g[0][c] * R1[k] + g[1][c] * R2[k];",
                              "ip->g1[k][c] = g[c][0] * R1[k] + g[c][1] * R2[k];"),
    # general extrusion: the thickness gradient along a itself instead of its dual vector
    "shell_r3_is_a": ("for (int c = 0; c < 3; ++c) ip->r3[c] = g[2][c];",
                      "for (int c = 0; c < 3; ++c) ip->r3[c] = A[2][c];"),
    # general extrusion: the cofactors not divided by det DF
    "shell_no_det_division": ("for (int c = 0; c < 3; ++c) g[k][c] = t[c] / det;",
                              "for (int c = 0; c < 3; ++c) g[k][c] = t[c];"),
    # general extrusion: only the z component of a taken
    "shell_extrusion_dropped": ("A[2][0] = pr->extrusion[0];\n    A[2][1] = pr->extrusion[1];",
                                "A[2][0] = 0.0;\n    A[2][1] = 0.0;"),
    # general extrusion: the third coordinate of the surface ignored
    "shell_surface_flattened": ("      for (int c = 0; c < cd; ++c) {\n        A[0][c] += R1[k] * X[c];",
                                "      for (int c = 0; c < 2; ++c) {\n        A[0][c] += R1[k] * X[c];"),
    # Gauss weights off by a factor
    "gauss_weight": ("w[n - 1 - k] = 2.0 / ((1.0 - z * z) * dpn * dpn);",
                     "w[n - 1 - k] = 1.0 / ((1.0 - z * z) * dpn * dpn);"),
    # the printed Eq. Q: Q_12 and Q_21 exchanged
    "q12_q21_swapped": ("q[1] += w * T[a] * dT[b];\n              q[2] += w * dT[a] * T[b];",
                        "q[1] += w * dT[a] * T[b];\n              q[2] += w * T[a] * dT[b];"),
    # Voigt matrix read with one index pair swapped (13 <-> 23)
    "voigt_index": ("if ((i == 0 && j == 2) || (i == 2 && j == 0)) return 4;\n  return 5;",
                    "if ((i == 0 && j == 2) || (i == 2 && j == 0)) return 5;\n  return 4;"),
    # NURBS quotient rule with a wrong sign
    "nurbs_quotient": ("R1[k] = wk * (N1[k] * W - N[k] * W1) / (W * W);", "R1[k] = wk * (N1[k] * W + N[k] * W1) / (W * W);"),
    # ply of a piece taken from the wrong neighbour
    "ply_lookup": ("if (mid < top) break;", "if (mid <= top - 1e-300 && l > 0) break;"),
}


def build_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: anchor not found exactly once"
    path = tmp_path / f"oracle_{name}.c"
    path.write_text(src.replace(old, new))
    (tmp_path / "oracle.h").write_text(open(os.path.join(os.path.dirname(SRC), "oracle.h")).read())
    so = tmp_path / f"liboracle_{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-I", str(tmp_path), "-o", str(so),
                           str(path), "-lm"])
    return O.configure(ctypes.CDLL(str(so)))


EXACT_C = X.exact_orthotropic_C21(**W.PLY_CONSTANTS)


def battery():
    """Quick pins; returns the names of the pins that fail."""
    failed = []
    x, w = O.gauss(4)
    xr, wr = np.polynomial.legendre.leggauss(4)
    if not (np.allclose(x, xr, atol=1e-14) and np.allclose(w, wr, atol=1e-14)):
        failed.append("gauss")
    knots = W.open_uniform_knots(3, 4)
    for e in range(4):
        xx = (e + 0.37) / 4
        first, val, der = O.basis1d_eval(0, 3, knots, e, xx)
        for k in range(4):
            c = np.zeros(len(knots) - 4)
            c[first + k] = 1.0
            if abs(val[k] - BSpline(knots, c, 3)(xx)) > 1e-13:
                failed.append("bspline")
                break
    rng = np.random.default_rng(3)
    C = W.random_C21(rng)
    Cm = np.zeros((6, 6))
    k = 0
    for I in range(6):
        for J in range(I, 6):
            Cm[I, J] = Cm[J, I] = C[k]
            k += 1
    th = 0.4
    D = O.rotated_D(C, th)
    c, s = math.cos(th), math.sin(th)
    R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
    A = rng.standard_normal((3, 3))
    Eg = 0.5 * (A + A.T)
    Em = R.T @ Eg @ R
    tv = lambda E: np.array([E[0, 0], E[1, 1], E[2, 2], 2 * E[0, 1], 2 * E[0, 2], 2 * E[1, 2]])
    if abs(tv(Eg) @ D @ tv(Eg) - tv(Em) @ Cm @ tv(Em)) > 1e-10 * abs(tv(Em) @ Cm @ tv(Em)):
        failed.append("rotation_energy")
    # exact rational brick with a 45-degree ply and a 0/90 pair
    lam = W.laminate("b", W.BSPLINE, 2, 1, [45.0, 0.0, 90.0], [0.3, 0.2, 0.2], mapping=W.scaled_map(1.0, 2.0))
    rp, col, val = O.assemble(lam)
    blocks = sorted({(r // 3, col[kk] // 3) for r in range(0, lam.n_dof, 7) for kk in range(rp[r], rp[r + 1], 5)})
    ex = X.exact_box_blocks(lam, 1.0, 2.0, [EXACT_C], [45, 0, 90], blocks)
    err = 0.0
    for r in range(0, lam.n_dof, 7):
        for kk in range(rp[r], rp[r + 1], 5):
            err = max(err, abs(val[kk] - ex[(r // 3, col[kk] // 3)][r % 3, col[kk] % 3]))
    if not err <= 1e-12 * np.abs(val).max():
        failed.append("exact_box")
    # curved map: rigid modes and the patch test, with random NURBS weights too
    for weighted in (False, True):
        lam = W.curved_plate(n_el=3, degree=2, repeats=1)
        if weighted:
            lam.weights = np.random.default_rng(5).uniform(0.5, 2.0, lam.n_s)
        rp, col, val = O.assemble(lam)
        K = O.to_dense(rp, col, val, lam.n_dof)
        zt = W.anchors(lam.t)
        P = np.zeros((lam.n_s * lam.n_t, 3))
        for it in range(lam.n_t):
            P[it * lam.n_s:(it + 1) * lam.n_s, :2] = lam.ctrl
            P[it * lam.n_s:(it + 1) * lam.n_s, 2] = zt[it]
        for Wm in (np.array([[0, 0, 0], [0, 0, -1.0], [0, 1.0, 0]]), np.array([[0, -1.0, 0], [1.0, 0, 0], [0, 0, 0]])):
            r = (P @ Wm.T).reshape(-1)
            if np.abs(K @ r).max() > 1e-11 * np.abs(K).max() * np.abs(r).max():
                failed.append("rigid_modes")
        if not weighted:
            lam.ply_angle[:] = 0.0
            rp, col, val = O.assemble(lam)
            Kh = O.to_dense(rp, col, val, lam.n_dof)
            u = (P @ rng.standard_normal((3, 3)).T).reshape(-1)
            res = (Kh @ u).reshape(-1, 3)
            nx, ny, nt = lam.u.n_functions, lam.v.n_functions, lam.n_t
            inner = [it * nx * ny + iy * nx + ix for it in range(1, nt - 1) for iy in range(1, ny - 1)
                     for ix in range(1, nx - 1)]
            if np.abs(res[inner]).max() > 1e-10 * np.abs(Kh).max() * np.abs(u).max():
                failed.append("patch")
    # general extrusion: exact rational rotated and sheared slab, rigid modes of a curved shell
    from tests import test_oracle_shell as S
    A = S.AFFINE_CASES["rotated_general"]
    lam = S.affine_laminate(A, n_el=1)
    rp, col, val = O.assemble(lam)
    blocks = sorted({(r // 3, col[kk] // 3) for r in range(0, lam.n_dof, 7) for kk in range(rp[r], rp[r + 1], 5)})
    ex = X.exact_affine_blocks(lam, A, [EXACT_C], [45, 0, 90], blocks)
    err = 0.0
    for r in range(0, lam.n_dof, 7):
        for kk in range(rp[r], rp[r + 1], 5):
            err = max(err, abs(val[kk] - ex[(r // 3, col[kk] // 3)][r % 3, col[kk] % 3]))
    if not err <= 1e-12 * np.abs(val).max():
        failed.append("exact_affine_extrusion")
    lam = W.shell_plate(n_el=2, degree=2, repeats=1, extrusion=(0.3, 0.2, 0.9))
    K = O.to_dense(*O.assemble(lam), lam.n_dof)
    if S.rigid_mode_residual(K, S.shell_coords(lam)) > 1e-12:
        failed.append("shell_rigid_modes")
    # split formula equals the standard one
    lam = W.curved_plate(n_el=2, degree=2, repeats=1)
    a = O.assemble(lam)[2]
    b = O.assemble_split(lam)[2]
    if np.abs(a - b).max() > 1e-12 * np.abs(a).max():
        failed.append("split_equals_standard")
    return failed


def test_unmodified_oracle_passes_the_battery():
    assert battery() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, monkeypatch, name):
    old, new = MUTATIONS[name]
    mutated = build_variant(tmp_path, name, old, new)
    monkeypatch.setattr(O, "_lib", mutated)
    try:
        failed = battery()
    except Exception as exc:  # a crash or a rejected problem also exposes the mistake
        failed = [f"exception: {exc!r}"]
    assert failed, f"planted mistake {name} passed every pin"
