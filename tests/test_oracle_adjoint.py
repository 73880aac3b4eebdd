"""Pins of the oracle's adjoint (gradients of L = sum gbar * K).

K is linear in every ply's Voigt matrix D_l (Eq. Km_0, Section 3), and D_l is
linear in the material constants and a trigonometric function of the ply angle
(Eq. D and the rotation remark of Section 3). The pins: the exact rational
coefficient of each D_l entry on affine boxes, Euler's identity for a
homogeneous function of degree one, central finite differences of the oracle's
assembly in the constants and the angles, the rotation derivative against
finite differences, isotropy (no angle dependence), the period pi in the angle,
and the rigid-body null space (a cotangent u v^T with u a rigid motion gives a
zero gradient). No GPU is needed.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests import exact_rational as X


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def random_cotangent(lam, seed):
    rp, col, _ = O.assemble(lam)
    g = np.random.default_rng(seed).standard_normal(len(col))
    return rp, col, g


def dense(rp, col, g, n_dof):
    D = np.zeros((n_dof, n_dof))
    rows = np.repeat(np.arange(n_dof), np.diff(rp))
    D[rows, col] = g
    n_b = n_dof // 3
    return D.reshape(n_b, 3, n_b, 3)


def L_of(lam, gbar):
    return float(gbar @ O.assemble(lam)[2])


BOXES = {
    "bspline_p2_three_plies": lambda: W.laminate("b", W.BSPLINE, 2, 2, [0, 90, 45], [0.1, 0.2, 0.1],
                                                 mapping=W.scaled_map(2.0, 1.5)),
    "lagrange_q1_linear_thickness": lambda: W.laminate("l", W.LAGRANGE, 1, 2, [0, 30], 0.25,
                                                       mapping=W.scaled_map(1.0, 3.0), thickness_kind=W.LAGRANGE,
                                                       thickness_degree=1, n_el_y=3),
    # one thickness element across three plies: pieces cut at the interfaces
    "single_thickness_element": lambda: W.laminate("s", W.BSPLINE, 1, 2, [0, 90, 0], [0.1, 0.3, 0.2],
                                                   mapping=W.scaled_map(1.0, 1.0),
                                                   thickness=W.single_element_thickness(0.6, 3)),
}


@pytest.mark.parametrize("name", sorted(BOXES))
def test_dL_dD_exact_on_boxes(name):
    lam = BOXES[name]()
    Lx, Ly = {"bspline_p2_three_plies": (2.0, 1.5), "lagrange_q1_linear_thickness": (1.0, 3.0),
              "single_thickness_element": (1.0, 1.0)}[name]
    rp, col, g = random_cotangent(lam, 3)
    ref = X.exact_box_dL_dD(lam, Lx, Ly, dense(rp, col, g, lam.n_dof))
    got = O.adjoint_D(lam, rp, col, g)
    assert rel(got, ref) <= 1e-12


def test_euler_identity_on_curved_nurbs_plate():
    lam = W.curved_plate(n_el=2, degree=2, repeats=1)
    lam.weights = np.random.default_rng(2).uniform(0.6, 1.7, lam.n_s)
    rp, col, g = random_cotangent(lam, 5)
    dD = O.adjoint_D(lam, rp, col, g)
    Ds = [O.rotated_D(lam.C21[lam.ply_material[l]], lam.ply_angle[l]) for l in range(len(lam.ply_angle))]
    lhs = sum(float(np.sum(dD[l] * Ds[l])) for l in range(len(Ds)))
    L = L_of(lam, g)
    assert abs(lhs - L) <= 1e-12 * np.abs(g).sum() * np.abs(O.assemble(lam)[2]).max()


def _two_material_plate():
    rng = np.random.default_rng(8)
    mats = np.array([W.ply_C21(), W.random_C21(rng)])
    return W.laminate("m2", W.BSPLINE, 2, 2, [0, 35, -60, 90], 0.05, mapping=W.curved_map(0.04),
                      materials=mats, ply_material=[0, 1, 1, 0])


def test_dC_matches_finite_differences():
    """L is linear in the constants, so the central difference is exact up to rounding."""
    lam = _two_material_plate()
    rp, col, g = random_cotangent(lam, 6)
    dC, _, _ = O.adjoint(lam, rp, col, g)
    fd = np.zeros_like(dC)
    base = lam.C21.copy()
    for m in range(base.shape[0]):
        for k in range(21):
            h = 1e-3 * max(abs(base[m, k]), 1.0)
            lam.C21 = base.copy(); lam.C21[m, k] += h
            Lp = L_of(lam, g)
            lam.C21 = base.copy(); lam.C21[m, k] -= h
            Lm = L_of(lam, g)
            fd[m, k] = (Lp - Lm) / (2 * h)
    lam.C21 = base
    assert rel(dC, fd) <= 1e-8


def test_dtheta_matches_finite_differences():
    lam = _two_material_plate()
    rp, col, g = random_cotangent(lam, 7)
    _, dth, _ = O.adjoint(lam, rp, col, g)
    base = lam.ply_angle.copy()
    h = 1e-5
    fd = np.zeros_like(dth)
    for l in range(len(base)):
        lam.ply_angle = base.copy(); lam.ply_angle[l] += h
        Lp = L_of(lam, g)
        lam.ply_angle = base.copy(); lam.ply_angle[l] -= h
        Lm = L_of(lam, g)
        fd[l] = (Lp - Lm) / (2 * h)
    lam.ply_angle = base
    assert rel(dth, fd) <= 1e-7


def test_rotation_derivative_matches_finite_differences():
    C = W.random_C21(np.random.default_rng(1))
    for th in (0.0, 0.3, -1.1, 2.5):
        h = 1e-5
        fd = (O.rotated_D(C, th + h) - O.rotated_D(C, th - h)) / (2 * h)
        assert rel(O.rotated_D_dtheta(C, th), fd) <= 1e-8


def test_isotropic_material_has_no_angle_gradient():
    lam = W.laminate("iso", W.BSPLINE, 2, 2, [10, 70, -20], 0.05, mapping=W.curved_map(0.03),
                     materials=W.isotropic_C21(70.0, 0.3)[None, :])
    rp, col, g = random_cotangent(lam, 9)
    dC, dth, dD = O.adjoint(lam, rp, col, g)
    assert np.abs(dth).max() <= 1e-12 * np.abs(dD).max() * np.abs(lam.C21).max()


def test_angle_period_pi():
    """A rotation by pi about z is diag(-1, -1, 1): it maps a material symmetric
    about the mid-plane (orthotropic here) onto itself, so K and dL/dtheta are
    unchanged, while the derivative in a constant that couples an odd number of
    z indices (exactly one Voigt index in {13, 23}) changes sign."""
    lam = _two_material_plate()
    C2 = W.ply_C21().copy()
    C2[0] *= 1.25
    lam.C21 = np.array([W.ply_C21(), C2])
    rp, col, g = random_cotangent(lam, 10)
    a = O.adjoint(lam, rp, col, g)
    lam.ply_angle = lam.ply_angle + np.pi
    b = O.adjoint(lam, rp, col, g)
    sign = np.array([-1.0 if ((I in (4, 5)) != (J in (4, 5))) else 1.0 for I in range(6) for J in range(I, 6)])
    assert rel(b[0], a[0] * sign) <= 1e-12
    assert rel(b[1], a[1]) <= 1e-10
    assert np.array_equal(b[2], a[2])  # dL/dD does not depend on D


def rigid_modes(lam):
    """Three translations and three rotations of the control net (z = the
    thickness coordinate of each thickness function's Greville point)."""
    X2 = lam.ctrl
    zt = W.greville(lam.t.knots, lam.t.degree)
    n_s = lam.n_s
    modes = []
    for k in range(3):
        r = np.zeros((lam.n_dof // 3, 3)); r[:, k] = 1.0
        modes.append(r.ravel())
    x = np.tile(X2[:, 0], len(zt)); y = np.tile(X2[:, 1], len(zt)); z = np.repeat(zt, n_s)
    for (i, j, a, b) in ((0, 1, x, y), (0, 2, x, z), (1, 2, y, z)):
        r = np.zeros((lam.n_dof // 3, 3)); r[:, i] = -b; r[:, j] = a
        modes.append(r.ravel())
    return modes


def test_rigid_motion_cotangent_has_zero_gradient():
    """K r = 0 for every D, so u^T K r has zero derivative in every D_l."""
    lam = W.curved_plate(n_el=2, degree=2, repeats=1)
    rp, col, val = O.assemble(lam)
    u = np.random.default_rng(12).standard_normal(lam.n_dof)
    scale = np.abs(O.adjoint_D(lam, rp, col, O.lowrank_cotangent(rp, col, u, u))).max()
    for r in rigid_modes(lam):
        dD = O.adjoint_D(lam, rp, col, O.lowrank_cotangent(rp, col, u, r))
        assert np.abs(dD).max() <= 1e-11 * scale * max(1.0, np.abs(r).max())


def test_lowrank_cotangent_is_the_outer_product_on_the_pattern():
    lam = W.cross_ply_plate(n_el=2, n_plies=2)
    rp, col, _ = O.assemble(lam)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal((2, lam.n_dof)), rng.standard_normal((2, lam.n_dof))
    g = O.lowrank_cotangent(rp, col, u, v)
    full = u.T @ v
    rows = np.repeat(np.arange(lam.n_dof), np.diff(rp))
    assert np.array_equal(g, full[rows, col]) or rel(g, full[rows, col]) < 1e-15


# ------------------------------------------------------------------ planted mistakes
ADJOINT_MUTATIONS = {
    # the cotangent block read transposed (c <-> d)
    "cotangent_transposed": ("gl[((size_t)a * nl + b) * 9 + c * 3 + d] = gbar[row_ptr[r] + 3 * k + d];",
                             "gl[((size_t)a * nl + b) * 9 + d * 3 + c] = gbar[row_ptr[r] + 3 * k + d];"),
    # one of the four product-rule terms of the rotation derivative dropped
    "dtheta_term_dropped": (" + R[i][p] * R[j][q] * R[kk][r] * dR[l][t];", ";"),
    # constants' derivative taken at the opposite angle
    "dC_angle_sign": ("ora_rotated_D(e, pr->ply_angle[l], R);", "ora_rotated_D(e, -pr->ply_angle[l], R);"),
    # the Jacobian determinant dropped from the adjoint's weights
    "adjoint_no_jacobian": ("wt[g] * 0.5 * (z1[pc] - z0[pc]) * ip.detJ;\n                for (int lt",
                            "wt[g] * 0.5 * (z1[pc] - z0[pc]) * 1.0;\n                for (int lt"),
    # a piece's contribution credited to the ply below
    "adjoint_wrong_ply": ("double* o = out + 36 * ply[pc];", "double* o = out + 36 * (ply[pc] > 0 ? ply[pc] - 1 : 1);"),
}


def adjoint_battery():
    failed = []
    lam = BOXES["bspline_p2_three_plies"]()
    rp, col, g = random_cotangent(lam, 3)
    ref = X.exact_box_dL_dD(lam, 2.0, 1.5, dense(rp, col, g, lam.n_dof))
    if not rel(O.adjoint_D(lam, rp, col, g), ref) <= 1e-12:
        failed.append("exact_box")
    lam = W.laminate("m2", W.BSPLINE, 1, 1, [0, 35, -60], 0.05, mapping=W.curved_map(0.04),
                     materials=np.array([W.ply_C21(), W.random_C21(np.random.default_rng(8))]), ply_material=[0, 1, 0])
    rp, col, g = random_cotangent(lam, 6)
    dC, dth, _ = O.adjoint(lam, rp, col, g)
    base_C, base_t = lam.C21.copy(), lam.ply_angle.copy()
    for (m, k) in ((0, 0), (1, 4), (1, 20), (0, 15)):
        h = 1e-3 * max(abs(base_C[m, k]), 1.0)
        lam.C21 = base_C.copy(); lam.C21[m, k] += h
        Lp = L_of(lam, g)
        lam.C21 = base_C.copy(); lam.C21[m, k] -= h
        Lm = L_of(lam, g)
        if abs((Lp - Lm) / (2 * h) - dC[m, k]) > 1e-8 * np.abs(dC).max():
            failed.append("dC_fd")
            break
    lam.C21 = base_C
    for l in range(3):
        h = 1e-5
        lam.ply_angle = base_t.copy(); lam.ply_angle[l] += h
        Lp = L_of(lam, g)
        lam.ply_angle = base_t.copy(); lam.ply_angle[l] -= h
        Lm = L_of(lam, g)
        if abs((Lp - Lm) / (2 * h) - dth[l]) > 1e-7 * np.abs(dth).max():
            failed.append("dtheta_fd")
            break
    lam.ply_angle = base_t
    return failed


def test_unmodified_oracle_passes_the_adjoint_battery():
    assert adjoint_battery() == []


@pytest.mark.parametrize("name", sorted(ADJOINT_MUTATIONS))
def test_planted_adjoint_mistake_is_caught(tmp_path, monkeypatch, name):
    from tests.test_oracle_mutations import build_variant
    old, new = ADJOINT_MUTATIONS[name]
    monkeypatch.setattr(O, "_lib", build_variant(tmp_path, name, old, new))
    try:
        failed = adjoint_battery()
    except Exception as exc:
        failed = [f"exception: {exc!r}"]
    assert failed, f"planted mistake {name} passed every pin"
