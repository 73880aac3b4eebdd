"""Pins of the oracle's general extrusion map (Eq. extrusion: F = S(xi1, xi2) +
xi3 a with S a surface in R^3 and a a constant direction) against things other
than itself: exact rational integrals for affine extrusions, the planar map as
a special case, rigid-body modes, rotation equivariance and definiteness.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests import exact_rational as X

# rational rotations (Pythagorean triples): about z by atan(4/3), about x by atan(12/5)
RZ = np.array([[0.6, -0.8, 0.0], [0.8, 0.6, 0.0], [0.0, 0.0, 1.0]])
RX = np.array([[1.0, 0.0, 0.0], [0.0, 5 / 13, -12 / 13], [0.0, 12 / 13, 5 / 13]])
RZ_EXACT = [["3/5", "-4/5", "0"], ["4/5", "3/5", "0"], ["0", "0", "1"]]
RX_EXACT = [["1", "0", "0"], ["0", "5/13", "-12/13"], ["0", "12/13", "5/13"]]


def _dense(lam):
    rp, col, val = O.assemble(lam)
    return O.to_dense(rp, col, val, lam.n_dof), (rp, col, val)


def shell_coords(lam):
    """Control point of the 3D function (i_t, i_s): S_i + z_t a, exact for
    linear fields because both bases are partitions of unity."""
    zt = W.anchors(lam.t)
    S = lam.ctrl if lam.ctrl.shape[1] == 3 else np.c_[lam.ctrl, np.zeros(lam.n_s)]
    a = np.array([0.0, 0.0, 1.0]) if lam.extrusion is None else lam.extrusion
    P = np.zeros((lam.n_s * lam.n_t, 3))
    for it in range(lam.n_t):
        P[it * lam.n_s:(it + 1) * lam.n_s] = S + zt[it] * a
    return P


def rigid_mode_residual(K, P):
    worst = 0.0
    for k in range(3):
        t = np.zeros(3)
        t[k] = 1.0
        r = np.tile(t, len(P))
        worst = max(worst, np.abs(K @ r).max() / np.abs(r).max())
        w = np.zeros(3)
        w[k] = 1.0
        Wm = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        r = (P @ Wm.T).reshape(-1)
        worst = max(worst, np.abs(K @ r).max() / np.abs(r).max())
    return worst / np.abs(K).max()


def _mat(rows):
    from fractions import Fraction
    return [[Fraction(x) for x in r] for r in rows]


def _matmul_exact(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(3)) for j in range(3)] for i in range(3)]


AFFINE_CASES = {
    # sheared extrusion of the unit square
    "sheared_a": _mat([["1", "0", "1/4"], ["0", "1", "-1/2"], ["0", "0", "1"]]),
    # a rotated, sheared, stretched slab: A = RZ RX [[2, 1/4, 1/8], [0, 1/2, -1/4], [0, 0, 3/2]]
    "rotated_general": _matmul_exact(_matmul_exact(_mat(RZ_EXACT), _mat(RX_EXACT)),
                                     _mat([["2", "1/4", "1/8"], ["0", "1/2", "-1/4"], ["0", "0", "3/2"]])),
}


def affine_laminate(A, degree=2, n_el=2, angles=(45.0, 0.0, 90.0), h=(0.3, 0.2, 0.2), n_el_y=1):
    Af = np.array([[float(x) for x in r] for r in A])
    return W.laminate("affine_shell", W.BSPLINE, degree, n_el, list(angles), list(h),
                      mapping=W.affine_surface_map(Af), extrusion=Af[:, 2], n_el_y=n_el_y)


EXACT_C = X.exact_orthotropic_C21(**W.PLY_CONSTANTS)


@pytest.mark.parametrize("case", sorted(AFFINE_CASES))
def test_exact_affine_extrusion(case):
    A = AFFINE_CASES[case]
    lam = affine_laminate(A)
    assert lam.ctrl.shape[1] == 3
    rp, col, val = O.assemble(lam)
    blocks = sorted({(r // 3, col[k] // 3) for r in range(0, lam.n_dof, 5) for k in range(rp[r], rp[r + 1], 3)})
    ex = X.exact_affine_blocks(lam, A, [EXACT_C], [45, 0, 90], blocks)
    err = 0.0
    for r in range(0, lam.n_dof, 5):
        for k in range(rp[r], rp[r + 1], 3):
            err = max(err, abs(val[k] - ex[(r // 3, col[k] // 3)][r % 3, col[k] % 3]))
    assert err <= 1e-12 * np.abs(val).max()


def test_exact_affine_reduces_to_the_box():
    """The affine checker itself: A = diag(Lx, Ly, 1) gives the box checker."""
    lam = W.laminate("b", W.BSPLINE, 2, 1, [45.0, 0.0, 90.0], [0.3, 0.2, 0.2], mapping=W.scaled_map(1.0, 2.0))
    blocks = [(0, 0), (0, 5), (3, 17), (20, 11)]
    a = X.exact_affine_blocks(lam, _mat([["1", "0", "0"], ["0", "2", "0"], ["0", "0", "1"]]), [EXACT_C],
                              [45, 0, 90], blocks)
    b = X.exact_box_blocks(lam, 1.0, 2.0, [EXACT_C], [45, 0, 90], blocks)
    for k in blocks:
        assert np.abs(a[k] - b[k]).max() <= 1e-15 * max(np.abs(b[k]).max(), 1.0)


@pytest.mark.parametrize("weighted", [False, True])
def test_planar_embedding_is_the_planar_map(weighted):
    lam = W.curved_plate(n_el=3, degree=2, repeats=1)
    if weighted:
        lam.weights = np.random.default_rng(5).uniform(0.5, 2.0, lam.n_s)
    K2, _ = _dense(lam)
    lam.ctrl = np.c_[lam.ctrl, np.zeros(lam.n_s)]
    lam.extrusion = np.array([0.0, 0.0, 1.0])
    K3, _ = _dense(lam)
    assert np.abs(K3 - K2).max() <= 1e-14 * np.abs(K2).max()


SHELLS = [
    lambda: W.shell_plate(n_el=3, degree=2, repeats=1),
    lambda: W.shell_plate(n_el=2, degree=3, repeats=1, extrusion=(0.3, 0.2, 0.9)),
    lambda: W.laminate("shell_lag", W.LAGRANGE, 2, 3, [0, 45, 90], 0.01, mapping=W.bump_map(0.1),
                       thickness_kind=W.LAGRANGE, extrusion=(-0.1, 0.05, 1.0)),
]


@pytest.mark.parametrize("make", SHELLS)
def test_curved_shell_symmetry_and_rigid_modes(make):
    lam = make()
    K, _ = _dense(lam)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    assert rigid_mode_residual(K, shell_coords(lam)) <= 1e-12


def test_nurbs_shell_rigid_modes():
    lam = W.shell_plate(n_el=3, degree=2, repeats=1)
    lam.weights = np.random.default_rng(7).uniform(0.5, 2.0, lam.n_s)
    K, _ = _dense(lam)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    assert rigid_mode_residual(K, shell_coords(lam)) <= 1e-12


def test_shell_psd_with_six_rigid_modes():
    lam = W.shell_plate(n_el=2, degree=2, repeats=1, extrusion=(0.2, -0.1, 1.0))
    lam.ply_thickness = np.full(len(lam.ply_thickness), 0.05)
    lam.t = W.thickness_basis(lam.ply_thickness)
    K, _ = _dense(lam)
    ev = np.linalg.eigvalsh(K)
    assert np.all(np.abs(ev[:6]) < 1e-12 * ev[-1])
    assert ev[6] > 1e-9 * ev[-1]


def _rotated(lam, Q):
    import dataclasses
    a = np.array([0.0, 0.0, 1.0]) if lam.extrusion is None else lam.extrusion
    S = lam.ctrl if lam.ctrl.shape[1] == 3 else np.c_[lam.ctrl, np.zeros(lam.n_s)]
    return dataclasses.replace(lam, ctrl=S @ Q.T, extrusion=Q @ a)


def test_rotation_equivariance_isotropic():
    """Rotating the solid (S -> Q S, a -> Q a) with an isotropic material gives
    K' = T K T^T, T = I (x) Q on the displacement components."""
    lam = W.shell_plate(n_el=2, degree=2, repeats=1)
    lam.C21 = W.isotropic_C21(70.0, 0.3)[None, :]
    K, _ = _dense(lam)
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((3, 3)))
    Q = Q * np.sign(np.linalg.det(Q))
    Kr, _ = _dense(_rotated(lam, Q))
    T = np.kron(np.eye(lam.n_dof // 3), Q)
    assert np.abs(Kr - T @ K @ T.T).max() <= 1e-12 * np.abs(K).max()


def test_rotation_about_z_turns_the_plies_too():
    """A rotation about z by phi of the geometry together with ply angles
    theta + phi is a rigid rotation of the whole anisotropic solid."""
    lam = W.shell_plate(n_el=2, degree=2, repeats=1)
    K, _ = _dense(lam)
    phi = 0.7
    Q = np.array([[math.cos(phi), -math.sin(phi), 0.0], [math.sin(phi), math.cos(phi), 0.0], [0.0, 0.0, 1.0]])
    lr = _rotated(lam, Q)
    lr.ply_angle = lam.ply_angle + phi
    Kr, _ = _dense(lr)
    T = np.kron(np.eye(lam.n_dof // 3), Q)
    assert np.abs(Kr - T @ K @ T.T).max() <= 1e-12 * np.abs(K).max()
    lr.ply_angle = lam.ply_angle  # plies left behind: a different solid
    Kw, _ = _dense(lr)
    assert np.abs(Kw - T @ K @ T.T).max() > 1e-6 * np.abs(K).max()


def test_split_formula_equals_standard_on_a_shell():
    """Assumption 1 holds for every extrusion, so Eq. Km_2 reaches Eq. Km_0."""
    lam = W.shell_plate(n_el=2, degree=2, repeats=1, extrusion=(0.2, -0.1, 1.0))
    a = O.assemble(lam)[2]
    b = O.assemble_split(lam)[2]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


# ------------------------------------------------------------------ adjoint of a general extrusion
def _cotangent(lam, seed):
    rp, col, _ = O.assemble(lam)
    return rp, col, np.random.default_rng(seed).standard_normal(len(col))


def _L(lam, g):
    return float(g @ O.assemble(lam)[2])


def _shell_two_materials():
    rng = np.random.default_rng(8)
    return W.laminate("sh2", W.BSPLINE, 2, 2, [0, 35, -60, 90], 0.05, mapping=W.bump_map(0.1),
                      materials=np.array([W.ply_C21(), W.random_C21(rng)]), ply_material=[0, 1, 1, 0],
                      extrusion=(0.2, -0.1, 1.0))


def test_shell_adjoint_euler_identity():
    """K is homogeneous of degree one in the D_l: sum_l <dL/dD_l, D_l> = L."""
    lam = W.shell_plate(n_el=2, degree=2, repeats=1, extrusion=(0.3, 0.2, 0.9))
    lam.weights = np.random.default_rng(2).uniform(0.6, 1.7, lam.n_s)
    rp, col, g = _cotangent(lam, 5)
    dD = O.adjoint_D(lam, rp, col, g)
    Ds = [O.rotated_D(lam.C21[lam.ply_material[l]], lam.ply_angle[l]) for l in range(len(lam.ply_angle))]
    lhs = sum(float(np.sum(dD[l] * Ds[l])) for l in range(len(Ds)))
    assert abs(lhs - _L(lam, g)) <= 1e-12 * np.abs(g).sum() * np.abs(O.assemble(lam)[2]).max()


def test_shell_adjoint_matches_finite_differences():
    """dL/dC by central differences (exact up to rounding: L is linear in C) and
    dL/dtheta by central differences, on a shell with two materials."""
    lam = _shell_two_materials()
    rp, col, g = _cotangent(lam, 6)
    dC, dth, _ = O.adjoint(lam, rp, col, g)
    base = lam.C21.copy()
    fd = np.zeros_like(dC)
    for m in range(base.shape[0]):
        for k in range(21):
            h = 1e-3 * max(abs(base[m, k]), 1.0)
            lam.C21 = base.copy(); lam.C21[m, k] += h
            Lp = _L(lam, g)
            lam.C21 = base.copy(); lam.C21[m, k] -= h
            Lm = _L(lam, g)
            fd[m, k] = (Lp - Lm) / (2 * h)
    lam.C21 = base
    assert np.abs(dC - fd).max() <= 1e-8 * np.abs(fd).max()
    ang = lam.ply_angle.copy()
    fdt = np.zeros_like(dth)
    for l in range(len(ang)):
        lam.ply_angle = ang.copy(); lam.ply_angle[l] += 1e-5
        Lp = _L(lam, g)
        lam.ply_angle = ang.copy(); lam.ply_angle[l] -= 1e-5
        Lm = _L(lam, g)
        fdt[l] = (Lp - Lm) / 2e-5
    lam.ply_angle = ang
    assert np.abs(dth - fdt).max() <= 1e-7 * np.abs(fdt).max()
