"""Pins of the oracle's in-plane operators P (Eq. P, one in-plane pair).

On affine boxes every block is a sum of D entries times exact 1D integrals
(Fractions, no quadrature); on a curved NURBS plate the operators must rebuild
the 3D block of Eq. Km_0 through Eq. Km_2 with exactly integrated thickness
factors. Planted mistakes in a copy of the oracle must fail a pin.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests import exact_rational as X

EXACT_C = X.exact_orthotropic_C21(**W.PLY_CONSTANTS)
V = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]


def exact_box_P(lam, Lx, Ly, angle_deg, i_s, j_s):
    """Eq. P on the box [0, Lx] x [0, Ly] from exact 1D integrals."""
    Ix, Iy = X.gram_1d(lam.u), X.gram_1d(lam.v)
    D = X.exact_rotated_D(EXACT_C, angle_deg)
    nx = lam.u.n_functions
    iy, ix = divmod(i_s, nx)
    jy, jx = divmod(j_s, nx)
    from fractions import Fraction
    Lx, Ly = Fraction(Lx), Fraction(Ly)

    def inplane(a, b):
        # int (d_a S^i)(d_b S^j) dx dy with a, b in {0: d/dx, 1: d/dy, 2: value}
        rx, sx = int(a == 0), int(b == 0)
        ry, sy = int(a == 1), int(b == 1)
        fx = Ix[(rx, sx)].get((ix, jx), 0) * Lx / Lx ** (rx + sx)
        fy = Iy[(ry, sy)].get((iy, jy), 0) * Ly / Ly ** (ry + sy)
        return float(fx * fy)

    P = np.zeros((4, 3, 3))
    groups = {0: ([0, 1], [0, 1]), 1: ([0, 1], [2]), 2: ([2], [0, 1]), 3: ([2], [2])}
    for blk, (As, Bs) in groups.items():
        for a in As:
            for b in Bs:
                f = inplane(a, b)
                for c in range(3):
                    for d in range(3):
                        P[blk, c, d] += D[V[c][a], V[d][b]] * f
    return P


@pytest.mark.parametrize("degree,angle", [(1, 0), (2, 45), (3, 90)])
def test_inplane_P_exact_on_boxes(degree, angle):
    lam = W.laminate("box", W.BSPLINE, degree, 3, [angle], 0.2, mapping=W.scaled_map(2.0, 1.5), n_el_y=2)
    rng = np.random.default_rng(degree)
    ns = lam.n_s
    nx = lam.u.n_functions
    pairs = [(0, 0), (ns - 1, ns - 1)]
    for _ in range(12):
        i = int(rng.integers(ns))
        iy, ix = divmod(i, nx)
        jx = int(np.clip(ix + rng.integers(-degree, degree + 1), 0, nx - 1))
        jy = int(np.clip(iy + rng.integers(-degree, degree + 1), 0, lam.v.n_functions - 1))
        pairs.append((i, jy * nx + jx))
    prob = O.Problem(lam)
    for i, j in pairs:
        got = O.inplane_P(lam, 0, i, j, prob)
        ref = exact_box_P(lam, 2.0, 1.5, angle, i, j)
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(got - ref).max() <= 1e-12 * scale, (i, j)


def test_split_rebuilds_the_3d_block_on_a_curved_nurbs_plate():
    """K^{ij} = sum_l sum_ab P_{l,ab}^{i_s j_s} Q_{l,ab}^{i_t j_t} (Eq. Km_2), Q
    integrated exactly from the thickness basis polynomials."""
    from fractions import Fraction
    lam = W.curved_plate(n_el=2, degree=2, repeats=1)
    lam.weights = np.random.default_rng(3).uniform(0.6, 1.8, lam.n_s)
    z = [Fraction(0)]
    for h in lam.ply_thickness:
        z.append(z[-1] + Fraction(float(h)))
    Iz = [X.gram_1d(lam.t, z[l], z[l + 1]) for l in range(len(lam.ply_thickness))]
    prob = O.Problem(lam)
    ns = lam.n_s
    rng = np.random.default_rng(8)
    rp, col = O.pattern(lam)
    for _ in range(15):
        r = int(rng.integers(lam.n_dof))
        k = int(rng.integers(rp[r], rp[r + 1]))
        i, j = r // 3, int(col[k]) // 3
        it, i_s = divmod(i, ns)
        jt, j_s = divmod(j, ns)
        K = np.zeros((3, 3))
        for l in range(len(lam.ply_thickness)):
            P = O.inplane_P(lam, l, i_s, j_s, prob)
            for blk, (rz, sz) in enumerate(((0, 0), (0, 1), (1, 0), (1, 1))):
                K += P[blk] * float(Iz[l][(rz, sz)].get((it, jt), 0))
        ref = O.block(lam, i, j, prob)
        assert np.abs(K - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-30)


MUTATIONS = {
    "P12_operands_swapped": ("add_btdb(w, Bi1, D, Bj2, out36 + 9);", "add_btdb(w, Bi2, D, Bj1, out36 + 9);"),
    "P_without_jacobian": ("double w = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va) * ip.detJ;\n          double gi1",
                           "double w = wu[a] * 0.5 * (ub - ua) * wv[b] * 0.5 * (vb - va);\n          double gi1"),
    "P_value_part_uses_derivative": ("grad3(&ip, li, 0.0, 1.0, gi2);", "grad3(&ip, li, 1.0, 0.0, gi2);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_in_P_is_caught(tmp_path, monkeypatch, name):
    from tests.test_oracle_mutations import build_variant
    old, new = MUTATIONS[name]
    monkeypatch.setattr(O, "_lib", build_variant(tmp_path, name, old, new))
    failed = False
    try:
        test_inplane_P_exact_on_boxes(2, 45)
    except AssertionError:
        failed = True
    assert failed, f"planted mistake {name} passed the pin"
