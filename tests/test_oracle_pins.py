"""Pins of the CPU oracle against things other than itself.

Each test ties one part of the oracle to a library routine, a closed form, an
exact rational computation or an invariant of linear elasticity, chosen so that
a dropped term, a wrong sign or index, or a transposed operand fails one of
them. No GPU is needed.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle as O
import workloads as W
from tests import exact_rational as X


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------------ quadrature
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 10])
def test_gauss_matches_numpy_and_is_exact(n):
    x, w = O.gauss(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=1e-15, rtol=0) and np.allclose(w, wr, atol=1e-15, rtol=0)
    for k in range(2 * n):  # exact up to degree 2n-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


# ------------------------------------------------------------------ bases
KNOTS = [
    (2, W.open_uniform_knots(2, 5)),
    (3, W.open_uniform_knots(3, 4)),
    (3, np.array([0, 0, 0, 0, 0.2, 0.2, 0.5, 0.7, 1, 1, 1, 1.0])),  # repeated interior knot
    (2, np.array([0, 0, 0, 0.1, 0.1, 0.4, 0.4, 1.0, 1, 1])),         # C0 quadratic (Bernstein pieces)
    (4, W.open_uniform_knots(4, 3, 0.0, 2.0)),
]


@pytest.mark.parametrize("p,knots", KNOTS)
def test_bspline_matches_scipy(p, knots):
    n = len(knots) - p - 1
    nel = O.n_elements(0, p, knots)
    assert nel == len(np.unique(knots)) - 1
    for e in range(nel):
        for xg in np.linspace(0.05, 0.95, 4):
            # element bounds: e-th nonempty span
            spans = [s for s in range(p, len(knots) - p - 1) if knots[s] < knots[s + 1]]
            a, b = knots[spans[e]], knots[spans[e] + 1]
            x = a + (b - a) * xg
            first, val, der = O.basis1d_eval(0, p, knots, e, x)
            assert first == spans[e] - p
            for k in range(p + 1):
                c = np.zeros(n)
                c[first + k] = 1.0
                spl = BSpline(knots, c, p)
                assert abs(val[k] - spl(x)) < 1e-14
                assert abs(der[k] - spl.derivative()(x)) < 1e-12 * max(1.0, abs(der).max())
            assert abs(val.sum() - 1.0) < 1e-14 and abs(der.sum()) < 1e-12 * abs(der).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_interpolates_and_reproduces_polynomials(p):
    bp = np.array([0.0, 0.3, 1.0])
    for e in range(2):
        a, b = bp[e], bp[e + 1]
        nodes = a + (b - a) * np.arange(p + 1) / p
        for k, xn in enumerate(nodes):  # Kronecker property at the nodes
            first, val, _ = O.basis1d_eval(1, p, bp, e, xn)
            assert first == p * e
            assert np.allclose(val, np.eye(p + 1)[k], atol=1e-13)
        rng = np.random.default_rng(p)
        coef = rng.standard_normal(p + 1)
        poly = np.polynomial.Polynomial(coef)
        for x in np.linspace(a, b, 7)[1:-1]:
            _, val, der = O.basis1d_eval(1, p, bp, e, x)
            assert abs(val @ poly(nodes) - poly(x)) < 1e-12
            assert abs(der @ poly(nodes) - poly.deriv()(x)) < 1e-10


# ------------------------------------------------------------------ material
def test_rotation_invariants():
    C = W.ply_C21()
    Cm = np.zeros((6, 6))
    k = 0
    for I in range(6):
        for J in range(I, 6):
            Cm[I, J] = Cm[J, I] = C[k]
            k += 1
    assert rel(O.rotated_D(C, 0.0), Cm) < 1e-15
    for th in (0.3, 1.1, -0.7):
        assert rel(O.rotated_D(C, th + math.pi), O.rotated_D(C, th)) < 1e-14
    # 90 degrees swaps the in-plane axes: 11<->22 and 13<->23
    D90 = O.rotated_D(C, math.pi / 2)
    perm = [1, 0, 2, 3, 5, 4]
    assert rel(D90, Cm[np.ix_(perm, perm)]) < 1e-14
    # an isotropic material does not see the angle
    Ci = W.isotropic_C21(70.0, 0.33)
    assert rel(O.rotated_D(Ci, 0.77), O.rotated_D(Ci, 0.0)) < 1e-14


def test_rotation_preserves_strain_energy():
    """eps_g^T D(theta) eps_g equals eps_m^T C eps_m, with the material-frame
    strain eps_m = R^T eps_g R obtained by rotating the 3x3 strain tensor."""
    rng = np.random.default_rng(3)
    C = W.random_C21(rng)
    Cm = np.zeros((6, 6))
    k = 0
    for I in range(6):
        for J in range(I, 6):
            Cm[I, J] = Cm[J, I] = C[k]
            k += 1

    def to_voigt(E):  # engineering shears
        return np.array([E[0, 0], E[1, 1], E[2, 2], 2 * E[0, 1], 2 * E[0, 2], 2 * E[1, 2]])

    for th in (0.0, 0.4, 2.0, -1.3):
        D = O.rotated_D(C, th)
        c, s = math.cos(th), math.sin(th)
        R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        for _ in range(5):
            A = rng.standard_normal((3, 3))
            Eg = 0.5 * (A + A.T)
            Em = R.T @ Eg @ R
            eg, em = to_voigt(Eg), to_voigt(Em)
            assert abs(eg @ D @ eg - em @ Cm @ em) < 1e-12 * abs(em @ Cm @ em)
            # stress transforms as a tensor too: sigma_g = R sigma_m R^T
            sm = Cm @ em
            Sm = np.array([[sm[0], sm[3], sm[4]], [sm[3], sm[1], sm[5]], [sm[4], sm[5], sm[2]]])
            Sg = R @ Sm @ R.T
            sg = D @ eg
            assert rel([sg[0], sg[1], sg[2], sg[3], sg[4], sg[5]],
                       [Sg[0, 0], Sg[1, 1], Sg[2, 2], Sg[0, 1], Sg[0, 2], Sg[1, 2]]) < 1e-12


# ------------------------------------------------------------------ exact rational boxes
EXACT_C = X.exact_orthotropic_C21(**W.PLY_CONSTANTS)


def _exact_check(lam, Lx, Ly, angles, n_samples=None, seed=0):
    rp, col, val = O.assemble(lam)
    n = lam.n_dof
    entries = []
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            entries.append((r, k))
    if n_samples is not None and n_samples < len(entries):
        rng = np.random.default_rng(seed)
        entries = [entries[k] for k in rng.choice(len(entries), n_samples, replace=False)]
    blocks = sorted({(r // 3, col[k] // 3) for r, k in entries})
    ex = X.exact_box_blocks(lam, Lx, Ly, [EXACT_C] * lam.C21.shape[0], angles, blocks)
    scale = np.abs(val).max()
    err = 0.0
    for r, k in entries:
        e = ex[(r // 3, col[k] // 3)][r % 3, col[k] % 3]
        err = max(err, abs(val[k] - e))
    assert err <= 1e-13 * scale, err / scale


def test_exact_single_brick_q1():
    lam = W.laminate("brick", W.BSPLINE, 1, 1, [30.0 * 0], 0.5, mapping=W.scaled_map(2.0, 1.5),
                     thickness_degree=1)
    _exact_check(lam, 2.0, 1.5, [0])


def test_exact_single_brick_q2_rotated():
    lam = W.laminate("brick2", W.BSPLINE, 2, 1, [45.0], 0.7, mapping=W.scaled_map(1.0, 3.0))
    _exact_check(lam, 1.0, 3.0, [45])


def test_exact_cross_ply_plate_sampled():
    lam = W.cross_ply_plate()
    _exact_check(lam, 1.0, 1.0, [0, 90, 0, 90], n_samples=4000)


def test_exact_quasi_isotropic_stack_lagrange_thickness():
    angles = [0, 45, -45, 90, 90, -45]
    lam = W.laminate("qi", W.BSPLINE, 2, 3, angles, [0.1, 0.2, 0.1, 0.15, 0.1, 0.05],
                     mapping=W.scaled_map(1.5, 1.0), thickness_kind=W.LAGRANGE, n_el_y=2, degree_y=3)
    _exact_check(lam, 1.5, 1.0, angles)


def test_exact_one_element_through_thickness():
    """The paper's own discretisation: one element of degree p through the
    whole thickness, so plies cut the thickness element into pieces."""
    angles = [0, 90, 0, 90, 0]
    h = [0.1, 0.1, 0.2, 0.1, 0.1]
    t = W.single_element_thickness(sum(h), 3)
    lam = W.laminate("solid_shell", W.BSPLINE, 3, 2, angles, h, thickness=t)
    _exact_check(lam, 1.0, 1.0, angles)


def test_exact_lagrange_inplane():
    lam = W.laminate("lag", W.LAGRANGE, 2, 2, [0, 90], 0.25, mapping=W.scaled_map(1.0, 2.0),
                     thickness_kind=W.LAGRANGE)
    _exact_check(lam, 1.0, 2.0, [0, 90])


# ------------------------------------------------------------------ invariants on curved maps
def _dense(lam):
    rp, col, val = O.assemble(lam)
    return O.to_dense(rp, col, val, lam.n_dof), (rp, col, val)


def _coords(lam):
    """Physical coordinates attached to each basis function: control points
    in-plane and Greville/nodal z (exact for linear fields)."""
    zt = W.anchors(lam.t)
    xy = lam.ctrl
    ns = lam.n_s
    P = np.zeros((lam.n_s * lam.n_t, 3))
    for it in range(lam.n_t):
        P[it * ns:(it + 1) * ns, :2] = xy
        P[it * ns:(it + 1) * ns, 2] = zt[it]
    return P


def _linear_field(P, A, b):
    U = P @ A.T + b
    return U.reshape(-1)


CURVED_SMALL = [
    lambda: W.curved_plate(n_el=3, degree=3, repeats=1),
    lambda: W.curved_plate(n_el=4, degree=2, repeats=1),
    lambda: W.laminate("curved_lag", W.LAGRANGE, 2, 3, [0, 45, 90], 0.01, mapping=W.curved_map(0.05),
                       thickness_kind=W.LAGRANGE),
]


@pytest.mark.parametrize("make", CURVED_SMALL)
def test_curved_symmetry_rigid_modes_and_patch(make):
    lam = make()
    K, _ = _dense(lam)
    scale = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-14 * scale
    P = _coords(lam)
    rng = np.random.default_rng(11)
    # rigid-body modes: translations and infinitesimal rotations
    for k in range(3):
        t = np.zeros(3)
        t[k] = 1.0
        r = _linear_field(P, np.zeros((3, 3)), t)
        assert np.abs(K @ r).max() <= 1e-12 * scale * np.abs(r).max()
    for k in range(3):
        w = np.zeros(3)
        w[k] = 1.0
        Wm = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        r = _linear_field(P, Wm, np.zeros(3))
        assert np.abs(K @ r).max() <= 1e-12 * scale * np.abs(r).max()
    # patch test: a linear field with constant strain in a homogeneous body
    # leaves zero residual at functions that vanish on the boundary
    lam_h = lam
    lam_h.ply_angle = np.zeros_like(lam.ply_angle)
    Kh, _ = _dense(lam_h)
    A = rng.standard_normal((3, 3))
    u = _linear_field(P, A, rng.standard_normal(3))
    res = (Kh @ u).reshape(-1, 3)
    nx, ny, nt = lam.u.n_functions, lam.v.n_functions, lam.n_t
    interior = []
    for it in range(1, nt - 1):
        for iy in range(1, ny - 1):
            for ix in range(1, nx - 1):
                interior.append(it * nx * ny + iy * nx + ix)
    assert len(interior) > 0
    assert np.abs(res[interior]).max() <= 1e-11 * np.abs(Kh).max() * np.abs(u).max()
    # ... and a nonzero residual somewhere on the boundary (the field is not trivial)
    assert np.abs(res).max() > 1e-6 * np.abs(Kh).max() * np.abs(u).max()


def test_cross_ply_psd_with_six_rigid_modes():
    lam = W.cross_ply_plate()
    K, _ = _dense(lam)
    ev = np.linalg.eigvalsh(K)
    scale = ev[-1]
    # six rigid-body modes at rounding level (~1e-17 relative), the softest
    # flexible mode of this thin plate near 5e-10 relative
    assert ev[0] > -1e-14 * scale
    assert np.all(np.abs(ev[:6]) < 1e-14 * scale)
    assert ev[6] > 1e-11 * scale


def test_nurbs_equal_weights_is_bspline_and_rigid_modes():
    lam = W.curved_plate(n_el=3, degree=2, repeats=1)
    K0, _ = _dense(lam)
    lam.weights = np.full(lam.n_s, 2.5)
    K1, _ = _dense(lam)
    assert rel(K1, K0) < 1e-13
    rng = np.random.default_rng(5)
    lam.weights = rng.uniform(0.5, 2.0, lam.n_s)
    K2, _ = _dense(lam)
    assert rel(K2, K0) > 1e-6           # weights matter
    assert np.abs(K2 - K2.T).max() <= 1e-14 * np.abs(K2).max()
    P = _coords(lam)
    for k in range(3):
        t = np.zeros(3)
        t[k] = 1.0
        assert np.abs(K2 @ _linear_field(P, np.zeros((3, 3)), t)).max() <= 1e-12 * np.abs(K2).max()
    Wm = np.array([[0, -1.0, 0], [1.0, 0, 0], [0, 0, 0]])
    r = _linear_field(P, Wm, np.zeros(3))
    assert np.abs(K2 @ r).max() <= 1e-12 * np.abs(K2).max() * np.abs(r).max()


# ------------------------------------------------------------------ stack invariances
def test_stack_invariances():
    base = W.curved_plate(n_el=2, degree=2, repeats=1)
    K, _ = _dense(base)
    # theta + pi on every ply
    b2 = W.curved_plate(n_el=2, degree=2, repeats=1)
    b2.ply_angle = b2.ply_angle + math.pi
    K2, _ = _dense(b2)
    assert rel(K2, K) < 1e-13
    # isotropic material: independent of all angles
    iso = W.isotropic_C21(50.0, 0.25)
    b3 = W.curved_plate(n_el=2, degree=2, repeats=1)
    b3.C21 = iso[None, :]
    K3, _ = _dense(b3)
    b3.ply_angle = np.zeros_like(b3.ply_angle)
    K4, _ = _dense(b3)
    assert rel(K3, K4) < 1e-13
    # one configuration in every ply == the homogeneous solid with one ply
    angles = [30.0] * 4
    lam = W.laminate("same", W.BSPLINE, 2, 2, angles, 0.25, mapping=W.curved_map(), n_el_y=3)
    Ka, _ = _dense(lam)
    one = W.laminate("one", W.BSPLINE, 2, 2, [30.0], 1.0, mapping=W.curved_map(), n_el_y=3,
                     thickness=lam.t)
    Kb, _ = _dense(one)
    assert rel(Ka, Kb) < 1e-13


def test_more_gauss_points_change_nothing_on_affine_maps():
    lam = W.laminate("b", W.BSPLINE, 2, 1, [0, 45], 0.5, mapping=W.scaled_map(2.0, 1.0))
    K1, _ = _dense(lam)
    lam.nq = (10, 10, 10)
    K2, _ = _dense(lam)
    assert rel(K2, K1) < 1e-13


# ------------------------------------------------------------------ split formula and blocks
@pytest.mark.parametrize("make", [W.cross_ply_plate, CURVED_SMALL[0], CURVED_SMALL[2]])
def test_split_formula_equals_standard(make):
    """Eq. Km_2 and Eq. Km_0 give the same matrix up to rounding."""
    lam = make()
    a = O.assemble(lam)
    b = O.assemble_split(lam)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert rel(b[2], a[2]) < 1e-13


def test_block_oracle_matches_assembly():
    lam = CURVED_SMALL[0]()
    rp, col, val = O.assemble(lam)
    rng = np.random.default_rng(2)
    prob = O.Problem(lam)
    for r in rng.choice(lam.n_dof, 40, replace=False):
        ks = rng.choice(np.arange(rp[r], rp[r + 1]), 3)
        for k in ks:
            B = O.block(lam, r // 3, col[k] // 3, prob)
            assert abs(B[r % 3, col[k] % 3] - val[k]) <= 1e-14 * np.abs(val).max()


def test_pattern_matches_kronecker_count():
    """nnz = 9 * (in-plane neighbour pairs) * (thickness neighbour pairs),
    with 1D neighbour ranges found by brute force over element supports."""
    def pairs_1d(b):
        n = b.n_functions
        nel = O.n_elements(b.kind, b.degree, b.knots)
        funcs = []
        for e in range(nel):
            first, _, _ = O.basis1d_eval(b.kind, b.degree, b.knots, e, 0.5 * sum(_elem(b, e)))
            funcs.append(set(range(first, first + b.degree + 1)))
        S = np.zeros((n, n), bool)
        for f in funcs:
            for i in f:
                for j in f:
                    S[i, j] = True
        return S.sum()

    for lam in (W.cross_ply_plate(), W.curved_plate(n_el=5, degree=3, repeats=1),
                W.lagrange_plate(n_el=3, n_plies=3)):
        n_dof, nnz = O.sizes(lam)
        assert nnz == 9 * pairs_1d(lam.u) * pairs_1d(lam.v) * pairs_1d(lam.t)
        assert n_dof == lam.n_dof


def _elem(b, e):
    if b.kind == 1:
        return b.knots[e], b.knots[e + 1]
    spans = [s for s in range(b.degree, len(b.knots) - b.degree - 1) if b.knots[s] < b.knots[s + 1]]
    return b.knots[spans[e]], b.knots[spans[e] + 1]


def test_config_sizes_match_published_counts():
    """DOF and nnz of the cross-ply plate (2700 DOFs, 574,992 nonzeros)."""
    lam = W.cross_ply_plate()
    assert O.sizes(lam) == (2700, 574992)


# ---------------------------------------------------------------- helpers of the timed baseline and the row checks
def test_element_colour_lists_on_threads_equal_the_assembly():
    """ora_assemble_elements over every element colour, each colour split over
    four threads, reproduces ora_assemble; the colours cover every element once."""
    from concurrent.futures import ThreadPoolExecutor
    lam = W.curved_plate(n_el=4, degree=3, repeats=1)
    rp, col, ref = O.assemble(lam)
    groups = O.element_colours(lam)
    seen = np.concatenate(groups)
    assert len(seen) == len(np.unique(seen, axis=0)) == 4 * 4 * 8
    val = np.zeros_like(ref)
    prob = O.Problem(lam)
    with ThreadPoolExecutor(4) as ex:
        for g in groups:
            list(ex.map(lambda c: O.assemble_elements(lam, rp, col, c, val, prob), np.array_split(g, 4)))
    assert np.abs(val - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("make", [lambda: W.curved_plate(n_el=4, degree=3, repeats=1),
                                  lambda: W.lagrange_plate(n_el=3, n_plies=4),
                                  lambda: W.shell_plate(n_el=3, degree=2, repeats=1)])
def test_inplane_row_blocks_equal_the_assembled_rows(make):
    """ora_inplane_row_blocks gives every stored entry of the rows (i_t, i_s, c)
    of ora_assemble, and zero for every block the pattern does not store."""
    lam = make()
    rp, col, val = O.assemble(lam)
    ns, nt = lam.n_s, lam.n_t
    nx = O.n_functions(lam.u.kind, lam.u.degree, lam.u.knots)
    for i_s in (0, ns // 2, ns - 1):
        bx0, by0, B = O.inplane_row_blocks(lam, i_s)
        for it in range(nt):
            for c in range(3):
                r = 3 * (it * ns + i_s) + c
                for k in range(rp[r], rp[r + 1]):
                    j, d = divmod(int(col[k]), 3)
                    jt, js = divmod(j, ns)
                    jy, jx = divmod(js, nx)
                    assert abs(val[k] - B[it, jt, jy - by0, jx - bx0, c, d]) <= 1e-14 * np.abs(val).max()
                    B[it, jt, jy - by0, jx - bx0, c, d] = 0.0
        assert np.abs(B).max() <= 1e-14 * np.abs(val).max()
