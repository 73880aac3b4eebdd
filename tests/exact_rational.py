"""Exact rational stiffness of an axis-aligned laminated box (test helper).

Independent of the oracle: no quadrature, no strain-displacement matrix. On the
box [0,Lx] x [0,Ly] x [0,H] with the affine map x = Lx xi, y = Ly eta, z = z,
every 3D basis function is a product N_ix(xi) N_iy(eta) T_it(z) of piecewise
polynomials, the elasticity bilinear form (Eq. a, Section 2.1) reads

  K^{ij}_{cd} = sum_plies sum_{a,b} C_l[V(c,a), V(d,b)]
                * Ix_{ab}(ix, jx) * Iy_{ab}(iy, jy) * Iz_{l,ab}(it, jt)

with V the Voigt index of a symmetric index pair, and each factor is an exact
1D integral of a product of (derivatives of) piecewise polynomials, computed
here with Fractions. Rotated ply matrices are computed exactly with sympy for
angles in {0, 90, +-45, 180} degrees, whose rotated monoclinic constants are
rational.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np


# ---------------------------------------------------------------- polynomials
def padd(p, q):
    n = max(len(p), len(q))
    return [(p[k] if k < len(p) else 0) + (q[k] if k < len(q) else 0) for k in range(n)]


def pmul(p, q):
    out = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def pscale(p, s):
    return [a * s for a in p]


def pderiv(p):
    return [k * p[k] for k in range(1, len(p))] or [Fraction(0)]


def pinteg(p, a, b):
    return sum(c * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k, c in enumerate(p))


def bspline_pieces(knots, degree):
    """Per knot span [t_s, t_{s+1}] (nonempty), the polynomials of all
    functions that are nonzero there: {span: (a, b, {i: poly})}."""
    t = [Fraction(k) for k in knots]
    n = len(t) - degree - 1
    out = {}
    for s in range(degree, len(t) - degree - 1):
        if not t[s] < t[s + 1]:
            continue
        # Cox-de Boor on polynomials restricted to span s
        N = {i: ([Fraction(1)] if i == s else [Fraction(0)]) for i in range(len(t) - 1)}
        for p in range(1, degree + 1):
            M = {}
            for i in range(len(t) - p - 1):
                acc = [Fraction(0)]
                d1 = t[i + p] - t[i]
                d2 = t[i + p + 1] - t[i + 1]
                if d1 != 0:
                    acc = padd(acc, pmul([-t[i] / d1, 1 / d1], N[i]))
                if d2 != 0:
                    acc = padd(acc, pmul([t[i + p + 1] / d2, -1 / d2], N[i + 1]))
                M[i] = acc
            N = M
        out[s] = (t[s], t[s + 1], {i: N[i] for i in range(s - degree, s + 1) if 0 <= i < n})
    return out


def lagrange_pieces(breakpoints, degree):
    bp = [Fraction(b) for b in breakpoints]
    out = {}
    for e in range(len(bp) - 1):
        a, b = bp[e], bp[e + 1]
        nodes = [a + (b - a) * k / degree for k in range(degree + 1)]
        polys = {}
        for k in range(degree + 1):
            p = [Fraction(1)]
            for m in range(degree + 1):
                if m != k:
                    p = pmul(p, [-nodes[m] / (nodes[k] - nodes[m]), 1 / (nodes[k] - nodes[m])])
            polys[degree * e + k] = p
        out[e] = (a, b, polys)
    return out


def pieces(basis):
    if basis.kind == 0:
        return bspline_pieces(tuple(basis.knots), basis.degree)
    return lagrange_pieces(tuple(basis.knots), basis.degree)


def gram_1d(basis, lo=None, hi=None):
    """I[r][s][(i, j)] = int_{lo}^{hi} d^r N_i d^s N_j, r, s in {0, 1}."""
    I = {(r, s): {} for r in (0, 1) for s in (0, 1)}
    lo = None if lo is None else Fraction(lo)
    hi = None if hi is None else Fraction(hi)
    for _, (a, b, polys) in pieces(basis).items():
        aa = a if lo is None else max(a, lo)
        bb = b if hi is None else min(b, hi)
        if not aa < bb:
            continue
        for i, pi in polys.items():
            for j, pj in polys.items():
                di, dj = pderiv(pi), pderiv(pj)
                for r, s, u, w in ((0, 0, pi, pj), (0, 1, pi, dj), (1, 0, di, pj), (1, 1, di, dj)):
                    I[(r, s)][(i, j)] = I[(r, s)].get((i, j), Fraction(0)) + pinteg(pmul(u, w), aa, bb)
    return I


# ---------------------------------------------------------------- materials
def voigt(i, j):
    if i == j:
        return i
    return {frozenset((0, 1)): 3, frozenset((0, 2)): 4, frozenset((1, 2)): 5}[frozenset((i, j))]


def exact_rotated_D(C21_exact, angle_deg):
    """Rotated Voigt matrix in exact arithmetic (sympy); returns floats."""
    import sympy as sp
    th = sp.rad(sp.Integer(int(angle_deg)))
    c, s = sp.cos(th), sp.sin(th)
    R = sp.Matrix([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    C = sp.zeros(6, 6)
    k = 0
    for I in range(6):
        for J in range(I, 6):
            C[I, J] = C[J, I] = sp.Rational(C21_exact[k])
            k += 1
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    D = np.zeros((6, 6))
    for I, (i, j) in enumerate(pairs):
        for J, (kk, l) in enumerate(pairs):
            acc = 0
            for p in range(3):
                for q in range(3):
                    for r in range(3):
                        for t in range(3):
                            f = R[i, p] * R[j, q] * R[kk, r] * R[l, t]
                            if f != 0:
                                acc += f * C[voigt(p, q), voigt(r, t)]
            v = sp.radsimp(sp.expand(acc))
            assert v.is_rational, f"rotated constant not rational: {v}"
            D[I, J] = float(v)
    return D


def exact_orthotropic_C21(E1, E2, E3, G12, G13, G23, nu12, nu13, nu23):
    """Orthotropic stiffness as exact rationals (Fractions of the decimal inputs)."""
    import sympy as sp
    F = lambda x: sp.Rational(str(x))
    S = sp.zeros(6, 6)
    S[0, 0], S[1, 1], S[2, 2] = 1 / F(E1), 1 / F(E2), 1 / F(E3)
    S[0, 1] = S[1, 0] = -F(nu12) / F(E1)
    S[0, 2] = S[2, 0] = -F(nu13) / F(E1)
    S[1, 2] = S[2, 1] = -F(nu23) / F(E2)
    S[3, 3], S[4, 4], S[5, 5] = 1 / F(G12), 1 / F(G13), 1 / F(G23)
    C = S.inv()
    return [C[i, j] for i in range(6) for j in range(i, 6)]


# ---------------------------------------------------------------- assembly
def exact_box_blocks(lam, Lx, Ly, C21_exact_per_material, angles_deg, blocks):
    """K^{ij} (3x3 float arrays) for the requested (i, j) basis pairs of an
    affine box laminate whose in-plane map is x = Lx xi, y = Ly eta."""
    Ix = gram_1d(lam.u)
    Iy = gram_1d(lam.v)
    z = [Fraction(0)]
    for h in lam.ply_thickness:
        z.append(z[-1] + Fraction(float(h)))
    Iz = [gram_1d(lam.t, z[l], z[l + 1]) for l in range(len(lam.ply_thickness))]
    Ds = {}
    nx = lam.u.n_functions
    ns = lam.n_s
    Lx, Ly = Fraction(Lx), Fraction(Ly)
    out = {}
    for (i, j) in blocks:
        it, is_ = divmod(i, ns)
        iy, ix = divmod(is_, nx)
        jt, js = divmod(j, ns)
        jy, jx = divmod(js, nx)
        K = np.zeros((3, 3))
        for l in range(len(lam.ply_thickness)):
            key = (int(lam.ply_material[l]), angles_deg[l])
            if key not in Ds:
                Ds[key] = exact_rotated_D(C21_exact_per_material[key[0]], key[1])
            D = Ds[key]
            for a in range(3):
                for b in range(3):
                    rx, sx = int(a == 0), int(b == 0)
                    ry, sy = int(a == 1), int(b == 1)
                    rz, sz = int(a == 2), int(b == 2)
                    fx = Ix[(rx, sx)].get((ix, jx), 0) * Lx / Lx ** (rx + sx)
                    fy = Iy[(ry, sy)].get((iy, jy), 0) * Ly / Ly ** (ry + sy)
                    fz = Iz[l][(rz, sz)].get((it, jt), 0)
                    f = float(fx * fy * fz)
                    if f == 0.0:
                        continue
                    for c in range(3):
                        for d in range(3):
                            K[c, d] += D[voigt(c, a), voigt(d, b)] * f
        out[(i, j)] = K
    return out


def exact_affine_blocks(lam, A, C21_exact_per_material, angles_deg, blocks):
    """K^{ij} (3x3 float arrays) for the requested (i, j) basis pairs of a
    laminate under the affine extrusion F(xi) = A (xi1, xi2, xi3) with a
    constant rational 3x3 matrix A (columns dS/dxi1, dS/dxi2 and the
    extrusion direction a). With the chain rule d/dx_a = sum_k (A^-1)[k][a]
    d/dxi_k and the constant Jacobian |det A|,

      K^{ij}_{cd} = |det A| sum_l sum_{a,b} C_l[V(c,a), V(d,b)]
                    sum_{k,m} (A^-1)[k][a] (A^-1)[m][b] Ix Iy Iz_l,

    Ix = int d^[k=0] N_ix d^[m=0] N_jx dxi1 and likewise in xi2 and (over
    layer l) xi3: exact 1D integrals in Fractions, as in exact_box_blocks."""
    import sympy as sp
    M = sp.Matrix(3, 3, lambda r, c: sp.Rational(A[r][c]))
    Mi = M.inv()
    det = abs(M.det())
    Ai = [[Fraction(int(sp.fraction(Mi[k, a])[0]), int(sp.fraction(Mi[k, a])[1])) for a in range(3)] for k in range(3)]
    detF = Fraction(int(sp.fraction(det)[0]), int(sp.fraction(det)[1]))
    Ix = gram_1d(lam.u)
    Iy = gram_1d(lam.v)
    z = [Fraction(float(lam.t.knots[0]))]
    for h in lam.ply_thickness:
        z.append(z[-1] + Fraction(float(h)))
    Iz = [gram_1d(lam.t, z[l], z[l + 1]) for l in range(len(lam.ply_thickness))]
    Ds = {}
    nx = lam.u.n_functions
    ns = lam.n_s
    out = {}
    for (i, j) in blocks:
        it, is_ = divmod(i, ns)
        iy, ix = divmod(is_, nx)
        jt, js = divmod(j, ns)
        jy, jx = divmod(js, nx)
        # parametric products: F[k][m] = int d_k N_i d_m N_j per layer
        K = np.zeros((3, 3))
        for l in range(len(lam.ply_thickness)):
            key = (int(lam.ply_material[l]), angles_deg[l])
            if key not in Ds:
                Ds[key] = exact_rotated_D(C21_exact_per_material[key[0]], key[1])
            D = Ds[key]
            Fp = [[Ix[(int(k == 0), int(m == 0))].get((ix, jx), 0) * Iy[(int(k == 1), int(m == 1))].get((iy, jy), 0)
                   * Iz[l][(int(k == 2), int(m == 2))].get((it, jt), 0) for m in range(3)] for k in range(3)]
            for a in range(3):
                for b in range(3):
                    f = sum(Ai[k][a] * Ai[m][b] * Fp[k][m] for k in range(3) for m in range(3)) * detF
                    f = float(f)
                    if f == 0.0:
                        continue
                    for c in range(3):
                        for d in range(3):
                            K[c, d] += D[voigt(c, a), voigt(d, b)] * f
        out[(i, j)] = K
    return out


def _dense_1d(basis, lo=None, hi=None):
    """The four Gram matrices of gram_1d as dense float arrays."""
    I = gram_1d(basis, lo, hi)
    n = basis.n_functions
    out = {}
    for key, entries in I.items():
        M = np.zeros((n, n))
        for (i, j), val in entries.items():
            M[i, j] = float(val)
        out[key] = M
    return out


def exact_box_dL_dD(lam, Lx, Ly, gbar_dense):
    """dL/dD_l (n_plies x 6 x 6, every entry independent) for
    L = sum gbar[i, c, j, d] K^{ij}_{cd} on an affine box laminate.

    K is linear in D_l with coefficient
      dK^{ij}_{cd} / dD_l[V(c,a), V(d,b)] = sum over (a, b) of Ix Iy Iz_l,
    the same exact 1D integrals as exact_box_blocks; the Kronecker product of
    the three 1D matrices gives the coefficient of every basis pair at once.
    """
    Mx = _dense_1d(lam.u)
    My = _dense_1d(lam.v)
    z = [Fraction(0)]
    for h in lam.ply_thickness:
        z.append(z[-1] + Fraction(float(h)))
    n_pl = len(lam.ply_thickness)
    out = np.zeros((n_pl, 6, 6))
    for l in range(n_pl):
        Mz = _dense_1d(lam.t, z[l], z[l + 1])
        for a in range(3):
            for b in range(3):
                rx, sx = int(a == 0), int(b == 0)
                ry, sy = int(a == 1), int(b == 1)
                rz, sz = int(a == 2), int(b == 2)
                fx = Mx[(rx, sx)] * float(Fraction(Lx) / Fraction(Lx) ** (rx + sx))
                fy = My[(ry, sy)] * float(Fraction(Ly) / Fraction(Ly) ** (ry + sy))
                F = np.kron(Mz[(rz, sz)], np.kron(fy, fx))
                for c in range(3):
                    for d in range(3):
                        out[l, voigt(c, a), voigt(d, b)] += np.sum(gbar_dense[:, c, :, d] * F)
    return out
