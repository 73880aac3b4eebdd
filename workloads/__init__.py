"""Seeded synthetic laminate inputs shared by the tests, smoke() and bench.py.

This module builds the INPUTS of an assembly problem (knot vectors, control
points, ply tables, material constants) and nothing else: it holds none of the
assembly arithmetic. Both the CPU oracle and the CUDA library consume what it
returns.

Workloads (all FP64, physical z through the thickness, ply 0 at z = 0):
  * ``cross_ply_plate``  -- unit square, open uniform B-spline of degree 2 on
    8x8 elements (affine map), 4 plies [0/90/0/90] of 0.0025, one quadratic C0
    element per ply (9 thickness functions, 2700 DOFs).
  * ``curved_plate``     -- cubic B-spline on 64x64 elements, curved map
    x = xi + 0.05 sin(2 pi xi) sin(2 pi eta), y = eta + 0.05 sin(2 pi eta)
    cos(2 pi xi), 48 plies [0/45/-45/90]_6s of 0.001 (97 thickness functions).
  * ``adjoint_plate``    -- cubic, 32x32, 24 plies [0/90]_12 of 0.0025.
  * ``lagrange_plate``   -- Lagrange Q2 on 96x96 elements of the unit square,
    64 plies [0/90]_32 (129 thickness nodes).
  * ``shell_plate``      -- the curved plate's map lifted onto the surface
    z = 0.05 sin(pi xi) sin(pi eta) in R^3 and extruded along the tilted
    direction a = (0.05, -0.03, 1) (Eq. extrusion), 48 plies as curved_plate.
  * ``batch``            -- a seeded list of uneven laminates.
Every generator takes size parameters so that tests can run the same recipe at
sizes a plain CPU code finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BSPLINE = 0
LAGRANGE = 1

# Orthotropic ply (GPa as plain numbers): E1, E2, E3, G12, G13, G23, nu12, nu13, nu23.
PLY_CONSTANTS = dict(E1=140.0, E2=10.0, E3=10.0, G12=5.0, G13=5.0, G23=3.4, nu12=0.3, nu13=0.3, nu23=0.49)
# the orthotropic material of the paper's numerical experiment (Section 4, GPa)
PAGANO_CONSTANTS = dict(E1=25.0, E2=1.0, E3=1.0, G12=0.2, G13=0.2, G23=0.5, nu12=0.25, nu13=0.25, nu23=0.25)


@dataclasses.dataclass
class Basis1D:
    kind: int          # BSPLINE or LAGRANGE
    degree: int
    knots: np.ndarray  # B-spline: open knot vector; Lagrange: element breakpoints

    @property
    def n_functions(self) -> int:
        if self.kind == BSPLINE:
            return len(self.knots) - self.degree - 1
        return self.degree * (len(self.knots) - 1) + 1


@dataclasses.dataclass
class Laminate:
    """One assembly problem: in-plane basis and map, thickness basis, plies."""
    name: str
    u: Basis1D
    v: Basis1D
    ctrl: np.ndarray                 # (n_s, 2) planar or (n_s, 3) surface control points, i_s = iy*nx + ix
    weights: Optional[np.ndarray]    # (n_s,) NURBS weights or None
    t: Basis1D                       # thickness basis, physical z
    ply_thickness: np.ndarray        # (n_plies,)
    ply_material: np.ndarray         # (n_plies,) int32
    ply_angle: np.ndarray            # (n_plies,) radians
    C21: np.ndarray                  # (n_materials, 21) upper-triangle Voigt constants
    nq: Sequence[int] = (0, 0, 0)    # Gauss points per element direction (0 = degree + 1)
    extrusion: Optional[np.ndarray] = None  # direction a of F = S + xi^3 a (None = e_z)

    @property
    def n_s(self) -> int:
        return self.u.n_functions * self.v.n_functions

    @property
    def n_t(self) -> int:
        return self.t.n_functions

    @property
    def n_dof(self) -> int:
        return 3 * self.n_s * self.n_t


# --------------------------------------------------------------------------
# materials
# --------------------------------------------------------------------------
def orthotropic_C21(E1, E2, E3, G12, G13, G23, nu12, nu13, nu23) -> np.ndarray:
    """Voigt stiffness (order 11,22,33,12,13,23, engineering shear) of an
    orthotropic material, as the inverse of its compliance, upper triangle."""
    S = np.zeros((6, 6))
    S[0, 0], S[1, 1], S[2, 2] = 1 / E1, 1 / E2, 1 / E3
    S[0, 1] = S[1, 0] = -nu12 / E1
    S[0, 2] = S[2, 0] = -nu13 / E1
    S[1, 2] = S[2, 1] = -nu23 / E2
    S[3, 3], S[4, 4], S[5, 5] = 1 / G12, 1 / G13, 1 / G23
    C = np.linalg.inv(S)
    C = 0.5 * (C + C.T)
    C[np.abs(C) < 1e-12 * np.abs(C).max()] = 0.0
    return np.array([C[i, j] for i in range(6) for j in range(i, 6)])


def isotropic_C21(E: float, nu: float) -> np.ndarray:
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[0, 0] = C[1, 1] = C[2, 2] = lam + 2 * mu
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    return np.array([C[i, j] for i in range(6) for j in range(i, 6)])


def ply_C21() -> np.ndarray:
    return orthotropic_C21(**PLY_CONSTANTS)


def pagano_C21() -> np.ndarray:
    return orthotropic_C21(**PAGANO_CONSTANTS)


def random_C21(rng: np.random.Generator, scale: float = 10.0) -> np.ndarray:
    """A fully anisotropic (triclinic) symmetric positive definite stiffness."""
    A = rng.standard_normal((6, 6))
    C = scale * (A @ A.T / 6.0 + np.eye(6))
    return np.array([C[i, j] for i in range(6) for j in range(i, 6)])


# --------------------------------------------------------------------------
# bases and maps
# --------------------------------------------------------------------------
def open_uniform_knots(degree: int, n_el: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    inner = np.linspace(a, b, n_el + 1)
    return np.concatenate([np.full(degree, a), inner, np.full(degree, b)])


def greville(knots: np.ndarray, degree: int) -> np.ndarray:
    n = len(knots) - degree - 1
    return np.array([knots[i + 1:i + degree + 1].mean() for i in range(n)])


def lagrange_nodes(breakpoints: np.ndarray, degree: int) -> np.ndarray:
    nodes = [breakpoints[0]]
    for e in range(len(breakpoints) - 1):
        a, b = breakpoints[e], breakpoints[e + 1]
        for k in range(1, degree + 1):
            nodes.append(a + (b - a) * k / degree)
    return np.array(nodes)


def anchors(b: Basis1D) -> np.ndarray:
    """Parametric anchor of each function: Greville abscissae (B-spline) or
    nodes (Lagrange). Control points placed at the image of the anchors."""
    if b.kind == BSPLINE:
        return greville(b.knots, b.degree)
    return lagrange_nodes(b.knots, b.degree)


def control_points(u: Basis1D, v: Basis1D, mapping) -> np.ndarray:
    """Control points X_i = F(anchor_i): (n_s, 2) for a planar map, (n_s, 3)
    when `mapping` returns three coordinates (a surface in R^3)."""
    au, av = anchors(u), anchors(v)
    dim = len(mapping(au[0], av[0]))
    X = np.zeros((len(av) * len(au), dim))
    for iy, eta in enumerate(av):
        for ix, xi in enumerate(au):
            X[iy * len(au) + ix] = mapping(xi, eta)
    return X


def identity_map(xi, eta):
    return (xi, eta)


def scaled_map(Lx, Ly):
    return lambda xi, eta: (Lx * xi, Ly * eta)


def curved_map(amp: float = 0.05):
    def F(xi, eta):
        x = xi + amp * math.sin(2 * math.pi * xi) * math.sin(2 * math.pi * eta)
        y = eta + amp * math.sin(2 * math.pi * eta) * math.cos(2 * math.pi * xi)
        return (x, y)
    return F


def bump_map(amp: float = 0.05, inner=None):
    """A surface in R^3: the planar map `inner` (the curved map by default)
    lifted onto z = amp sin(pi xi) sin(pi eta)."""
    inner = curved_map() if inner is None else inner

    def F(xi, eta):
        x, y = inner(xi, eta)
        return (x, y, amp * math.sin(math.pi * xi) * math.sin(math.pi * eta))
    return F


def affine_surface_map(A):
    """S(xi, eta) = A[:, 0] xi + A[:, 1] eta for a 3x3 matrix A (columns
    dS/dxi1, dS/dxi2 and, used as the extrusion direction, a)."""
    A = np.asarray(A, np.float64)
    return lambda xi, eta: tuple(A[:, 0] * xi + A[:, 1] * eta)


def thickness_basis(ply_thickness: Sequence[float], degree: int = 2, kind: int = BSPLINE,
                    elements_per_ply: int = 1) -> Basis1D:
    """C0 thickness basis with `elements_per_ply` elements of degree `degree`
    in every ply (interfaces repeated `degree` times for B-splines)."""
    z = [0.0]
    for h in ply_thickness:
        z0 = z[-1]
        for k in range(1, elements_per_ply + 1):
            z.append(z0 + h * k / elements_per_ply)
    z = np.array(z)
    if kind == LAGRANGE:
        return Basis1D(LAGRANGE, degree, z)
    knots = [z[0]] * (degree + 1)
    for zi in z[1:-1]:
        knots += [zi] * degree
    knots += [z[-1]] * (degree + 1)
    return Basis1D(BSPLINE, degree, np.array(knots))


def single_element_thickness(H: float, degree: int) -> Basis1D:
    """One B-spline element of degree `degree` through the full thickness."""
    return Basis1D(BSPLINE, degree, np.array([0.0] * (degree + 1) + [H] * (degree + 1)))


def stack(pattern: Sequence[float], repeats: int, symmetric: bool) -> List[float]:
    s = list(pattern) * repeats
    if symmetric:
        s = s + s[::-1]
    return s


def laminate(name: str, inplane_kind: int, degree: int, n_el: int, angles_deg: Sequence[float],
             ply_h, mapping=identity_map, thickness_degree: int = 2, thickness_kind: int = BSPLINE,
             materials: Optional[np.ndarray] = None, ply_material: Optional[Sequence[int]] = None,
             n_el_y: Optional[int] = None, degree_y: Optional[int] = None, weights=None,
             thickness: Optional[Basis1D] = None, nq=(0, 0, 0), extrusion=None) -> Laminate:
    n_el_y = n_el if n_el_y is None else n_el_y
    degree_y = degree if degree_y is None else degree_y
    if inplane_kind == BSPLINE:
        u = Basis1D(BSPLINE, degree, open_uniform_knots(degree, n_el))
        v = Basis1D(BSPLINE, degree_y, open_uniform_knots(degree_y, n_el_y))
    else:
        u = Basis1D(LAGRANGE, degree, np.linspace(0.0, 1.0, n_el + 1))
        v = Basis1D(LAGRANGE, degree_y, np.linspace(0.0, 1.0, n_el_y + 1))
    n_plies = len(angles_deg)
    h = np.full(n_plies, ply_h) if np.isscalar(ply_h) else np.asarray(ply_h, dtype=np.float64)
    t = thickness if thickness is not None else thickness_basis(h, thickness_degree, thickness_kind)
    mats = ply_C21()[None, :] if materials is None else np.atleast_2d(materials)
    pm = np.zeros(n_plies, np.int32) if ply_material is None else np.asarray(ply_material, np.int32)
    return Laminate(name=name, u=u, v=v, ctrl=control_points(u, v, mapping),
                    weights=None if weights is None else np.asarray(weights, np.float64),
                    t=t, ply_thickness=h, ply_material=pm,
                    ply_angle=np.deg2rad(np.asarray(angles_deg, np.float64)), C21=mats, nq=tuple(nq),
                    extrusion=None if extrusion is None else np.asarray(extrusion, np.float64))


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------
def cross_ply_plate(n_el: int = 8, degree: int = 2, n_plies: int = 4) -> Laminate:
    """Unit square, open uniform B-spline, [0/90/...] plies of 0.0025."""
    angles = [0.0 if k % 2 == 0 else 90.0 for k in range(n_plies)]
    return laminate(f"cross_ply_p{degree}_{n_el}x{n_el}_{n_plies}plies", BSPLINE, degree, n_el, angles, 0.0025)


def curved_plate(n_el: int = 64, degree: int = 3, repeats: int = 6) -> Laminate:
    """Curved plate, [0/45/-45/90]_{repeats}s, plies of 0.001."""
    angles = stack([0.0, 45.0, -45.0, 90.0], repeats, True)
    return laminate(f"curved_p{degree}_{n_el}x{n_el}_{len(angles)}plies", BSPLINE, degree, n_el, angles, 0.001,
                    mapping=curved_map())


def shell_plate(n_el: int = 64, degree: int = 3, repeats: int = 6,
                extrusion=(0.05, -0.03, 1.0)) -> Laminate:
    """Curved shell: the curved plate's map lifted onto the bump
    z = 0.05 sin(pi xi) sin(pi eta) and extruded along a tilted direction a
    (Eq. extrusion), [0/45/-45/90]_{repeats}s, plies of 0.001 in xi^3."""
    angles = stack([0.0, 45.0, -45.0, 90.0], repeats, True)
    return laminate(f"shell_p{degree}_{n_el}x{n_el}_{len(angles)}plies", BSPLINE, degree, n_el, angles, 0.001,
                    mapping=bump_map(), extrusion=extrusion)


def adjoint_plate(n_el: int = 32, degree: int = 3, n_plies: int = 24) -> Laminate:
    angles = [0.0 if k % 2 == 0 else 90.0 for k in range(n_plies)]
    return laminate(f"adjoint_p{degree}_{n_el}x{n_el}_{n_plies}plies", BSPLINE, degree, n_el, angles, 0.0025)


def lagrange_plate(n_el: int = 96, n_plies: int = 64, ply_h: float = 0.0025) -> Laminate:
    angles = [0.0 if k % 2 == 0 else 90.0 for k in range(n_plies)]
    return laminate(f"lagrange_q2_{n_el}x{n_el}_{n_plies}plies", LAGRANGE, 2, n_el, angles, ply_h,
                    thickness_kind=LAGRANGE)


def batch_laminates(count: int = 256, seed: int = 517, meshes=(16, 24, 32, 48), plies=(8, 64)) -> List[Laminate]:
    """Uneven laminates: quadratic B-spline meshes drawn from `meshes` on the
    unit square, ply count uniform in `plies`, angles from {0, +-45, 90}, 1-4
    materials (material k: the ply constants with E1 scaled by 1 + 0.25 k),
    ply thickness U[0.0005, 0.002]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n_el = int(rng.choice(meshes))
        n_plies = int(rng.integers(plies[0], plies[1] + 1))
        n_mat = int(rng.integers(1, 5))
        angles = rng.choice([0.0, 45.0, -45.0, 90.0], size=n_plies)
        pm = rng.integers(0, n_mat, size=n_plies)
        h = rng.uniform(0.0005, 0.002, size=n_plies)
        mats = []
        for k in range(n_mat):
            c = dict(PLY_CONSTANTS)
            c["E1"] = c["E1"] * (1.0 + 0.25 * k)
            mats.append(orthotropic_C21(**c))
        out.append(laminate(f"batch{b}_{n_el}x{n_el}_{n_plies}plies", BSPLINE, 2, n_el, angles, h,
                            materials=np.array(mats), ply_material=pm))
    return out


def pagano_sweep_plate(degree: int, n_el: int, n_layers: int, stack: str = "cross", thickness: float = 0.1) -> Laminate:
    """The shape of the paper's experiment (Section 4): a flat unit-square plate
    of n_layers equal layers of the Pagano material, stacked 0/90/0/90/...
    ("cross") or 0/45/-45/90/... ("quasi"), open uniform C^{p-1} B-splines of
    the same degree p in all directions on n_el x n_el in-plane elements, and
    ONE element of degree p through the whole thickness."""
    cycle = [0.0, 90.0] if stack == "cross" else [0.0, 45.0, -45.0, 90.0]
    angles = [cycle[k % len(cycle)] for k in range(n_layers)]
    return laminate(f"pagano_{stack}_p{degree}_{n_el}x{n_el}_{n_layers}layers", BSPLINE, degree, n_el, angles,
                    thickness / n_layers, materials=pagano_C21()[None, :],
                    thickness=single_element_thickness(thickness, degree))
