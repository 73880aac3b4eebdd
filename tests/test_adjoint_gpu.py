"""Parity of lam_adjoint (GPU) with the oracle's adjoint, and its properties
at full size (GPU required).

Bar: dL/dD, dL/dC and dL/dtheta within 1e-12 of the largest oracle entry for
the default FP64 evaluation; 1e-10 for the opt-in double-float pass (about
2^-44 per term; sums of up to 10^5 signed terms of similar size stay three
orders of magnitude inside). At the full 32 x 32 cubic 24-ply size the oracle is too slow, so
the checks are properties that hold at any size: Euler's identity against the
split assembly, central finite differences of the split assembly in the
angles and constants (step 1e-6, agreement 1e-6), and the double-float pass
against the FP64 pass.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_1905_05417_gb300 import build
    build.build()
    import paper_1905_05417_gb300 as lam
    lam.load()
    return lam


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def gpu_adjoint(L, lam, g=None, u=None, v=None, fp64=False, double_float=False):
    """double_float: the whole double-float pipeline (plan arithmetic and the
    adjoint's flag); fp64: LAM_ADJOINT_FP64 (low rank through the generic pass)."""
    import torch
    p = L.Plan.from_laminate(lam, arith=L.ARITH_DOUBLE_FLOAT if double_float else L.ARITH_FP64)
    kw = {}
    if g is not None:
        kw["values"] = torch.from_numpy(g).cuda()
    else:
        kw["u"] = torch.from_numpy(np.atleast_2d(u)).cuda()
        kw["v"] = torch.from_numpy(np.atleast_2d(v)).cuda()
    dC, dth, dD = p.adjoint(fp64=fp64, double_float=double_float, **kw)
    torch.cuda.synchronize()
    out = dC.cpu().numpy(), dth.cpu().numpy(), dD.cpu().numpy()
    p.close()
    return out


CASES = {
    "cross_ply_8x8_p2": W.cross_ply_plate,
    "curved_p3_3x3_8plies": lambda: W.curved_plate(n_el=3, degree=3, repeats=1),
    "lagrange_q2_3x3": lambda: W.lagrange_plate(n_el=3, n_plies=4),
    "triclinic_two_materials": lambda: W.laminate(
        "tri", W.BSPLINE, 2, 3, [0, 20, -35, 90], 0.01, mapping=W.curved_map(),
        materials=np.array([W.random_C21(np.random.default_rng(11)), W.random_C21(np.random.default_rng(12))]),
        ply_material=[0, 1, 1, 0]),
    # one thickness element across five plies: every pair meets every ply
    "single_thickness_element": lambda: W.laminate(
        "ss", W.BSPLINE, 3, 3, [0, 90, 0, 90, 0], [0.1, 0.1, 0.2, 0.1, 0.1], mapping=W.curved_map(),
        thickness=W.single_element_thickness(0.6, 3)),
    "nurbs_p2_4x4": lambda: _nurbs(),
    "quartic_inplane": lambda: W.laminate("p4", W.BSPLINE, 4, 5, [0, 45], 0.02, mapping=W.curved_map(),
                                          n_el_y=4, thickness_degree=1),
    "single_element_single_ply": lambda: W.laminate("min", W.BSPLINE, 1, 1, [30.0], 0.5, thickness_degree=1),
    # general extrusions (Eq. extrusion): the FP64 contraction over the 6 x 6 Gram blocks
    "shell_bump_p2": lambda: W.shell_plate(n_el=3, degree=2, repeats=1, extrusion=(0.3, 0.2, 0.9)),
    "shell_triclinic": lambda: W.laminate(
        "shtri", W.BSPLINE, 2, 3, [0, 20, -35, 90], 0.01, mapping=W.bump_map(0.15), extrusion=(0.1, -0.2, 1.0),
        materials=np.array([W.random_C21(np.random.default_rng(11)), W.random_C21(np.random.default_rng(12))]),
        ply_material=[0, 1, 1, 0]),
    # one sextic element through five plies: 49 thickness pairs per ply, the FP64-only path
    "shell_one_thickness_element": lambda: W.laminate(
        "shss", W.BSPLINE, 2, 2, [0, 90, 0, 90, 0], [0.1, 0.1, 0.2, 0.1, 0.1], mapping=W.bump_map(0.1),
        thickness=W.single_element_thickness(0.6, 6), extrusion=(0.2, 0.1, 1.0)),
}


def _nurbs():
    lam = W.curved_plate(n_el=4, degree=2, repeats=1)
    lam.weights = np.random.default_rng(7).uniform(0.5, 2.0, lam.n_s)
    return lam


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("double_float", [False, True])
def test_csr_cotangent_parity(L, name, double_float):
    lam = CASES[name]()
    rp, col = O.pattern(lam)
    g = np.random.default_rng(1905).standard_normal(len(col))
    ref = O.adjoint(lam, rp, col, g)
    got = gpu_adjoint(L, lam, g=g, double_float=double_float)
    tol = 1e-10 if double_float else 1e-12
    assert rel(got[2], ref[2]) <= tol, "dL/dD"
    assert rel(got[0], ref[0]) <= tol, "dL/dC"
    # dtheta = <dL/dD, dD/dtheta>: its error scales with |dL/dD| |C|
    assert np.abs(got[1] - ref[1]).max() <= tol * max(np.abs(ref[1]).max(),
                                                      np.abs(ref[2]).max() * np.abs(lam.C21).max()), "dL/dtheta"


@pytest.mark.parametrize("name", ["curved_p3_3x3_8plies", "lagrange_q2_3x3", "single_thickness_element",
                                  "shell_bump_p2"])
@pytest.mark.parametrize("generic", [False, True])
def test_lowrank_cotangent_parity(L, name, generic):
    """The factorised FP64 contraction (default) and the generic FP64 pass
    (LAM_ADJOINT_FP64) of a rank-2 cotangent."""
    lam = CASES[name]()
    rp, col = O.pattern(lam)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal((2, lam.n_dof)), rng.standard_normal((2, lam.n_dof))
    ref = O.adjoint(lam, rp, col, O.lowrank_cotangent(rp, col, u, v))
    got = gpu_adjoint(L, lam, u=u, v=v, fp64=generic)
    assert rel(got[2], ref[2]) <= 1e-12
    assert rel(got[0], ref[0]) <= 1e-12


@pytest.mark.parametrize("double_float", [False, True])
def test_nonfinite_and_out_of_range_cotangents(L, double_float):
    """Cotangents scaled by 2^+-200 give the exactly scaled gradient (the
    double-float pass rejects them and the FP64 pass recomputes); an infinite
    entry gives a non-finite gradient."""
    lam = W.curved_plate(n_el=3, degree=3, repeats=1)
    rp, col = O.pattern(lam)
    g = np.random.default_rng(5).standard_normal(len(col))
    ref = O.adjoint(lam, rp, col, g)
    for scale in (2.0 ** 200, 2.0 ** -200):   # beyond float range either way: exact scaling of the result
        got = gpu_adjoint(L, lam, g=g * scale, double_float=double_float)
        assert rel(got[2], ref[2] * scale) <= 1e-12
        assert rel(got[0], ref[0] * scale) <= 1e-12
    g2 = g.copy()
    g2[len(g2) // 2] = np.inf
    got = gpu_adjoint(L, lam, g=g2, double_float=double_float)
    assert not np.all(np.isfinite(got[2]))


def test_zero_cotangent_gives_zero(L):
    lam = W.cross_ply_plate(n_el=2, n_plies=2)
    rp, col = O.pattern(lam)
    got = gpu_adjoint(L, lam, g=np.zeros(len(col)))
    assert np.all(got[0] == 0) and np.all(got[1] == 0) and np.all(got[2] == 0)


# ---------------------------------------------------------------- full size (32 x 32 cubic, 24 plies)
@pytest.fixture(scope="module")
def full(L):
    import torch
    lam = W.adjoint_plate()
    p = L.Plan.from_laminate(lam)
    g = torch.randn(p.nnz, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1905))
    return lam, p, g


def test_full_size_double_float_matches_fp64(L, full):
    lam, p, g = full
    a = [x.cpu().numpy() for x in p.adjoint(values=g, double_float=True)]
    b = [x.cpu().numpy() for x in p.adjoint(values=g)]
    assert rel(a[2], b[2]) <= 1e-10 and rel(a[0], b[0]) <= 1e-10
    for kw in ({}, {"double_float": True}):
        c = [x.cpu().numpy() for x in p.adjoint(values=g, **kw)]
        ref = b if not kw else a
        assert all(np.array_equal(x, y) for x, y in zip(ref, c))  # bitwise repeatable


def test_full_size_euler_identity(L, full):
    import torch
    lam, p, g = full
    _, _, dD = p.adjoint(values=g)
    K = p.assemble_split()
    Lval = float(torch.dot(g, K))
    scale = float(torch.dot(g.abs(), K.abs()))
    Ds = [O.rotated_D(lam.C21[lam.ply_material[l]], lam.ply_angle[l]) for l in range(len(lam.ply_angle))]
    lhs = float(sum(np.sum(dD[l].cpu().numpy() * Ds[l]) for l in range(len(Ds))))
    assert abs(lhs - Lval) <= 1e-11 * scale


def test_full_size_finite_differences(L, full):
    """Central differences of L = g . K(theta, C) through lam_assemble_split."""
    import torch
    lam, p, g = full
    dC, dth, _ = p.adjoint(values=g)
    dC, dth = dC.cpu().numpy(), dth.cpu().numpy()
    ang0, C0 = lam.ply_angle.copy(), lam.C21.copy()

    def Lof(ang, C):
        p.update(ply_angle=ang, C21=C)
        return float(torch.dot(g, p.assemble_split()))

    h = 1e-6
    for l in (0, 5, 23):
        a1, a2 = ang0.copy(), ang0.copy()
        a1[l] += h
        a2[l] -= h
        fd = (Lof(a1, C0) - Lof(a2, C0)) / (2 * h)
        assert abs(fd - dth[l]) <= 1e-6 * np.abs(dth).max(), (l, fd, dth[l])
    for k in (0, 1, 6, 9, 14, 20):
        hk = 1e-6 * abs(C0[0, k]) if C0[0, k] != 0 else 1e-6
        c1, c2 = C0.copy(), C0.copy()
        c1[0, k] += hk
        c2[0, k] -= hk
        fd = (Lof(ang0, c1) - Lof(ang0, c2)) / (2 * hk)
        assert abs(fd - dC[0, k]) <= 1e-6 * np.abs(dC).max(), (k, fd, dC[0, k])
    p.update(ply_angle=ang0, C21=C0)


def test_autograd_function(L):
    import torch
    lam = W.cross_ply_plate(n_el=3, n_plies=3)
    p = L.Plan.from_laminate(lam)
    C = torch.tensor(lam.C21, dtype=torch.float64, requires_grad=True)
    th = torch.tensor(lam.ply_angle, dtype=torch.float64, requires_grad=True)
    K = L.StiffnessFunction.apply(p, C, th)
    g = torch.randn(K.shape, dtype=torch.float64, device=K.device, generator=torch.Generator("cuda").manual_seed(2))
    (K * g).sum().backward()
    rp, col = O.pattern(lam)
    ref = O.adjoint(lam, rp, col, g.cpu().numpy())
    assert rel(C.grad.numpy(), ref[0]) <= 1e-10
    assert rel(th.grad.numpy(), ref[1]) <= 1e-9


def test_full_size_compliance_gradient_finite_differences(L, full):
    """The compliance loss L = u^T K u (a rank-one cotangent u u^T) on the full
    plate: the factorised low-rank adjoint against central differences of
    u^T K(theta, C) u computed with the split assembly and a CSR product."""
    import torch
    lam, p, _ = full
    u = torch.randn(p.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    row_ptr, col = p.pattern()
    col = col.long()  # torch's CSR wants one index type
    dC, dth, _ = p.adjoint(u=u[None, :], v=u[None, :], want_dD=False)
    dC, dth = dC.cpu().numpy(), dth.cpu().numpy()
    ang0, C0 = lam.ply_angle.copy(), lam.C21.copy()

    def Lof(ang, C):
        p.update(ply_angle=ang, C21=C)
        K = torch.sparse_csr_tensor(row_ptr, col, p.assemble_split(), size=(p.n_dof, p.n_dof))
        return float(torch.dot(u, K @ u))

    h = 1e-6
    for l in (0, 11, 23):
        a1, a2 = ang0.copy(), ang0.copy()
        a1[l] += h
        a2[l] -= h
        fd = (Lof(a1, C0) - Lof(a2, C0)) / (2 * h)
        assert abs(fd - dth[l]) <= 1e-6 * np.abs(dth).max(), (l, fd, dth[l])
    for k in (0, 3, 9, 15, 20):
        hk = 1e-6 * abs(C0[0, k]) if C0[0, k] != 0 else 1e-6
        c1, c2 = C0.copy(), C0.copy()
        c1[0, k] += hk
        c2[0, k] -= hk
        fd = (Lof(ang0, c1) - Lof(ang0, c2)) / (2 * hk)
        assert abs(fd - dC[0, k]) <= 1e-6 * np.abs(dC).max(), (k, fd, dC[0, k])
    p.update(ply_angle=ang0, C21=C0)
