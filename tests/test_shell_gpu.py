"""General extrusion maps (Eq. extrusion: F = S(xi1, xi2) + xi3 a, S a surface
in R^3, a a constant direction) on the GPU: the split path (6 x 6 Gram blocks
per in-plane pair, P of every configuration, the combine) and the standard
path against the CPU oracle, with the same bar as the plates (pattern
bit-exact, values within 1e-12 of max|K|)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.test_parity_gpu import TOL, assert_parity, gpu_matrix, _sampled_parity
from tests.test_inplane_operators_gpu import inplane_pairs

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


def _nurbs_shell():
    lam = W.shell_plate(n_el=3, degree=2, repeats=1)
    lam.weights = np.random.default_rng(7).uniform(0.5, 2.0, lam.n_s)
    return lam


def _sheared_planar():
    """A planar surface extruded along a tilted direction (S in the plane, a != e_z)."""
    return W.laminate("sheared", W.BSPLINE, 3, 3, [0, 45, -45, 90], 0.01, mapping=W.curved_map(),
                      extrusion=(0.3, -0.2, 1.1))


SHELLS = {
    "bump_p2_3x3": lambda: W.shell_plate(n_el=3, degree=2, repeats=1),
    "bump_p3_4x3_steep_a": lambda: W.laminate("steep", W.BSPLINE, 3, 4, [0, 45, -45, 90, 90, -45], 0.002,
                                              mapping=W.bump_map(0.2), n_el_y=3, extrusion=(0.5, 0.4, 0.8)),
    "bump_nurbs": _nurbs_shell,
    "lagrange_q2_bump": lambda: W.laminate("lag", W.LAGRANGE, 2, 3, [0, 45, 90], 0.01, mapping=W.bump_map(0.1),
                                           thickness_kind=W.LAGRANGE, extrusion=(-0.1, 0.05, 1.0)),
    "sheared_planar": _sheared_planar,
    "triclinic_two_materials": lambda: W.laminate(
        "tri", W.BSPLINE, 2, 3, [0, 20, -35, 90], 0.01, mapping=W.bump_map(0.15), n_el_y=4,
        materials=np.array([W.random_C21(np.random.default_rng(11)), W.random_C21(np.random.default_rng(12))]),
        ply_material=[0, 1, 1, 0], extrusion=(0.1, 0.1, 1.0)),
    # rows of 81 in-plane neighbours: the class-major combine
    "quartic_class_major": lambda: W.laminate("p4", W.BSPLINE, 4, 6, [0, 45], 0.02, mapping=W.bump_map(0.1),
                                              n_el_y=6, thickness_degree=1, extrusion=(0.0, 0.2, 1.0)),
    # 40 configurations: the D tables of the P formation read from global memory
    "many_configurations": lambda: W.laminate("many_cfg", W.BSPLINE, 2, 3, list(np.linspace(-85.0, 85.0, 40)), 0.002,
                                              mapping=W.bump_map(0.1), extrusion=(0.1, 0.0, 1.0)),
    # uneven plies: the streaming combine in chunks
    "uneven_plies_chunked": lambda: W.laminate(
        "uneven", W.BSPLINE, 1, 3, list(np.random.default_rng(4).choice([0.0, 45.0, -45.0, 90.0], 70)),
        np.random.default_rng(5).uniform(0.0005, 0.002, 70), mapping=W.bump_map(0.05), thickness_degree=1,
        extrusion=(0.05, 0.0, 1.0)),
}


@pytest.mark.parametrize("path,arith", [("split", "fp64"), ("split", "double_float"), ("standard", "fp64")])
@pytest.mark.parametrize("name", sorted(SHELLS))
def test_shell_parity(L, name, path, arith):
    lam = SHELLS[name]()
    p = L.Plan.from_laminate(lam)
    assert p.info["shell"] == 1
    if name == "quartic_class_major":
        assert p.info["combine_streaming"] == 0
    if name == "uneven_plies_chunked":
        assert p.info["combine_streaming"] == 1 and p.info["combine_chunks"] >= 2
    p.close()
    assert_parity(gpu_matrix(L, lam, path, arith=arith), O.assemble(lam))


def test_planar_surface_through_the_shell_path(L):
    """(x, y, 0) control points with a = e_z take the general path and give the
    planar plate's matrix."""
    import torch
    lam = W.curved_plate(n_el=4, degree=3, repeats=1)
    plate = L.Plan.from_laminate(lam)
    assert plate.info["shell"] == 0
    a = plate.assemble_split()
    lam.ctrl = np.c_[lam.ctrl, np.zeros(lam.n_s)]
    lam.extrusion = np.array([0.0, 0.0, 1.0])
    shell = L.Plan.from_laminate(lam)
    assert shell.info["shell"] == 1
    b = shell.assemble_split()
    c = shell.assemble_standard()
    torch.cuda.synchronize()
    a, b, c = a.cpu().numpy(), b.cpu().numpy(), c.cpu().numpy()
    assert np.abs(b - a).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(c - a).max() <= 1e-13 * np.abs(a).max()
    plate.close()
    shell.close()


def test_shell_host_output_and_repeatability(L):
    import torch
    lam = W.shell_plate(n_el=6, degree=3, repeats=1)
    p = L.Plan.from_laminate(lam)
    d1 = p.assemble_split()
    d2 = p.assemble_split()
    torch.cuda.synchronize()
    h = np.empty(p.nnz)
    p.assemble_split_host(h)
    assert np.array_equal(d1.cpu().numpy(), d2.cpu().numpy())
    assert np.array_equal(d1.cpu().numpy(), h)
    p.close()


def test_shell_update_angles_then_reassemble(L):
    import torch
    lam = W.shell_plate(n_el=3, degree=2, repeats=1)
    p = L.Plan.from_laminate(lam)
    p.assemble_split()
    new = np.deg2rad(np.linspace(-80.0, 80.0, len(lam.ply_angle)))
    p.update(ply_angle=new)
    lam.ply_angle = new
    vals = p.assemble_split()
    torch.cuda.synchronize()
    ref = O.assemble(lam)
    assert np.abs(vals.cpu().numpy() - ref[2]).max() <= TOL * np.abs(ref[2]).max()
    p.close()


def test_shell_update_materials_then_reassemble_and_differentiate(L):
    """New constants (a triclinic material and a scaled ply material) on a
    shell: the configuration tables, the scaled D of the P formation and the
    adjoint follow the update."""
    import torch
    lam = W.laminate("sh_m", W.BSPLINE, 2, 3, [0, 30, -45, 90], 0.01, mapping=W.bump_map(0.1),
                     materials=np.array([W.ply_C21(), W.ply_C21()]), ply_material=[0, 1, 1, 0],
                     extrusion=(0.15, -0.05, 1.0))
    p = L.Plan.from_laminate(lam)
    p.assemble_split()
    new = np.array([W.random_C21(np.random.default_rng(31)), 3.0 * W.ply_C21()])
    p.update(C21=new)
    lam.C21 = new
    vals = p.assemble_split()
    torch.cuda.synchronize()
    rp, col, ref = O.assemble(lam)
    assert np.abs(vals.cpu().numpy() - ref).max() <= TOL * np.abs(ref).max()
    g = np.random.default_rng(5).standard_normal(len(col))
    dC, dth, dD = p.adjoint(values=torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    rdC, rdth, rdD = O.adjoint(lam, rp, col, g)
    assert np.abs(dD.cpu().numpy().reshape(rdD.shape) - rdD).max() <= 1e-10 * np.abs(rdD).max()
    assert np.abs(dC.cpu().numpy() - rdC).max() <= 1e-10 * np.abs(rdC).max()
    p.close()


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
@pytest.mark.parametrize("scale", [2.0 ** -60, 2.0 ** 60])
def test_shell_extreme_geometry_scale(L, scale, arith):
    """Surface and extrusion scaled by 2^+-60 (double-float: the per-element
    powers of two of the shell K-a keep its float pairs in range)."""
    bump = W.bump_map(0.1)
    lam = W.laminate("geom", W.BSPLINE, 2, 3, [0, 45, 90], 0.01 * scale,
                     mapping=lambda xi, eta: tuple(scale * c for c in bump(xi, eta)),
                     extrusion=(0.1, -0.1, 1.0))
    assert_parity(gpu_matrix(L, lam, "split", arith=arith), O.assemble(lam))


def test_shell_inplane_operators_match_the_oracle(L):
    """Eq. P of a shell from the 6 x 6 Gram blocks and by Appendix A's
    construction with the full DF^-1, against the oracle's Eq. P."""
    import torch
    lam = W.laminate("tri", W.BSPLINE, 3, 3, [0, 30, -60, 90], 0.01, mapping=W.bump_map(0.15), n_el_y=4,
                     extrusion=(0.2, -0.1, 1.0))
    lam.weights = np.random.default_rng(3).uniform(0.5, 2.0, lam.n_s)
    p = L.Plan.from_laminate(lam)
    pairs = inplane_pairs(lam)
    prob = O.Problem(lam)
    rng = np.random.default_rng(1)
    for ply in (0, 2):
        a = p.inplane_operators(ply, L.P_FROM_GRAM)
        b = p.inplane_operators(ply, L.P_VOIGT_FREE)
        torch.cuda.synchronize()
        a, b = a.cpu().numpy(), b.cpu().numpy()
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-13 * scale
        for k in list(rng.choice(len(pairs), 25, replace=False)) + [0, len(pairs) - 1]:
            i_s, j_s = pairs[k]
            ref = O.inplane_P(lam, ply, i_s, j_s, prob)
            assert np.abs(b[k] - ref).max() <= 1e-12 * scale, (ply, i_s, j_s)
            assert np.abs(a[k] - ref).max() <= 1e-12 * scale, (ply, i_s, j_s)
    p.close()


def test_shell_plate_full_size_sampled(L):
    """The shell workload bench.py times (cubic, 64x64, 48 plies): the whole
    pattern, sampled blocks against the oracle and symmetry."""
    _sampled_parity(L, W.shell_plate(), "split", n_rows=40, seed=2)
