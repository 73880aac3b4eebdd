"""Parity of the CUDA assembly paths with the CPU oracle (GPU required).

Bar (FP64 throughout): the sparsity pattern is bit-exact, and the values agree
to max|K_gpu - K_oracle| <= 1e-12 * max|K_oracle| (the paper states that the
split and the standard matrices agree to machine precision, Section 3 after
Eq. Q and Section 4). Small cases are compared element by element over the
whole matrix; the full-size workloads, in the launch configuration bench.py
times, are compared on the whole pattern and on sampled blocks that the
oracle integrates one by one, plus symmetry.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def gpu_matrix(L, lam, path="split", class_tol=-1.0):
    import torch
    p = L.Plan.from_laminate(lam, class_tol=class_tol)
    row_ptr, col = p.pattern()
    vals = p.assemble_split() if path == "split" else p.assemble_standard()
    torch.cuda.synchronize()
    out = row_ptr.cpu().numpy(), col.cpu().numpy(), vals.cpu().numpy()
    p.close()
    return out


def assert_parity(got, ref, tol=TOL):
    rp, col, val = got
    rp_o, col_o, val_o = ref
    assert np.array_equal(rp, rp_o), "row_ptr differs"
    assert np.array_equal(col, col_o), "col_ind differs"
    assert np.all(np.isfinite(val))
    err = np.abs(val - val_o).max() / np.abs(val_o).max()
    assert err <= tol, f"max rel error {err:.3e}"
    return err


SMALL = {
    "cross_ply_8x8_p2": W.cross_ply_plate,
    "curved_p3_3x3_8plies": lambda: W.curved_plate(n_el=3, degree=3, repeats=1),
    "curved_p2_5x4_mixed": lambda: W.laminate("c", W.BSPLINE, 2, 5, [0, 45, -45, 90, 90, -45], 0.002,
                                               mapping=W.curved_map(), n_el_y=4, degree_y=3),
    "lagrange_q2_3x3": lambda: W.lagrange_plate(n_el=3, n_plies=4),
    "lagrange_q1_4x3": lambda: W.laminate("q1", W.LAGRANGE, 1, 4, [0, 90, 30], 0.01, n_el_y=3,
                                           mapping=W.curved_map(0.02), thickness_kind=W.LAGRANGE,
                                           thickness_degree=1),
    "one_element_through_thickness": lambda: W.laminate(
        "ss", W.BSPLINE, 3, 3, [0, 90, 0, 90, 0], [0.1, 0.1, 0.2, 0.1, 0.1], mapping=W.curved_map(),
        thickness=W.single_element_thickness(0.6, 3)),
    "two_elements_per_ply": lambda: W.laminate(
        "two", W.BSPLINE, 2, 3, [0, 45, 90], 0.01, mapping=W.curved_map(),
        thickness=W.thickness_basis([0.01] * 3, 2, W.BSPLINE, elements_per_ply=2)),
    "single_element_single_ply": lambda: W.laminate("min", W.BSPLINE, 1, 1, [30.0], 0.5, thickness_degree=1),
    "more_gauss_points": lambda: W.laminate("nq", W.BSPLINE, 2, 3, [0, 90], 0.05, mapping=W.curved_map(),
                                            nq=(5, 4, 4)),
    # rows of 81 in-plane neighbours (729 values > 512 threads): the class-major combine
    "quartic_inplane": lambda: W.laminate("p4", W.BSPLINE, 4, 8, [0, 45], 0.02, mapping=W.curved_map(),
                                          n_el_y=8, thickness_degree=1),
    # uneven plies: hundreds of distinct Q vectors, the streaming combine in chunks
    "uneven_plies_many_classes": lambda: W.laminate(
        "uneven", W.BSPLINE, 1, 3, list(np.random.default_rng(4).choice([0.0, 45.0, -45.0, 90.0], 70)),
        np.random.default_rng(5).uniform(0.0005, 0.002, 70), mapping=W.curved_map(), thickness_degree=1),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("path", ["split", "standard"])
def test_small_full_parity(L, name, path):
    lam = SMALL[name]()
    assert_parity(gpu_matrix(L, lam, path), O.assemble(lam))


def test_nurbs_parity(L):
    lam = W.curved_plate(n_el=4, degree=2, repeats=1)
    lam.weights = np.random.default_rng(7).uniform(0.5, 2.0, lam.n_s)
    ref = O.assemble(lam)
    for path in ("split", "standard"):
        assert_parity(gpu_matrix(L, lam, path), ref)


def test_fully_anisotropic_materials(L):
    """Triclinic constants: every coupling of D is nonzero (general combine)."""
    rng = np.random.default_rng(11)
    lam = W.laminate("tri", W.BSPLINE, 2, 3, [0, 20, -35, 90], 0.01, mapping=W.curved_map(),
                     materials=np.array([W.random_C21(rng), W.random_C21(rng)]), ply_material=[0, 1, 1, 0])
    p = L.Plan.from_laminate(lam)
    assert p.info["monoclinic"] == 0
    ref = O.assemble(lam)
    for path in ("split", "standard"):
        assert_parity(gpu_matrix(L, lam, path), ref)


def test_exact_classes_and_merged_classes_agree(L):
    lam = W.curved_plate(n_el=3, degree=3, repeats=1)
    a = gpu_matrix(L, lam, "split", class_tol=0.0)
    b = gpu_matrix(L, lam, "split")
    assert np.abs(a[2] - b[2]).max() <= 1e-14 * np.abs(a[2]).max()


def test_split_equals_standard_on_gpu(L):
    """The split path forms its in-plane Gram blocks in double-float arithmetic
    on the FP32 pipes (about 2^-47 per term); against the all-FP64 standard
    path it stays two orders of magnitude inside the parity bar."""
    lam = W.curved_plate(n_el=6, degree=3, repeats=2)
    s = gpu_matrix(L, lam, "split")
    t = gpu_matrix(L, lam, "standard")
    assert np.array_equal(s[1], t[1])
    assert np.abs(s[2] - t[2]).max() <= 1e-14 * 20 * np.abs(t[2]).max()


def test_host_output_path_matches_device_path(L):
    import torch
    lam = W.curved_plate(n_el=8, degree=3, repeats=1)
    p = L.Plan.from_laminate(lam)
    d = p.assemble_split()
    torch.cuda.synchronize()
    h = np.empty(p.nnz)
    pinned = torch.empty(p.nnz, dtype=torch.float64, pin_memory=True)
    p.assemble_split_host(pinned)
    p.assemble_split_host(h)
    assert np.array_equal(d.cpu().numpy(), h)
    assert np.array_equal(pinned.numpy(), h)
    p.close()


def test_repeated_calls_are_bitwise_stable(L):
    import torch
    lam = W.curved_plate(n_el=5, degree=3, repeats=1)
    p = L.Plan.from_laminate(lam)
    a = p.assemble_split().cpu().numpy()
    b = p.assemble_split().cpu().numpy()
    c = p.assemble_standard().cpu().numpy()
    d = p.assemble_standard().cpu().numpy()
    assert np.array_equal(a, b) and np.array_equal(c, d)
    p.close()


def test_update_angles_then_reassemble(L):
    lam = W.cross_ply_plate()
    p = L.Plan.from_laminate(lam)
    new = np.deg2rad([45.0, -45.0, 30.0, 0.0])
    p.update(ply_angle=new)
    lam.ply_angle = new
    import torch
    vals = p.assemble_split()
    torch.cuda.synchronize()
    ref = O.assemble(lam)
    err = np.abs(vals.cpu().numpy() - ref[2]).max() / np.abs(ref[2]).max()
    assert err <= TOL
    p.close()


# ---------------------------------------------------------------- full sizes, sampled
def _sampled_parity(L, lam, path, n_rows=120, seed=0, whole_pattern=True):
    import torch
    p = L.Plan.from_laminate(lam)
    row_ptr, col = p.pattern()
    vals = p.assemble_split() if path == "split" else p.assemble_standard()
    torch.cuda.synchronize()
    rp = row_ptr.cpu().numpy()
    cl = col.cpu().numpy()
    v = vals.cpu().numpy()
    if whole_pattern:
        # the whole pattern, bit for bit, against the oracle's own construction
        rp_o, cl_o = O.pattern(lam)
        assert np.array_equal(rp, rp_o) and np.array_equal(cl, cl_o)
        del rp_o, cl_o
    else:
        assert rp[0] == 0 and rp[-1] == p.nnz and np.all(np.diff(rp) > 0)
    assert np.all(np.isfinite(v))
    rng = np.random.default_rng(seed)
    n = p.n_dof
    rows = list(rng.choice(n, n_rows, replace=False)) + [0, 1, 2, n - 3, n - 2, n - 1]
    prob = O.Problem(lam)
    scale = np.abs(v).max()
    worst = 0.0
    for r in rows:
        ks = np.arange(rp[r], rp[r + 1])
        pick = np.unique(np.concatenate([ks[:3], ks[-3:], rng.choice(ks, 6)]))
        for k in pick:
            i, j = r // 3, cl[k] // 3
            B = O.block(lam, i, j, prob)
            ref = B[r % 3, cl[k] % 3]
            worst = max(worst, abs(v[k] - ref))
            # symmetry: the transposed entry is stored and equal
            rj = int(cl[k])
            kk = rp[rj] + np.searchsorted(cl[rp[rj]:rp[rj + 1]], r)
            assert cl[kk] == r
            assert abs(v[kk] - v[k]) <= 1e-14 * scale
    # the oracle's blocks scale like the matrix (sampled max vs true max)
    assert worst <= TOL * scale, worst / scale
    p.close()


def test_adjoint_plate_full_size_sampled(L):
    _sampled_parity(L, W.adjoint_plate(), "split")


def test_curved_plate_full_size_sampled_split(L):
    """The benchmark workload (cubic, 64x64 curved, 48 plies), as bench.py launches it."""
    _sampled_parity(L, W.curved_plate(), "split", n_rows=60)


def test_adjoint_plate_full_size_sampled_standard(L):
    _sampled_parity(L, W.adjoint_plate(), "standard", n_rows=60, seed=1)


def _uneven(materials, seed):
    rng = np.random.default_rng(seed)
    n = 9
    return W.laminate("uneven_q", W.BSPLINE, 2, 5, list(rng.choice([0.0, 45.0, -45.0, 90.0], n)),
                      rng.uniform(0.0005, 0.002, n), mapping=W.curved_map(0.03), materials=materials,
                      ply_material=list(rng.integers(0, len(materials), n)))


def test_uneven_plies_four_materials(L):
    """A batch-like stack (quadratic in-plane, uneven plies, four materials)."""
    mats = np.array([W.ply_C21() * (1 + 0.25 * k) for k in range(4)])
    lam = _uneven(mats, 21)
    p = L.Plan.from_laminate(lam)
    assert p.info["combine_streaming"] == 1 and p.info["monoclinic"] == 1
    assert_parity(gpu_matrix(L, lam, "split"), O.assemble(lam))


def test_uneven_plies_triclinic(L):
    rng = np.random.default_rng(3)
    lam = _uneven(np.array([W.random_C21(rng), W.random_C21(rng)]), 22)
    p = L.Plan.from_laminate(lam)
    assert p.info["combine_streaming"] == 1 and p.info["monoclinic"] == 0
    assert_parity(gpu_matrix(L, lam, "split"), O.assemble(lam))


def test_chunked_host_output_uneven_plies(L):
    lam = _uneven(np.array([W.ply_C21()]), 23)
    p = L.Plan.from_laminate(lam)
    import torch
    d = p.assemble_split()
    torch.cuda.synchronize()
    h = np.empty(p.nnz)
    p.assemble_split_host(h)
    assert np.array_equal(d.cpu().numpy(), h)
    p.close()


# ---------------------------------------------------------------- scale robustness of the double-float steps
@pytest.mark.parametrize("scale", [2.0 ** -90, 2.0 ** 90])
def test_extreme_geometry_scale(L, scale):
    """In-plane coordinates scaled by 2^+-90: K-a's per-element power-of-two
    scaling keeps its float pairs in range; entries of K then span ~2^360, the
    largest ones overflow float in the combine's double-float pass (2^90) and
    the FP64 pass recomputes."""
    curved = W.curved_map(0.04)
    lam = W.laminate("geom", W.BSPLINE, 2, 3, [0, 45, 90], 0.01,
                     mapping=lambda xi, eta: tuple(scale * c for c in curved(xi, eta)))
    assert_parity(gpu_matrix(L, lam, "split"), O.assemble(lam))


@pytest.mark.parametrize("scale", [2.0 ** -200, 2.0 ** 200])
def test_extreme_material_scale(L, scale):
    """Constants scaled by 2^+-200: every entry of K is beyond float range, the
    combine's double-float pass flags it and the FP64 pass recomputes."""
    lam = W.curved_plate(n_el=3, degree=3, repeats=1)
    lam.C21 = lam.C21 * scale
    got = gpu_matrix(L, lam, "split")
    assert_parity(got, O.assemble(lam))


def test_lagrange_plate_full_size_sampled(L):
    """Lagrange Q2 96x96, 64 plies (2.73e9 stored entries, int64 row pointers):
    sampled blocks against the oracle's block integrator and symmetry; the
    pattern's construction is checked whole on the other plates."""
    _sampled_parity(L, W.lagrange_plate(), "split", n_rows=40, whole_pattern=False)


def test_split_on_a_side_stream_and_in_a_cuda_graph(L):
    """lam_assemble_split is stream-ordered (K-b runs on a stream forked from the
    caller's and joined back): on a non-default stream after an angle update,
    and captured into a CUDA graph and replayed, it gives the oracle's matrix."""
    import torch
    lam = W.curved_plate(n_el=4, degree=3, repeats=1)
    p = L.Plan.from_laminate(lam)
    side = torch.cuda.Stream()
    out = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(side):
        p.assemble_split(out)                       # warm: device tables, workspace
        new = np.deg2rad(np.linspace(-60.0, 75.0, len(lam.ply_angle)))
        p.update(ply_angle=new)
        p.assemble_split(out)
    side.synchronize()
    lam.ply_angle = new
    ref = O.assemble(lam)
    assert np.abs(out.cpu().numpy() - ref[2]).max() <= TOL * np.abs(ref[2]).max()
    g = torch.cuda.CUDAGraph()
    graph_out = torch.full((p.nnz,), np.nan, dtype=torch.float64, device="cuda")
    with torch.cuda.graph(g):
        p.assemble_split(graph_out)
    graph_out.fill_(np.nan)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(graph_out.cpu().numpy(), out.cpu().numpy())
    p.close()
