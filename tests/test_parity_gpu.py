"""Parity of the CUDA assembly paths with the CPU oracle (GPU required).

Bar: the sparsity pattern is bit-exact, and the values agree to
max|K_gpu - K_oracle| <= 1e-12 * max|K_oracle| (the paper states that the
split and the standard matrices agree to machine precision, Section 3 after
Eq. Q and Section 4). The split path runs in both arithmetics of
lam_options.arith: FP64 (the default: every product and sum an FP64
operation) and the opt-in double-float form; on the GPU the FP64 split and the
FP64 standard matrices agree to 1e-14 of max|K|. Small cases are compared
element by element over the whole matrix; the full-size workloads, in the
launch configuration bench.py times, are compared on the whole pattern, on
sampled blocks that the oracle integrates one by one, and on every entry of
whole in-plane rows (all thickness rows and chunks), plus symmetry.
"""
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
ARITH = {"fp64": 0, "double_float": 1}


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


def gpu_matrix(L, lam, path="split", class_tol=-1.0, arith="fp64"):
    import torch
    p = L.Plan.from_laminate(lam, class_tol=class_tol, arith=ARITH[arith])
    assert p.info["arith"] == ARITH[arith]
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
@pytest.mark.parametrize("path,arith", [("split", "fp64"), ("split", "double_float"), ("standard", "fp64")])
def test_small_full_parity(L, name, path, arith):
    lam = SMALL[name]()
    assert_parity(gpu_matrix(L, lam, path, arith=arith), O.assemble(lam))


def test_nurbs_parity(L):
    lam = W.curved_plate(n_el=4, degree=2, repeats=1)
    lam.weights = np.random.default_rng(7).uniform(0.5, 2.0, lam.n_s)
    ref = O.assemble(lam)
    for path, arith in (("split", "fp64"), ("split", "double_float"), ("standard", "fp64")):
        assert_parity(gpu_matrix(L, lam, path, arith=arith), ref)


def test_fully_anisotropic_materials(L):
    """Triclinic constants: every coupling of D is nonzero (general combine)."""
    rng = np.random.default_rng(11)
    lam = W.laminate("tri", W.BSPLINE, 2, 3, [0, 20, -35, 90], 0.01, mapping=W.curved_map(),
                     materials=np.array([W.random_C21(rng), W.random_C21(rng)]), ply_material=[0, 1, 1, 0])
    p = L.Plan.from_laminate(lam)
    assert p.info["monoclinic"] == 0
    ref = O.assemble(lam)
    for path, arith in (("split", "fp64"), ("split", "double_float"), ("standard", "fp64")):
        assert_parity(gpu_matrix(L, lam, path, arith=arith), ref)


def test_exact_classes_and_merged_classes_agree(L):
    lam = W.curved_plate(n_el=3, degree=3, repeats=1)
    a = gpu_matrix(L, lam, "split", class_tol=0.0)
    b = gpu_matrix(L, lam, "split")
    assert np.abs(a[2] - b[2]).max() <= 1e-14 * np.abs(a[2]).max()


@pytest.mark.parametrize("arith,bar", [("fp64", 1e-14), ("double_float", 2e-13)])
def test_split_equals_standard_on_gpu(L, arith, bar):
    """Both matrices of the GPU, FP64 split against FP64 standard: they sum the
    same integrals in different orders and agree to 1e-14 of max|K| (machine
    precision, Section 3 after Eq. Q). The opt-in double-float split (about
    2^-44 per term) stays within 2e-13."""
    lam = W.curved_plate(n_el=6, degree=3, repeats=2)
    s = gpu_matrix(L, lam, "split", arith=arith)
    t = gpu_matrix(L, lam, "standard")
    assert np.array_equal(s[1], t[1])
    assert np.abs(s[2] - t[2]).max() <= bar * np.abs(t[2]).max()


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
def test_host_output_path_matches_device_path(L, arith):
    import torch
    lam = W.curved_plate(n_el=8, degree=3, repeats=1)
    p = L.Plan.from_laminate(lam, arith=ARITH[arith])
    d = p.assemble_split()
    torch.cuda.synchronize()
    h = np.empty(p.nnz)
    pinned = torch.empty(p.nnz, dtype=torch.float64, pin_memory=True)
    p.assemble_split_host(pinned)
    p.assemble_split_host(h)
    assert np.array_equal(d.cpu().numpy(), h)
    assert np.array_equal(pinned.numpy(), h)
    p.close()


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
def test_repeated_calls_are_bitwise_stable(L, arith):
    import torch
    lam = W.curved_plate(n_el=5, degree=3, repeats=1)
    p = L.Plan.from_laminate(lam, arith=ARITH[arith])
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


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
def test_chunked_host_output_uneven_plies(L, arith):
    lam = _uneven(np.array([W.ply_C21()]), 23)
    p = L.Plan.from_laminate(lam, arith=ARITH[arith])
    import torch
    d = p.assemble_split()
    torch.cuda.synchronize()
    h = np.empty(p.nnz)
    p.assemble_split_host(h)
    assert np.array_equal(d.cpu().numpy(), h)
    p.close()


# ---------------------------------------------------------------- scale robustness (the double-float steps above all)
@pytest.mark.parametrize("arith", ["fp64", "double_float"])
@pytest.mark.parametrize("scale", [2.0 ** -90, 2.0 ** 90])
def test_extreme_geometry_scale(L, scale, arith):
    """In-plane coordinates scaled by 2^+-90: entries of K then span ~2^360.
    Double-float: K-a's per-element power-of-two scaling keeps its float pairs
    in range, the largest entries overflow float in the combine (2^90) and the
    FP64 pass recomputes. FP64: nothing to rescale."""
    curved = W.curved_map(0.04)
    lam = W.laminate("geom", W.BSPLINE, 2, 3, [0, 45, 90], 0.01,
                     mapping=lambda xi, eta: tuple(scale * c for c in curved(xi, eta)))
    assert_parity(gpu_matrix(L, lam, "split", arith=arith), O.assemble(lam))


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
@pytest.mark.parametrize("scale", [2.0 ** -200, 2.0 ** 200])
def test_extreme_material_scale(L, scale, arith):
    """Constants scaled by 2^+-200: every entry of K is beyond float range (the
    double-float combine flags it and the FP64 pass recomputes)."""
    lam = W.curved_plate(n_el=3, degree=3, repeats=1)
    lam.C21 = lam.C21 * scale
    got = gpu_matrix(L, lam, "split", arith=arith)
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


# ---------------------------------------------------------------- the paper's own discretisation (Section 4)
# One element of degree p through the whole thickness, cut into m layers (the
# paper's experiment: Pagano material, p = 1..4, 0/90/... and 0/45/-45/90/...
# stacks), 3 x 3 in-plane elements; p = 4 at m = 64 on one in-plane element (its
# oracle is the slowest: 64 pieces of 125 Gauss points per element) and on
# 4 x 4 elements, whose rows of 64 in-plane neighbours take the class-major combine.
SWEEP = ([(p, m, 3, "cross") for p in (1, 2, 3) for m in (1, 2, 8, 64)] + [(4, m, 3, "cross") for m in (1, 2, 8)]
         + [(4, 64, 1, "cross"), (4, 2, 4, "cross"), (2, 8, 3, "quasi"), (3, 64, 3, "quasi")])


def _sweep_reference(case):
    """The oracle's matrix of one sweep point (runs in a spawned worker)."""
    import oracle as O_
    import workloads as W_
    p, m, n, stack = case
    return O_.assemble(W_.pagano_sweep_plate(p, n, m, stack))


@pytest.fixture(scope="module")
def sweep_references():
    """Every sweep point's oracle matrix, computed by a pool of spawned
    processes (no fork after the CUDA context exists) while the GPU tests run."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    ex = ProcessPoolExecutor(max_workers=max(1, min(len(SWEEP), os.cpu_count() or 1)),
                             mp_context=mp.get_context("spawn"))
    futures = {case: ex.submit(_sweep_reference, case) for case in SWEEP}
    yield futures
    ex.shutdown(cancel_futures=True)


@pytest.mark.parametrize("case", SWEEP, ids=[f"p{p}_m{m}_{n}x{n}_{s}" for p, m, n, s in SWEEP])
def test_pagano_sweep_parity(L, sweep_references, case):
    p, m, n, stack = case
    lam = W.pagano_sweep_plate(p, n, m, stack)
    plan = L.Plan.from_laminate(lam)
    assert plan.info["n_pieces"] == m  # one thickness element cut into m pieces
    if n >= 4 and p == 4:
        assert plan.info["combine_streaming"] == 0
    plan.close()
    ref = sweep_references[case].result()
    for path, arith in (("split", "fp64"), ("split", "double_float"), ("standard", "fp64")):
        assert_parity(gpu_matrix(L, lam, path, arith=arith), ref)


# ---------------------------------------------------------------- whole in-plane rows at full size
def _rows_to_check(lam, extra_seed=0):
    """Eight or more in-plane rows: the four corners, edge midpoints, the centre
    and two seeded interior rows."""
    nx = O.n_functions(lam.u.kind, lam.u.degree, lam.u.knots)
    ny = O.n_functions(lam.v.kind, lam.v.degree, lam.v.knots)
    ns = nx * ny
    rng = np.random.default_rng(100 + extra_seed)
    rows = {0, nx - 1, ns - nx, ns - 1, nx // 2, (ny // 2) * nx, (ny // 2) * nx + nx // 2, (ny - 1) * nx + nx // 3}
    rows.update(int(r) for r in rng.integers(0, ns, 2))
    return sorted(rows)


def _row_references(lam, rows):
    """The oracle's blocks of each row, on host threads (the C call releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    prob = O.Problem(lam)
    ex = ThreadPoolExecutor(max(1, min(len(rows), os.cpu_count() or 1)))
    return ex, {i_s: ex.submit(O.inplane_row_blocks, lam, i_s, prob) for i_s in rows}


def _check_rows(lam, row_ptr, col, vals, refs):
    """Every stored entry of the CSR rows (i_t, i_s, c), all i_t and c, of each
    row i_s against the oracle's blocks, and every oracle block of those rows
    that the pattern does not store is zero (the pattern misses nothing)."""
    import torch
    nx = O.n_functions(lam.u.kind, lam.u.degree, lam.u.knots)
    ny = O.n_functions(lam.v.kind, lam.v.degree, lam.v.knots)
    nt = O.n_functions(lam.t.kind, lam.t.degree, lam.t.knots)
    ns = nx * ny
    rp = row_ptr.cpu().numpy()
    scale = float(vals.abs().max())
    assert np.isfinite(scale) and scale > 0
    worst = 0.0
    for i_s, fut in refs.items():
        bx0, by0, B = fut.result()
        B = B.copy()
        rows = (3 * (np.arange(nt)[:, None] * ns + i_s) + np.arange(3)[None, :]).ravel()
        lens = rp[rows + 1] - rp[rows]
        idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
        it_c = np.repeat(np.arange(len(rows)), lens)
        it, c = it_c // 3, it_c % 3
        t_idx = torch.from_numpy(idx).to(vals.device)
        v = vals[t_idx].cpu().numpy()
        cc = col[t_idx].cpu().numpy().astype(np.int64)
        j, d = cc // 3, cc % 3
        jt, js = j // ns, j % ns
        jy, jx = js // nx, js % nx
        assert np.all((jx - bx0 >= 0) & (jx - bx0 < B.shape[3]) & (jy - by0 >= 0) & (jy - by0 < B.shape[2]))
        ref = B[it, jt, jy - by0, jx - bx0, c, d]
        worst = max(worst, float(np.abs(v - ref).max()))
        B[it, jt, jy - by0, jx - bx0, c, d] = 0.0
        assert np.abs(B).max() <= 1e-14 * scale, f"row {i_s}: an oracle block outside the pattern"
    assert worst <= TOL * scale, worst / scale
    return worst / scale


@pytest.mark.parametrize("arith", ["fp64", "double_float"])
def test_curved_plate_full_size_whole_rows(L, arith):
    """The benchmark workload (cubic, 64x64 curved, 48 plies) as bench.py
    launches it: every entry of ten in-plane rows, all 97 thickness rows."""
    import torch
    lam = W.curved_plate()
    ex, refs = _row_references(lam, _rows_to_check(lam))
    p = L.Plan.from_laminate(lam, arith=ARITH[arith])
    row_ptr, col = p.pattern()
    vals = p.assemble_split()
    torch.cuda.synchronize()
    _check_rows(lam, row_ptr, col, vals, refs)
    ex.shutdown()
    p.close()


def test_lagrange_plate_full_size_whole_rows(L):
    """Lagrange Q2 96x96, 64 plies (2.73e9 entries, int64 row pointers): every
    entry of ten in-plane rows, all 129 thickness rows."""
    import torch
    lam = W.lagrange_plate()
    ex, refs = _row_references(lam, _rows_to_check(lam, 1))
    p = L.Plan.from_laminate(lam)
    row_ptr, col = p.pattern()
    vals = p.assemble_split()
    torch.cuda.synchronize()
    _check_rows(lam, row_ptr, col, vals, refs)
    ex.shutdown()
    p.close()
    del vals, col, row_ptr
    torch.cuda.empty_cache()


def test_curved_shell_full_size_whole_rows(L):
    """The curved shell (general extrusion) at the benchmark's size."""
    import torch
    lam = W.shell_plate()
    ex, refs = _row_references(lam, _rows_to_check(lam, 2))
    p = L.Plan.from_laminate(lam)
    row_ptr, col = p.pattern()
    vals = p.assemble_split()
    torch.cuda.synchronize()
    _check_rows(lam, row_ptr, col, vals, refs)
    ex.shutdown()
    p.close()


def test_batch_uneven_instances_whole_rows(L):
    """Three uneven-ply instances of the 256-laminate batch recipe (12, 8 and 3
    thickness chunks) assembled by one lam_batch_assemble: whole rows of each."""
    import torch
    lams = [W.batch_laminates()[k] for k in (0, 2, 3)]
    plans = [L.Plan.from_laminate(x) for x in lams]
    assert [p.info["combine_chunks"] for p in plans] == [12, 8, 3]
    refs = [_row_references(x, _rows_to_check(x, 3 + k)) for k, x in enumerate(lams)]
    values = [torch.empty(p.nnz, dtype=torch.float64, device="cuda") for p in plans]
    b = L.Batch(plans)
    b.assemble(values)
    b.assemble(values)  # the replayed graph
    torch.cuda.synchronize()
    for x, p, v, (ex, r) in zip(lams, plans, values, refs):
        row_ptr, col = p.pattern()
        _check_rows(x, row_ptr, col, v, r)
        ex.shutdown()
    b.close()
    for p in plans:
        p.close()
