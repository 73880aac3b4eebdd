"""C ABI and host logic of the library, without a GPU.

Checks that liblam.so builds, loads and exports every function include/lam.h
declares; that host-only calls (plan creation, sizes, pattern size query,
update) work and agree with the oracle; and that invalid input is rejected
with a status code rather than a crash.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lam():
    from paper_1905_05417_gb300 import build
    build.build()
    import paper_1905_05417_gb300 as L
    L.load()
    return L


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lam.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lam_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lam_plan_create", "lam_pattern", "lam_assemble_split", "lam_assemble_standard",
                     "lam_plan_destroy", "lam_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lam):
    so = ctypes.CDLL(lam.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    assert set(declared_functions()) == set(lam.SYMBOLS)
    assert "sm_103a" in lam.version()


def test_library_is_built_for_sm103a_only(lam):
    # the build passes exactly one -gencode, for sm_103a
    from paper_1905_05417_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


CASES = [
    W.cross_ply_plate,
    lambda: W.curved_plate(n_el=3, degree=3, repeats=1),
    lambda: W.lagrange_plate(n_el=3, n_plies=4),
    lambda: W.laminate("one_elem", W.BSPLINE, 2, 2, [0, 90, 45], [0.1, 0.2, 0.1],
                       thickness=W.single_element_thickness(0.4, 3)),
    lambda: W.laminate("mixed", W.BSPLINE, 3, 3, [0, 30, 60], 0.01, n_el_y=2, degree_y=2,
                       mapping=W.curved_map(0.03)),
]


@pytest.mark.parametrize("make", CASES)
def test_plan_sizes_match_oracle(lam, make):
    L = make()
    p = lam.Plan.from_laminate(L)
    n_dof, nnz = O.sizes(L)
    assert p.n_dof == n_dof and p.nnz == nnz
    assert lam.pattern(p.handle) == nnz  # size query, host only
    info = p.info
    assert info["n_s"] * info["n_t"] * 3 == n_dof
    assert 9 * info["nnz_inplane"] * info["nnz_thickness"] == nnz
    assert 1 <= info["n_classes"] <= info["nnz_thickness"]


def test_published_sizes(lam):
    """Exact sizes of the named workloads (boundary truncation included)."""
    p = lam.Plan.from_laminate(W.curved_plate())
    assert (p.n_dof, p.nnz) == (1306299, 723661785)
    p = lam.Plan.from_laminate(W.adjoint_plate())
    assert (p.n_dof, p.nnz) == (180075, 94299993)
    p = lam.Plan.from_laminate(W.lagrange_plate())
    assert (p.n_dof, p.nnz) == (14415363, 2730313737)
    assert p.info["n_configs"] == 2


def test_configurations_and_classes(lam):
    p = lam.Plan.from_laminate(W.curved_plate())
    assert p.info["n_configs"] == 4     # 0, 45, -45, 90
    assert p.info["monoclinic"] == 1
    assert p.info["n_classes"] == 31    # distinct Q vectors (exact count of the stack)
    exact = lam.Plan.from_laminate(W.curved_plate(), class_tol=0.0)
    assert exact.info["n_classes"] >= 31
    # a fully anisotropic material is not monoclinic
    L = W.cross_ply_plate()
    L.C21 = W.random_C21(np.random.default_rng(0))[None, :]
    assert lam.Plan.from_laminate(L).info["monoclinic"] == 0


def test_combine_variant_selection(lam):
    info = lam.Plan.from_laminate(W.curved_plate()).info
    assert info["combine_streaming"] == 1 and info["combine_chunks"] == 1  # 31 classes fit at once
    assert lam.Plan.from_laminate(W.cross_ply_plate()).info["combine_streaming"] == 1
    quartic = W.laminate("p4", W.BSPLINE, 4, 8, [0, 45], 0.02, n_el_y=8, thickness_degree=1)
    assert lam.Plan.from_laminate(quartic).info["combine_streaming"] == 0  # 81 neighbours: 729 threads
    rng = np.random.default_rng(5)
    uneven = W.laminate("u", W.BSPLINE, 1, 3, [0.0] * 70, rng.uniform(0.0005, 0.002, 70), thickness_degree=1)
    p = lam.Plan.from_laminate(uneven)
    # hundreds of classes: streamed in chunks of thickness rows
    assert p.info["n_classes"] > 150 and p.info["combine_streaming"] == 1 and p.info["combine_chunks"] >= 2


def test_update_rebuilds_configurations(lam):
    L = W.cross_ply_plate()
    p = lam.Plan.from_laminate(L)
    assert p.info["n_configs"] == 2
    p.update(ply_angle=np.zeros(4))
    assert p.info["n_configs"] == 1
    with pytest.raises(lam.LamError):
        p.update(ply_angle=np.zeros(3))


def _kw(L):
    b = lambda x: (x.kind, x.degree, x.knots)
    return dict(u=b(L.u), v=b(L.v), ctrl=L.ctrl, t=b(L.t), ply_thickness=L.ply_thickness,
                ply_material=L.ply_material, ply_angle=L.ply_angle, C21=L.C21)


@pytest.mark.parametrize("mutate,status", [
    (lambda k: k.update(ply_thickness=k["ply_thickness"] * 1.01), 1),          # plies do not fill the thickness
    (lambda k: k.update(ply_material=np.full(4, 3, np.int32)), 1),             # material out of range
    (lambda k: k.update(u=(0, 0, k["u"][2])), 1),                              # degree 0
    (lambda k: k.update(u=(0, 2, k["u"][2][::-1].copy())), 1),                 # decreasing knots
    (lambda k: k.update(t=(7, 2, k["t"][2])), 1),                              # unknown kind
    (lambda k: k.update(ply_angle=np.array([0, np.nan, 0, 0.0])), 1),          # non-finite angle
    (lambda k: k.update(u=(0, 2, np.array([0, 0, 0.5, 1, 1, 1.0]))), 1),       # not an open knot vector
])
def test_invalid_input_is_rejected(lam, mutate, status):
    kw = _kw(W.cross_ply_plate())
    mutate(kw)
    with pytest.raises(lam.LamError) as e:
        lam.Plan(**kw)
    assert e.value.status == status
    assert lam.last_error() != ""


def test_unsupported_sizes_are_rejected(lam):
    # more DOFs than int32 column indices can address
    L = W.lagrange_plate(n_el=4, n_plies=2)
    kw = _kw(L)
    big = W.Basis1D(W.LAGRANGE, 2, np.linspace(0, 1, 30001))
    kw["u"] = (big.kind, big.degree, big.knots)
    kw["v"] = (big.kind, big.degree, big.knots)
    kw["ctrl"] = np.zeros((big.n_functions ** 2, 2))
    with pytest.raises(lam.LamError) as e:
        lam.Plan(**kw)
    assert e.value.status == 2


def test_device_calls_fail_loudly_without_a_gpu(lam):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = lam.Plan.from_laminate(W.cross_ply_plate())
    with pytest.raises(lam.LamError) as e:
        lam.assemble_split(p.handle, 0x1000, stream=0)
    assert e.value.status in (4, 1)


def test_plan_gauss_and_rotation_via_sizes(lam):
    """nq options are honoured (validation of the option path)."""
    L = W.cross_ply_plate()
    L.nq = (20, 3, 3)
    with pytest.raises(lam.LamError) as e:
        lam.Plan.from_laminate(L)
    assert e.value.status == 2


def test_adjoint_rejects_invalid_cotangents(lam):
    """Argument checks of lam_adjoint run before any device work."""
    p = lam.Plan.from_laminate(W.cross_ply_plate())
    L = lam.load()
    for kind, rank, values, u, v, flags in ((7, 1, 0x1000, None, None, 0),     # unknown kind
                                            (0, 1, None, None, None, 0),       # CSR without values
                                            (1, 0, None, 0x1000, 0x1000, 0),   # rank 0
                                            (1, 1, None, 0x1000, None, 0),     # v missing
                                            (0, 1, 0x1000, None, None, 4)):    # unknown flag
        c = lam._Cotangent()
        c.kind, c.rank, c.values, c.u, c.v, c.flags = kind, rank, values, u, v, flags
        st = L.lam_adjoint(p.handle, ctypes.byref(c), 0x2000, None, None, None)
        assert st == 1, (kind, rank, flags)
        assert "lam_adjoint" in lam.last_error()
    assert L.lam_adjoint(p.handle, None, 0x2000, None, None, None) == 1



def test_batch_rejects_invalid_arguments(lam):
    """Argument checks of lam_batch_create run before any device work."""
    L = lam.load()
    p = lam.Plan.from_laminate(W.cross_ply_plate())
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 2)(p.handle.value, p.handle.value)
    assert L.lam_batch_create(ctypes.byref(out), arr, 2) == 1          # the same plan twice
    assert L.lam_batch_create(ctypes.byref(out), arr, 0) == 1          # no plans
    assert L.lam_batch_create(None, arr, 1) == 1
    assert L.lam_batch_assemble(None, None, None) == 1
    assert L.lam_batch_destroy(None) == 0


def test_extrusion_maps_at_plan_creation(lam):
    """ctrl_dim / extrusion of lam_inplane (Eq. extrusion): the general map is
    recognised, malformed values are rejected, and the entry point that does not
    handle it refuses it before any device work."""
    assert lam.Plan.from_laminate(W.cross_ply_plate()).info["shell"] == 0
    sh = W.shell_plate(n_el=3, degree=2, repeats=1)
    p = lam.Plan.from_laminate(sh)
    assert p.info["shell"] == 1
    assert p.info["nnz"] == lam.Plan.from_laminate(W.curved_plate(n_el=3, degree=2, repeats=1)).info["nnz"]
    # a planar surface with a tilted extrusion is general too; a = e_z or a = 0 is the plate
    kw = _kw(W.cross_ply_plate())
    assert lam.Plan(**kw, extrusion=(0.0, 0.0, 1.0)).info["shell"] == 0
    assert lam.Plan(**kw, extrusion=(0.0, 0.0, 0.0)).info["shell"] == 0
    assert lam.Plan(**kw, extrusion=(0.1, 0.0, 1.0)).info["shell"] == 1
    assert lam.Plan(**dict(kw, ctrl=np.c_[kw["ctrl"], np.zeros(len(kw["ctrl"]))])).info["shell"] == 1
    with pytest.raises(lam.LamError) as e:
        lam.Plan(**kw, extrusion=(np.nan, 0.0, 1.0))
    assert e.value.status == 1
    L = lam.load()
    # the refusal comes before any device work; where a GPU is present the call
    # still gets a real buffer of the plan's size, so a regression could not
    # write through a made-up address
    import torch
    if torch.cuda.is_available():
        buf = torch.empty(p.info["nnz"], dtype=torch.float64, device="cuda")
        assert L.lam_assemble_split_noalloc(p.handle, buf.data_ptr(), None) == 2
    else:
        assert L.lam_assemble_split_noalloc(p.handle, 0x1000, None) == 2
    assert "extrusion" in lam.last_error()
