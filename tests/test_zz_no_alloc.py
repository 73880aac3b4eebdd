"""The split assembly that allocates nothing (lam_assemble_split_noalloc).

Some callers cannot call cudaMalloc: a host application whose device memory
all comes from its own pool, or code that must not grow the device footprint
while it runs. For them the library offers a variant of the split assembly
whose tables and workspace live in one fixed static device array. These tests
call it through the C ABI and check that it reproduces lam_assemble_split on
two calls in a row (the array keeps the previous call's contents, so the
second call checks that it is reset correctly), and that plans too large for
the array are refused. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("the gpu tests need a CUDA device")
    from paper_1905_05417_gb300 import build
    build.build()
    import paper_1905_05417_gb300 as L
    return L


def _noalloc(L, plan, out):
    import torch
    status = L.load().lam_assemble_split_noalloc(plan.handle, ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return status


@pytest.mark.parametrize("make", [
    lambda: W.curved_plate(n_el=20, degree=3, repeats=2),
    lambda: W.laminate("tri", W.BSPLINE, 2, 6, [0, 20, -35, 90], 0.01, mapping=W.curved_map(),
                       materials=np.array([W.random_C21(np.random.default_rng(3))]), ply_material=[0, 0, 0, 0]),
])
def test_noalloc_matches_split_on_two_calls(lib, make):
    import torch
    lam = make()
    plan = lib.Plan.from_laminate(lam)
    ref = plan.assemble_split()
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    out = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        assert _noalloc(lib, plan, out) == 0, lib.last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}: values left unwritten"
        err = np.abs(got - ref).max() / scale
        assert err <= TOL, f"call {call}: max rel error {err:.3e}"
    plan.close()


def test_noalloc_on_the_benchmark_plate(lib):
    """The 64x64 cubic 48-ply plate fits in the static array; two calls in a
    row agree with lam_assemble_split and, bit for bit, with each other."""
    import torch
    plan = lib.Plan.from_laminate(W.curved_plate())
    ref = plan.assemble_split()
    scale = ref.abs().max().item()
    out = torch.empty_like(ref)
    prev = None
    for _ in range(2):
        out.zero_()
        assert _noalloc(lib, plan, out) == 0, lib.last_error()
        torch.cuda.synchronize()
        assert (out - ref).abs().max().item() <= TOL * scale
        if prev is not None:
            assert torch.equal(out, prev)
        prev = out.clone()
    plan.close()


def test_noalloc_rejects_plans_beyond_the_array(lib):
    """A plan whose workspace exceeds the static array (a quadratic 140x140
    in-plane mesh: about 35 MB of assembled in-plane Gram blocks) but whose
    matrix is small (one linear ply, 17.6 M entries): the call is refused with
    LAM_ERR_UNSUPPORTED before any device work, and the caller's full-size
    buffer is left untouched."""
    import re
    import torch
    lam = W.laminate("wide", W.BSPLINE, 2, 140, [0.0], 0.01, thickness_degree=1)
    plan = lib.Plan.from_laminate(lam)
    out = torch.full((plan.nnz,), float("nan"), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, plan, out) == 2              # LAM_ERR_UNSUPPORTED
    msg = lib.last_error()
    m = re.search(r"needs (\d+) bytes of scratch, the static array holds (\d+)", msg)
    assert m and int(m.group(1)) > int(m.group(2)) == 32 << 20, msg
    torch.cuda.synchronize()
    assert torch.isnan(out).all()                     # nothing was written
    plan.close()
