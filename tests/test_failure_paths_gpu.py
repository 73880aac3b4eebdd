"""Failure paths of the device calls (GPU required; no device fault).

A failed device allocation is injected on the host: with LAM_FAIL_ALLOC=n in
the environment the library's n-th device allocation (counted from the moment
the variable took that value) fails as an out-of-memory cudaMalloc would. For
every device call and every allocation that call makes on a fresh plan, the
call must return LAM_ERR_OOM, and once the injection is off the same plan must
assemble the same matrix, bit for bit, as a plan that never failed.
"""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
LAM_ERR_INVALID_ARG = 1
LAM_ERR_OOM = 3


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


def _calls(L):
    import torch

    def adjoint(p):
        g = torch.ones(p.nnz, dtype=torch.float64, device="cuda")
        return torch.cat([x.flatten() for x in p.adjoint(values=g, want_dD=False) if x is not None])

    return {
        "pattern": lambda p: torch.cat([x.double() for x in p.pattern()]),
        "split": lambda p: p.assemble_split(),
        "split_double_float": None,  # the same call on a plan with the opt-in arithmetic
        "standard": lambda p: p.assemble_standard(),
        "split_host": lambda p: torch.from_numpy(p.assemble_split_host()),
        "adjoint": adjoint,
        "inplane_operators": lambda p: p.inplane_operators(0).flatten(),
    }


@pytest.mark.parametrize("name", ["pattern", "split", "split_double_float", "standard", "split_host", "adjoint",
                                  "inplane_operators"])
def test_every_allocation_failure_returns_oom_and_the_plan_recovers(L, name):
    import torch
    lam = W.curved_plate(n_el=3, degree=3, repeats=1)
    arith = L.ARITH_DOUBLE_FLOAT if name == "split_double_float" else L.ARITH_FP64
    call = _calls(L)["split" if name == "split_double_float" else name]
    clean = L.Plan.from_laminate(lam, arith=arith)
    ref = call(clean).cpu().numpy()
    clean.close()
    failures = 0
    for n in range(1, 400):
        p = L.Plan.from_laminate(lam, arith=arith)
        os.environ["LAM_FAIL_ALLOC"] = str(n)
        try:
            try:
                call(p)
                torch.cuda.synchronize()
                ok = True
            except L.LamError as e:
                assert e.status == LAM_ERR_OOM, (n, str(e))
                ok = False
        finally:
            del os.environ["LAM_FAIL_ALLOC"]
        if ok:
            p.close()
            break
        failures += 1
        got = call(p).cpu().numpy()     # the same plan, injection off
        torch.cuda.synchronize()
        assert np.array_equal(got, ref), f"allocation {n}: the plan gives a different result after the failure"
        p.close()
    else:
        pytest.fail("the call kept failing after 400 injected allocation failures")
    assert failures >= 1


def test_batch_creation_allocation_failure(L):
    """lam_batch_create: an injected failure returns LAM_ERR_OOM, releases the
    batch's memory, and a batch created afterwards matches the plans alone."""
    import torch
    lams = [W.curved_plate(n_el=3, degree=3, repeats=1), W.cross_ply_plate(n_el=4, n_plies=3)]
    plans = [L.Plan.from_laminate(x) for x in lams]
    refs = [p.assemble_split().cpu().numpy() for p in plans]
    failures = 0
    for n in range(1, 200):
        os.environ["LAM_FAIL_ALLOC"] = str(n)
        try:
            b = L.Batch(plans)
        except L.LamError as e:
            assert e.status == LAM_ERR_OOM, str(e)
            failures += 1
            continue
        finally:
            del os.environ["LAM_FAIL_ALLOC"]
        vals = [torch.empty(p.nnz, dtype=torch.float64, device="cuda") for p in plans]
        b.assemble(vals)
        torch.cuda.synchronize()
        # the plans carry the chunk depth the batch chose: bit for bit against their own assembly,
        # and within rounding of the matrices they gave before
        for p, v, r in zip(plans, vals, refs):
            own = p.assemble_split().cpu().numpy()
            assert np.array_equal(v.cpu().numpy(), own)
            assert np.abs(own - r).max() <= 1e-13 * np.abs(r).max()
        b.close()
        break
    assert failures >= 1
    for p in plans:
        p.close()


def test_batch_tuning_allocation_failure(L):
    """A failed allocation while the first lam_batch_assemble tunes (the plans'
    tables are re-uploaded per chunk depth) returns LAM_ERR_OOM; the batch then
    refuses every call (its launch tables may point at released plan tables),
    and a batch created anew from the same plans matches them."""
    import torch
    rng = np.random.default_rng(5)
    lams = [W.laminate("uneven", W.BSPLINE, 2, 4, list(rng.choice([0.0, 45.0, 90.0], 9)),
                       rng.uniform(0.0005, 0.002, 9)),
            W.cross_ply_plate(n_el=4, n_plies=3)]
    plans = [L.Plan.from_laminate(x) for x in lams]
    vals = [torch.empty(p.nnz, dtype=torch.float64, device="cuda") for p in plans]
    b = L.Batch(plans)
    os.environ["LAM_FAIL_ALLOC"] = "1"
    try:
        with pytest.raises(L.LamError) as e:
            b.assemble(vals)
        assert e.value.status == LAM_ERR_OOM, str(e.value)
    finally:
        del os.environ["LAM_FAIL_ALLOC"]
    torch.cuda.synchronize()
    with pytest.raises(L.LamError) as e:
        b.assemble(vals)
    assert e.value.status == LAM_ERR_INVALID_ARG and "recreate" in str(e.value)
    b.close()
    b = L.Batch(plans)
    b.assemble(vals)
    torch.cuda.synchronize()
    for p, v in zip(plans, vals):
        assert np.array_equal(v.cpu().numpy(), p.assemble_split().cpu().numpy())
    b.close()
    for p in plans:
        p.close()
