"""lam_batch_*: many laminates assembled together (GPU required).

Every instance of a batch must equal, bit for bit, the same plan assembled on
its own (the batch runs the same arithmetic: Eq. Q per instance, Gram blocks
per distinct mesh, the streaming combine per in-plane row); two instances are
also checked against the oracle.
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


def mixed_laminates():
    rng = np.random.default_rng(17)
    cubic = lambda angles, h, **kw: W.laminate("cubic", W.BSPLINE, 3, 3, angles, h, mapping=W.curved_map(), **kw)
    quad = lambda angles, h, **kw: W.laminate("quad", W.BSPLINE, 2, 5, angles, h, n_el_y=4, **kw)
    tri = np.array([W.random_C21(rng), W.ply_C21()])
    return [
        cubic([0, 45, -45, 90], 0.002),
        cubic(list(rng.choice([0.0, 45.0, 90.0], 7)), rng.uniform(0.0005, 0.002, 7)),          # uneven plies
        cubic([0, 30, 90], 0.003, materials=tri, ply_material=[0, 1, 0]),                         # triclinic
        quad([0, 90, 0, 90], 0.0025),
        quad(list(rng.choice([0.0, -45.0, 45.0], 9)), rng.uniform(0.0005, 0.002, 9),
             materials=np.array([W.ply_C21() * (1 + 0.25 * k) for k in range(3)]),
             ply_material=list(rng.integers(0, 3, 9))),
        quad([45, -45], 0.004),
        W.laminate("quartic", W.BSPLINE, 4, 5, [0, 45], 0.02, mapping=W.curved_map(), n_el_y=4,
                   thickness_degree=1),                                                            # class-major
        W.laminate("one_elem", W.BSPLINE, 3, 3, [0, 90, 0], [0.1, 0.2, 0.1], mapping=W.curved_map(),
                   thickness=W.single_element_thickness(0.4, 3)),
    ]


def test_batch_equals_single_plans_bitwise(L):
    import torch
    lams = mixed_laminates()
    plans = [L.Plan.from_laminate(l) for l in lams]
    ref = []
    for p in plans:
        ref.append(p.assemble_split().cpu().numpy())
    b = L.Batch(plans)
    info = b.info
    assert info["n_plans"] == len(plans) and info["n_meshes"] == 3  # cubic (4 stacks), quadratic, quartic
    assert info["n_persistent"] == len(plans) - 1  # the quartic rows take the class-major form
    out = b.assemble()
    torch.cuda.synchronize()
    info = b.info
    assert info["graph"] == 1 and 1 <= info["ctas_per_sm"] <= 4
    assert info["chunk_ctas"] in (4, 3, 2) and info["rows_per_item"] in (1, 2, 4)
    assert sum(t > 0 for t in info["tuned_ms"]) >= 9  # three chunk depths x three row blocks at least
    # the plans now carry the chunk depth the batch chose: their own assembly gives the batch's bits
    own = [p.assemble_split().cpu().numpy() for p in plans]
    for k in range(len(plans)):
        assert np.array_equal(out[k].cpu().numpy(), own[k]), k
    # regrouping the thickness rows moves only rounding (slices shared between pairs whose Q agree up to
    # rounding take the first pair's Q of the chunk)
    for k in range(len(plans)):
        assert np.abs(own[k] - ref[k]).max() <= 1e-13 * np.abs(ref[k]).max(), k
    ref = own
    # replay into fresh buffers (the value pointers change)
    out2 = b.assemble([torch.full((p.nnz,), np.nan, dtype=torch.float64, device="cuda") for p in plans])
    torch.cuda.synchronize()
    for k in range(len(plans)):
        assert np.array_equal(out2[k].cpu().numpy(), ref[k]), k
    # and against the oracle, for an uneven stack and the triclinic one
    for k in (1, 2):
        rp, col, val = O.assemble(lams[k])
        err = np.abs(out2[k].cpu().numpy() - val).max() / np.abs(val).max()
        assert err <= 1e-12
    b.close()


def test_batch_refuses_updated_plans(L):
    import torch
    lams = mixed_laminates()[:2]
    plans = [L.Plan.from_laminate(l) for l in lams]
    b = L.Batch(plans)
    b.assemble()
    plans[0].update(ply_angle=np.zeros(4))
    with pytest.raises(L.LamError) as e:
        b.assemble()
    assert e.value.status == 1
    b.close()


def test_batch_of_seeded_laminates(L):
    """The first 24 laminates of the seeded batch workload (uneven ply counts,
    thicknesses and materials on four meshes), bit for bit against their plans."""
    import torch
    lams = W.batch_laminates()[:24]
    plans = [L.Plan.from_laminate(l) for l in lams]
    b = L.Batch(plans)
    out = b.assemble()
    torch.cuda.synchronize()
    assert b.info["n_meshes"] == len({(len(l.u.knots)) for l in lams})
    buf = torch.empty(max(p.nnz for p in plans), dtype=torch.float64, device="cuda")
    for k, p in enumerate(plans):
        v = buf[:p.nnz]
        p.assemble_split(v)
        torch.cuda.synchronize()
        assert torch.equal(v, out[k]), k
    b.close()


def test_batch_with_general_extrusions(L):
    """Shells (general extrusion maps) in a batch: assembled one by one after the
    persistent launch, outside the mesh groups even when they share a plate's
    in-plane discretisation; bit for bit against their own plans and against
    the oracle."""
    import torch
    plate = W.curved_plate(n_el=3, degree=3, repeats=1)
    shell_same_mesh = W.shell_plate(n_el=3, degree=3, repeats=1)        # the plate's knots, lifted and tilted
    shell_other = W.laminate("sh", W.BSPLINE, 2, 4, [0, 45, 90], 0.004, mapping=W.bump_map(0.1), n_el_y=3,
                             extrusion=(0.1, -0.2, 1.0))
    lams = [plate, shell_same_mesh, shell_other]
    plans = [L.Plan.from_laminate(l) for l in lams]
    ref = [p.assemble_split().cpu().numpy() for p in plans]
    b = L.Batch(plans)
    info = b.info
    assert info["n_meshes"] == 1 and info["n_persistent"] == 1
    out = b.assemble()
    torch.cuda.synchronize()
    for k in range(len(plans)):
        assert np.array_equal(out[k].cpu().numpy(), ref[k]), k
    for k in (1, 2):
        rp, col, val = O.assemble(lams[k])
        assert np.abs(out[k].cpu().numpy() - val).max() <= 1e-12 * np.abs(val).max()
    b.close()
