"""lam_inplane_operators: Eq. P from the Gram blocks of the split path and by
Appendix A's Voigt-free construction (GPU required). The two must agree to
rounding, and both must match the oracle's Eq. P on sampled in-plane pairs."""
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


def _nurbs():
    lam = W.curved_plate(n_el=4, degree=3, repeats=1)
    lam.weights = np.random.default_rng(7).uniform(0.5, 2.0, lam.n_s)
    return lam


CASES = {
    "curved_nurbs_cubic": _nurbs,
    "lagrange_q2": lambda: W.lagrange_plate(n_el=3, n_plies=4),
    "triclinic_quadratic": lambda: W.laminate(
        "tri", W.BSPLINE, 2, 3, [0, 20, -35, 90], 0.01, mapping=W.curved_map(), n_el_y=4,
        materials=np.array([W.random_C21(np.random.default_rng(11)), W.random_C21(np.random.default_rng(12))]),
        ply_material=[0, 1, 1, 0]),
    "quartic": lambda: W.laminate("p4", W.BSPLINE, 4, 3, [30, -60], 0.02, mapping=W.curved_map(), thickness_degree=1),
}


def inplane_pairs(lam):
    """(i_s, j_s) of every in-plane pair in the library's order, from the 3D pattern's first thickness row."""
    rp, col = O.pattern(lam)
    ns = lam.n_s
    out = []
    for i_s in range(ns):
        cols = col[rp[3 * i_s]:rp[3 * i_s + 1]:3] // 3
        out += [(i_s, int(j)) for j in cols if j < ns]
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_two_constructions_agree_and_match_the_oracle(L, name):
    import torch
    lam = CASES[name]()
    p = L.Plan.from_laminate(lam)
    pairs = inplane_pairs(lam)
    assert len(pairs) == p.info["nnz_inplane"]
    prob = O.Problem(lam)
    rng = np.random.default_rng(1)
    for ply in sorted({0, len(lam.ply_angle) - 1}):
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
