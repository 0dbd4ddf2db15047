"""Adaptive refinement with the geometric mapping of the volume fraction
(Sec. 3, Alg. 2).

CPU: the cell map of two octrees against a brute-force box overlap, and the
oracle's mapping against what fixes it -- conservation of the phase volume,
the identity on the same mesh, and exactness for a planar interface (the new
cells' fractions equal the closed-form cut-box volumes).  GPU: vof_remap
against the oracle cell by cell, and the deformation case on a re-refined
octree (conservation across every remap, boundedness).
"""
import itertools

import numpy as np
import pytest

from paper_1305_3417_gb300 import amr
from paper_1305_3417_gb300 import inputs as I


def boxes(m):
    o = m.octree["origin"].astype(float)
    return o, o + m.octree["size"][:, None]


def plane_fraction_of_box(lo, hi, n, d):
    """|box ^ {n.x <= d}| / |box| by inclusion-exclusion over the corners
    (Scardovelli & Zaleski 2000), in the box's unit-cube coordinates."""
    h = hi - lo
    nn = n * h
    dd = d - n @ lo
    dd -= nn[nn < 0].sum()
    nn = np.abs(nn)
    if np.any(nn < 1e-12):
        raise ValueError("axis-parallel plane")
    s = 0.0
    for v in itertools.product((0, 1), repeat=3):
        s += (-1) ** sum(v) * max(0.0, dd - nn @ np.array(v, float)) ** 3
    return min(max(s / (6 * nn.prod()), 0.0), 1.0)


@pytest.fixture(scope="module")
def meshes():
    m0 = I.octree_mesh(8, 2, (0.35, 0.35, 0.35), 0.15)
    a0 = I.sampled_fraction(m0, I.sphere_sdf((0.4, 0.37, 0.33), 0.15))
    m1 = amr.refine_near_interface(m0, a0, 3.0)
    return m0, a0, m1


def test_cell_pairs_match_box_overlap(meshes):
    m0, a0, m1 = meshes
    assert m1.n_cells != m0.n_cells
    for dst, src in ((m1, m0), (m0, m1)):
        ptr, s = amr.cell_pairs(dst, src)
        lo1, hi1 = boxes(dst)
        lo0, hi0 = boxes(src)
        ov = np.all(np.minimum(hi1[:, None, :], hi0[None, :, :]) > np.maximum(lo1[:, None, :], lo0[None, :, :]), 2)
        bd, bs = np.nonzero(ov)
        ref = np.zeros(dst.n_cells + 1, int)
        np.add.at(ref, bd + 1, 1)
        assert np.array_equal(np.cumsum(ref), ptr) and np.array_equal(bs, s)
        # nested: every pair is one box inside the other
        for c in range(0, dst.n_cells, 7):
            for q in range(ptr[c], ptr[c + 1]):
                a_in_b = np.all(lo1[c] >= lo0[s[q]]) and np.all(hi1[c] <= hi0[s[q]])
                b_in_a = np.all(lo0[s[q]] >= lo1[c]) and np.all(hi0[s[q]] <= hi1[c])
                assert a_in_b or b_in_a


def test_refinement_follows_the_interface(meshes):
    m0, a0, m1 = meshes
    N = m1.octree["N"]
    lv1 = m1.octree["level"]
    cc = (m1.octree["origin"] + 0.5 * m1.octree["size"][:, None]) / N
    r = np.linalg.norm(cc - np.array([0.4, 0.37, 0.33]), axis=1)
    near = np.abs(r - 0.15) < 0.5 / N
    assert np.all(lv1[near] == m1.octree["levels"])   # cells on the new interface are finest
    assert np.all(lv1[np.abs(r - 0.15) > 0.5] == 0)   # far ones stay coarse
    assert (np.abs(r - 0.15) > 0.5).sum() > 10


def test_remap_conserves_and_is_identity(oracle_lib, meshes):
    m0, a0, m1 = meshes
    om0, om1 = oracle_lib.OracleMesh(m0), oracle_lib.OracleMesh(m1)
    n, d, fl, _, st = om0.reconstruct(a0)
    assert st == 0
    _, v0, _, _ = om0.geometry()
    _, v1, _, _ = om1.geometry()
    ptr, src = amr.cell_pairs(m1, m0)
    a1 = om1.remap_from(om0, a0, n, d, fl, ptr, src)
    assert abs((a1 * v1).sum() - (a0 * v0).sum()) <= 1e-13 * (a0 * v0).sum()
    assert a1.min() >= -1e-14 and a1.max() <= 1 + 1e-14
    # and back: un-refinement sums the finer cells' phase volumes
    n1, d1, fl1, _, _ = om1.reconstruct(a1)
    ptr2, src2 = amr.cell_pairs(m0, m1)
    a2 = om0.remap_from(om1, a1, n1, d1, fl1, ptr2, src2)
    assert abs((a2 * v0).sum() - (a0 * v0).sum()) <= 1e-13 * (a0 * v0).sum()
    ident = om0.remap_from(om0, a0, n, d, fl, np.arange(m0.n_cells + 1), np.arange(m0.n_cells))
    assert np.abs(ident - a0).max() < 1e-15


def test_remap_exact_for_a_plane(oracle_lib, meshes):
    """A planar interface with its exact planes: every new cell's fraction is
    the closed-form fraction of its box below the plane, refined or not."""
    m0, a0, m1 = meshes
    nrm = np.array([0.48, -0.6, 0.64])
    nrm /= np.linalg.norm(nrm)
    dpl = nrm @ np.array([0.52, 0.47, 0.5])
    N = m0.octree["N"]
    lo0, hi0 = boxes(m0)
    a = np.array([plane_fraction_of_box(l / N, h / N, nrm, dpl) for l, h in zip(lo0, hi0)])
    O = oracle_lib
    fl = np.where(a >= 1 - 1e-9, O.FULL, np.where(a > 1e-9, O.INTERFACE | O.ORIENTED, 0)).astype(np.uint8)
    n = np.repeat(nrm[:, None], m0.n_cells, 1)
    d = np.full(m0.n_cells, dpl)
    om0, om1 = O.OracleMesh(m0), O.OracleMesh(m1)
    ptr, src = amr.cell_pairs(m1, m0)
    a1 = om1.remap_from(om0, a, n, d, fl, ptr, src)
    lo1, hi1 = boxes(m1)
    want = np.array([plane_fraction_of_box(l / N, h / N, nrm, dpl) for l, h in zip(lo1, hi1)])
    assert np.abs(a1 - want).max() < 1e-12


# ---------------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3417_gb300 import build
    build.build()
    return torch


@pytest.mark.gpu
def test_remap_matches_oracle(torch, oracle_lib, meshes):
    from paper_1305_3417_gb300 import vof
    m0, a0, m1 = meshes
    c0, c1 = vof.VofContext(m0), vof.VofContext(m1)
    om0, om1 = oracle_lib.OracleMesh(m0), oracle_lib.OracleMesh(m1)
    ta = torch.from_numpy(a0).cuda()
    n, d, fl, _ = c0.reconstruct(ta)
    for dst, src, cd, cs, od, os_, a_src, nn, dd, ff in (
            (m1, m0, c1, c0, om1, om0, ta, n, d, fl),):
        ptr, ps = amr.cell_pairs(dst, src)
        out = torch.zeros(dst.n_cells, dtype=torch.float64, device="cuda")
        vof.vof_remap(cd.h, cs.h, a_src, nn, dd, ff, torch.from_numpy(ptr).cuda(), torch.from_numpy(ps).cuda(), out)
        got = out.cpu().numpy()
        want = od.remap_from(os_, a_src.cpu().numpy(), nn.cpu().numpy(), dd.cpu().numpy(), ff.cpu().numpy(),
                             ptr, ps)
        assert np.abs(got - want).max() < 1e-13
    assert c0.status() == 0 and c1.status() == 0
    c0.close()
    c1.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_amr_deformation_run(torch, precision):
    """The deformation case on an octree re-refined around the interface every
    4 steps to t = T = 3 (8^3 base, two levels, finest h = 1/32): the volume is
    conserved across every step and every remap, alpha stays in [0, 1], and
    the shape error at t = T against the sphere's fractions on the final mesh
    is that of a uniform mesh of the finest size."""
    from paper_1305_3417_gb300 import vof
    case = amr.AmrCase(n0=8, levels=2, band=3.0, precision=precision, every=4)
    v0 = case.volume()
    stats = torch.zeros(vof.S_LEN, dtype=torch.float64, device="cuda")
    worst = 0.0
    while case.t < 3.0 - 1e-12:
        if case.steps and case.steps % case.every == 0:
            case.remap()
        case.step(3.0, stats)
        s = stats.cpu().numpy()
        worst = max(worst, abs(s[1] - s[0]) / s[0])
        assert s[4] >= -1e-12 and s[5] <= 1 + 1e-12
        assert case.ctx.status() == 0
    assert case.remaps >= 50
    assert worst <= 1e-12
    assert max(abs(x) for x in case.mass_change) <= 1e-12
    assert abs(case.volume() / v0 - 1) <= 1e-11
    ex = I.sampled_fraction(case.mesh, I.sphere_sdf(case.center, case.R))
    a = case.alpha.cpu().numpy()
    vc = case.vc.cpu().numpy()
    l1 = float((vc * np.abs(a - ex)).sum())
    print(f"AMR deformation ({'mixed' if precision else 'fp64'}): {case.steps} steps, {case.remaps} remaps, "
          f"{case.mesh.n_cells} cells at t = T, L1 {l1:.4e} ({l1 / (vc * ex).sum():.3e} of the volume), "
          f"worst remap volume change {max(abs(x) for x in case.mass_change):.1e}")
    # the finest cells are those of a uniform 32^3 mesh: the error stays within
    # the paper's E_g for the uniform 32^3 deformation case at Co 0.5
    # (tests/golden/paper_deformation_eg.txt)
    assert l1 <= 8.15757e-3
    case.ctx.close()
