"""Pins of the oracle on periodic meshes (reading R21 of the paper's periodic
translation case, Sec. 4.2).

What fixes them: a uniform translation at Courant number one moves every
cell's fraction one cell downstream, across the period too, and a whole period
of such steps returns the field exactly; a rolled field reconstructs to the
rolled planes; images of one point take one value; the volume is conserved
with no boundary flux; and the paper's printed translation errors.
"""
import os

import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore")


def _random_field(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, n)
    a[rng.uniform(size=n) < 0.2] = 0.0
    a[rng.uniform(size=n) < 0.2] = 1.0
    return a


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_exact_shift_across_the_period(oracle_lib, axis):
    """U along one axis, dt = h: every face normal to it sweeps exactly its
    upwind cell, the seam's faces included, so alpha rolls by one cell; after
    a whole period of steps it is back (any field)."""
    shape = (5, 4, 3)
    m = I.hex_mesh(shape, (1.0, 0.8, 0.6), periodic="xyz")       # cubic cells, h = 0.2
    om = oracle_lib.OracleMesh(m)
    a0 = _random_field(m.n_cells, 40 + axis)
    U = np.zeros(3)
    U[axis] = 1.0
    fld = I.translation_field(U)
    F = I.face_flux_stokes(m, fld.A)
    Uc = I.cell_velocity(m, fld.u)
    a, stats, st = om.advect(a0, Uc, F, m.h, bound=False)
    assert st == 0
    A0 = a0.reshape(shape[::-1])
    A1 = a.reshape(shape[::-1])
    assert np.abs(A1 - np.roll(A0, 1, axis=2 - axis)).max() < 1e-12
    assert stats[oracle_lib.S["boundary_out"]] == 0.0
    for _ in range(shape[axis] - 1):
        a, stats, st = om.advect(a, Uc, F, m.h, bound=False)
    assert np.abs(a - a0).max() < 1e-11


def test_rolled_field_reconstructs_to_rolled_planes(oracle_lib):
    """On a uniform periodic mesh the seam is invisible: reconstructing the
    field rolled by one cell gives the rolled normals, and planes moved by the
    cell's translation (n.t added to d, t = h or h - L where the roll wraps)."""
    nx, ny, nz = 6, 5, 4
    m = I.hex_mesh((nx, ny, nz), (1.0, 5 / 6, 4 / 6), periodic="xyz")
    om = oracle_lib.OracleMesh(m)
    # a sphere that crosses the x = 0 seam
    a = I.sampled_fraction(m, lambda x: np.sqrt(((np.where(x[..., 0] > 0.5, x[..., 0] - 1, x[..., 0]) - 0.05) ** 2)
                                                + (x[..., 1] - 0.5) ** 2 + (x[..., 2] - 0.45) ** 2) - 0.3)
    ar = np.roll(a.reshape(nz, ny, nx), 1, axis=2).reshape(-1)
    n0, d0, f0, _, s0 = om.reconstruct(a)
    n1, d1, f1, _, s1 = om.reconstruct(ar)
    assert s0 == 0 and s1 == 0
    roll = lambda v: np.roll(v.reshape(-1, nz, ny, nx), 1, axis=3).reshape(v.shape)
    assert np.array_equal(f1, roll(f0[None])[0])
    cells = np.flatnonzero(f1 & oracle_lib.ORIENTED)
    assert cells.size > 30
    n0r = roll(n0.reshape(3, -1))
    assert np.abs(n1[:, cells] - n0r[:, cells]).max() < 1e-12
    i = cells % nx
    shift = np.where(i == 0, m.h - 1.0, m.h)
    d0r = roll(d0[None])[0]
    assert np.abs(d1[cells] - (d0r[cells] + n1[0, cells] * shift)).max() < 1e-12


def test_point_images_take_one_value(oracle_lib):
    m = I.hex_mesh((5, 4, 6), jitter=0.2, seed=7, periodic="xz")
    om = oracle_lib.OracleMesh(m)
    a = _random_field(m.n_cells, 9)
    v = om.point_interp(a)
    assert np.abs(v - v[m.point_master]).max() < 1e-14
    # the weights of a point are a partition of unity over all images' cells
    assert np.abs(om.point_interp(np.ones(m.n_cells)) - 1).max() < 1e-14
    # fully periodic: every face sees 18 cells, on the seam as inside
    m3 = I.hex_mesh((5, 4, 6), jitter=0.2, seed=7, periodic="xyz")
    om3 = oracle_lib.OracleMesh(m3)
    sizes = np.array([om3.stencil(f).size for f in range(m3.n_internal)])
    assert sizes.min() == sizes.max() == 18
    cells, codes = om3.stencil_codes(m3.n_internal - 1)
    assert (codes != 13).any() and (codes == 13).any()


def test_conservation_on_a_jittered_periodic_mesh(oracle_lib):
    m = I.hex_mesh((6, 6, 6), jitter=0.2, seed=11, periodic="xyz")
    om = oracle_lib.OracleMesh(m)
    a = I.sampled_fraction(m, I.sphere_sdf((0.9, 0.1, 0.5), 0.3))
    fld = I.translation_field((1.0, 0.6, -0.3))
    F = I.face_flux_stokes(m, fld.A)
    Uc = I.cell_velocity(m, fld.u)
    S = oracle_lib.S
    for _ in range(8):
        a, stats, st = om.advect(a, Uc, F, 0.5 * m.h / np.linalg.norm([1.0, 0.6, -0.3]))
        assert st == 0
        assert abs(stats[S["mass_after"]] - stats[S["mass_before"]]) <= 1e-13 * stats[S["mass_before"]]
        assert stats[S["boundary_out"]] == 0.0
        assert stats[S["min_post"]] >= -1e-12 and stats[S["max_post"]] <= 1 + 1e-12


def test_periodic_disc_translation(oracle_lib):
    """The 2D disc of the first test case on the periodic 32x32 box: it leaves
    through y = 1 and comes back at y = 0; the volume stays to round-off and
    the shape error against the wrapped exact disc is small."""
    w = I.make_workload("disc2d")
    om = oracle_lib.OracleMesh(w.mesh)
    _, vc, _, _ = om.geometry()
    a = w.alpha0.copy()
    S = oracle_lib.S
    for k in range(w.n_steps):
        F, U, dt = w.step_inputs(k)
        a, stats, st = om.advect(a, U, F, dt)
        assert st == 0 and stats[S["boundary_out"]] == 0.0
    ex = w.exact(w.n_steps * w.dt)
    assert (a * vc).sum() == pytest.approx((w.alpha0 * vc).sum(), rel=1e-14)
    assert ex.reshape(32, 32)[:3].sum() > 1.0       # the exact disc has wrapped to y = 0
    assert a.reshape(32, 32)[:3].sum() == pytest.approx(ex.reshape(32, 32)[:3].sum(), rel=0.01)
    assert (np.abs(a - ex) * vc).sum() / (ex * vc).sum() < 0.005


@pytest.mark.parametrize("co", [0.5, 0.75])
def test_translation_error_near_paper_table(oracle_lib, co):
    """The paper's periodic translation case at 16^3 (R21: to the corner
    (1,1,1), back to (0,0,0) and to the centre, t = 2; Courant number on the
    speed): the oracle's L1 error within [0.8, 1.25] of the printed E_g
    (table tab:errors:translation; tests/golden/paper_translation_eg.txt)."""
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "paper_translation_eg.txt"))
    paper = rows[rows[:, 0] == co][0, 1]
    w = I.make_workload("translate3d", n=16, co=co)
    om = oracle_lib.OracleMesh(w.mesh)
    _, vc, _, _ = om.geometry()
    a, t, k = w.alpha0.copy(), 0.0, 0
    while t < w.t_end - 1e-12:
        d = min(w.dt, w.t_end - t)
        F, U, _ = w.step_inputs(k, d)
        a, stats, st = om.advect(a, U, F, d)
        assert st == 0
        t += d
        k += 1
    l1 = float((vc * np.abs(a - w.alpha0)).sum())
    print(f"Co {co}: oracle L1 {l1:.5e}, paper E_g {paper:.5e}")
    assert abs(float((vc * (a - w.alpha0)).sum())) < 1e-15
    assert 0.8 * paper <= l1 <= 1.25 * paper
