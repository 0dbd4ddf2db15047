"""Config 5's mesh: a static octree (base lattice split twice near a sphere,
2:1 face-balanced, hanging points on face edges).

CPU: the generator's mesh is a closed, balanced partition of the unit cube,
and the oracle's step on it conserves volume and stays bounded.  GPU: the
CUDA path against the oracle on the same octree -- reconstruction (cells of
up to 96 tetrahedra: three per lane) and full steps by replay, FP64 and mixed.
"""
import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

N0 = 12   # 13.4k cells; some cells have 96 tetrahedra, some faces 6 points


@pytest.fixture(scope="module")
def wl():
    return I.make_workload("octree", n=N0)


@pytest.mark.parametrize("levels", [2, 3])
def test_octree_mesh_is_a_balanced_closed_partition(oracle_lib, wl, levels):
    """Two levels: the workload's octree; three: a 5^3 base split three times,
    where the 2:1 balance has to cascade over several levels."""
    m = wl.mesh if levels == 2 else I.octree_mesh(5, 3, (0.3, 0.6, 0.5), 0.25, band=2.0)
    n0 = N0 if levels == 2 else 5
    om = oracle_lib.OracleMesh(m)
    cc, vc, cf, sf = om.geometry()
    sf = sf.reshape(3, -1) if sf.ndim == 1 else sf
    sf = sf if sf.shape[0] == 3 else sf.T
    # volumes: the boxes', summing to the cube
    box = m.points[m.cell_verts]
    ext = box.max(1) - box.min(1)
    np.testing.assert_allclose(vc, ext.prod(1), rtol=1e-12, atol=0)
    assert abs(vc.sum() - 1.0) < 1e-13
    # every cell's surface is closed
    net = np.zeros((3, m.n_cells))
    ni = m.n_internal
    for d in range(3):
        np.add.at(net[d], m.owner, sf[d])
        np.add.at(net[d], m.neighbour, -sf[d][:ni])
    assert np.abs(net).max() < 1e-15
    # 2:1 balance across faces, faces of 4..8 points, every point used
    h = ext[:, 0]
    r = h[m.owner[:ni]] / h[m.neighbour]
    assert set(np.unique(np.round(r, 12))) <= {0.5, 1.0, 2.0}
    npf = np.diff(m.face_ptr)
    assert npf.min() >= 4 and npf.max() <= 8 and (npf > 4).any()
    assert np.unique(m.face_pts).size == m.n_points
    # levels + 1 cell sizes
    assert np.unique(np.round(1.0 / h).astype(int)).tolist() == [n0 << L for L in range(levels + 1)]


def test_octree_oracle_steps_conserve_and_stay_bounded(oracle_lib, wl):
    om = oracle_lib.OracleMesh(wl.mesh)
    S = oracle_lib.S
    a = wl.alpha0.copy()
    assert ((a > 1e-9) & (a < 1 - 1e-9)).sum() > 100
    for k in range(3):
        F, U, dt = wl.step_inputs(k)
        a, st, status = om.advect(a, U, F, dt)
        assert status == 0
        drift = abs(st[S["mass_after"]] - st[S["mass_before"]]) / st[S["mass_before"]]
        assert drift <= 1e-12
        assert st[S["min_post"]] >= -1e-12 and st[S["max_post"]] <= 1 + 1e-12


# ------------------------------------------------------------------ GPU parity

@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3417_gb300 import build
    build.build()
    return torch


def _T(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1).copy()).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_octree_reconstruct_parity(torch, oracle_lib, wl, precision):
    from paper_1305_3417_gb300 import vof
    m = wl.mesh
    ctx = vof.VofContext(m, precision=precision)
    om = oracle_lib.OracleMesh(m)
    a = wl.alpha0
    n, d, fl, it = (t.cpu().numpy() for t in ctx.reconstruct(_T(torch, a)))
    on, od, ofl, _, _ = om.reconstruct(a)
    assert np.array_equal(fl, ofl)
    cells = np.flatnonzero(fl & oracle_lib.ORIENTED)
    assert cells.size > 100
    n = n.reshape(3, -1)
    assert np.abs(n[:, cells] - on[:, cells]).max() < 1e-11
    _, vc, _, _ = om.geometry()
    for c in cells[:: max(1, cells.size // 300)]:
        g = om.cut_volume(c, n[:, c], d[c]) / vc[c] - a[c]
        assert abs(g) <= 3e-13, (c, g)
    assert ctx.status() == 0


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5)])
def test_octree_step_replay_parity(torch, oracle_lib, wl, precision, tol):
    from paper_1305_3417_gb300 import vof
    m = wl.mesh
    ctx = vof.VofContext(m, precision=precision)
    om = oracle_lib.OracleMesh(m)
    ta = _T(torch, wl.alpha0)
    for k in range(4):
        F, U, dt = wl.step_inputs(k)
        a_in = ta.cpu().numpy().copy()
        st = ctx.advect(ta, _T(torch, U), _T(torch, F), dt).cpu().numpy()
        oa, ost, status = om.advect(a_in, U, F, dt)
        assert status == 0 and ctx.status() == 0
        assert np.abs(ta.cpu().numpy() - oa).max() < tol, k
        assert st[6] == ost[6] and st[7] == ost[7]      # interface cells, band faces
        assert abs(st[1] + st[10] - st[0]) <= 1e-12 * st[0]


def test_octree_nag_exact_on_uniform_neighbourhoods(oracle_lib, wl):
    """NAG reproduces a linear field's gradient where every cell around every
    point of the cell is a box of the same size with no hanging points and no
    point is on the boundary (as on a uniform lattice's interior): checks the
    octree's topology and face orientation through the oracle's gradient."""
    m = wl.mesh
    om = oracle_lib.OracleMesh(m)
    cc, _, _, _ = om.geometry()
    cc = cc.reshape(3, -1) if cc.ndim == 1 else (cc if cc.shape[0] == 3 else cc.T)
    gr = np.array([0.7, -1.1, 0.4])
    alpha = 0.3 + gr @ cc
    g = om.nag_gradient(alpha)
    # point -> cells through the faces (hanging points included)
    npf = np.diff(m.face_ptr)
    fid = np.repeat(np.arange(m.n_faces), npf)
    P = np.concatenate([m.face_pts, m.face_pts[fid < m.n_internal]])
    C = np.concatenate([m.owner[fid], m.neighbour[fid[fid < m.n_internal]]])
    pc = np.unique(np.stack([P, C], 1), axis=0)
    npts = np.bincount(pc[:, 1], minlength=m.n_cells)                # distinct points per cell
    box = m.points[m.cell_verts]
    h = (box.max(1) - box.min(1))[:, 0]
    plain = (npts == 8) & np.isclose(h, h.max())                    # coarsest boxes, no hanging points
    # a point on the boundary has a one-sided neighbourhood (as the hex pin's
    # boundary layer): its cells are left out
    bad_at_point = np.any(np.isclose(m.points, 0.0) | np.isclose(m.points, 1.0), axis=1)
    np.logical_or.at(bad_at_point, pc[:, 0], ~plain[pc[:, 1]])
    cell_bad = np.zeros(m.n_cells, bool)
    np.logical_or.at(cell_bad, pc[:, 1], bad_at_point[pc[:, 0]])
    sel = np.flatnonzero(plain & ~cell_bad)
    assert sel.size > 100
    assert np.abs(g[:, sel] - gr[:, None]).max() < 1e-11


def test_octree_stokes_fluxes_divergence_free(wl):
    """Face fluxes from the vector potential (Stokes, edge by edge) sum to zero
    over every cell's faces to round-off: every face that shares an edge with a
    hanging point splits it the same way, so the edge integrals cancel."""
    m = wl.mesh
    F = wl.F_spatial
    ni = m.n_internal
    div = np.zeros(m.n_cells)
    np.add.at(div, m.owner, F)
    np.add.at(div, m.neighbour, -F[:ni])
    scale = np.zeros(m.n_cells)
    np.add.at(scale, m.owner, np.abs(F))
    np.add.at(scale, m.neighbour, np.abs(F[:ni]))
    assert np.abs(div).max() <= 1e-14 * scale.max()


def test_octree_initial_fractions_hold_the_sphere(wl):
    """The initial fractions (8^3-point rule per box near the surface) hold the
    sphere's volume 4/3 pi R^3 to the rule's accuracy, and lie in [0, 1]."""
    m = wl.mesh
    box = m.points[m.cell_verts]
    V = np.prod(box.max(1) - box.min(1), axis=1)
    a = wl.alpha0
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert abs((V * a).sum() / (4.0 / 3.0 * np.pi * 0.15 ** 3) - 1.0) < 1e-3


@pytest.mark.gpu
def test_octree_full_size_sampled(torch, oracle_lib):
    """One mixed-precision step of config 5's octree (64^3 base, two levels,
    508k cells) in the benchmark's launch configuration, compared with the
    oracle on sampled cells (the oracle reconstructs the stencil cells and
    corrects and fluxes the faces it needs)."""
    from paper_1305_3417_gb300 import vof
    O = oracle_lib
    w = I.make_workload("octree")
    m = w.mesh
    ctx = vof.VofContext(m, precision=vof.MIXED, bound=False)
    om = O.OracleMesh(m)
    F, U, dt = w.step_inputs(0)
    ta = torch.from_numpy(w.alpha0.copy()).cuda()
    stats = ctx.advect(ta, torch.from_numpy(np.ascontiguousarray(U).reshape(-1).copy()).cuda(),
                       torch.from_numpy(F.copy()).cuda(), dt).cpu().numpy()
    assert ctx.status() == 0
    a1 = ta.cpu().numpy()
    rng = np.random.default_rng(29)
    cls = om.classify_faces(w.alpha0)
    band = np.flatnonzero((cls == 2) & (F != 0))
    assert stats[7] == band.size
    band_cells = np.unique(np.concatenate([m.owner[band], m.neighbour[band[band < m.n_internal]]]))
    cells = np.unique(np.concatenate([rng.choice(band_cells, 50, replace=False),
                                      rng.choice(m.n_cells, 20, replace=False)]))
    own = {c: np.flatnonzero(m.owner == c) for c in cells}
    nei = {c: np.flatnonzero(m.neighbour == c) for c in cells}
    faces = np.unique(np.concatenate(list(own.values()) + list(nei.values())))
    sten = np.unique(np.concatenate([om.stencil(f) for f in faces]))
    on, od, ofl, _, _ = om.reconstruct(w.alpha0, sel=sten)
    oUp = om.point_velocity(U)
    olam, _, _ = om.correct_flux(oUp, F, dt, sel=faces)
    oVa, ost = om.phase_flux(w.alpha0, on, od, ofl, oUp, F, olam, dt, sel=faces)
    assert ost == 0
    _, vc, _, _ = om.geometry()
    worst = 0.0
    for c in cells:
        pre = w.alpha0[c] - (oVa[own[c]].sum() - oVa[nei[c]].sum()) / vc[c]
        worst = max(worst, abs(a1[c] - pre))
    print(f"octree 64^3 base, mixed, one step: max |d alpha| on {cells.size} sampled cells = {worst:.2e}")
    assert worst < 2e-5
    assert abs(stats[1] - stats[0]) / stats[0] < 1e-12
    ctx.close()
