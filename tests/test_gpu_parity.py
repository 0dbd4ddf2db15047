"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Each stage is checked twice: fed the oracle's own inputs (isolating the
kernel), and end to end.  Tolerances follow from the arithmetic: the FP64
kernels differ from the oracle only in summation order and fused
multiply-adds, so geometric quantities agree to ~1e-14 relative; plane offsets
are compared through the oracle's fill function (both sides stop at a fill
residual of 1e-13); phase volumes within 1e-12 of the cell volume.
"""
import math

import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3417_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def T(torch, x, dtype=None):
    x = np.ascontiguousarray(x)
    t = torch.from_numpy(x.reshape(-1).copy())
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def H(t):
    return t.detach().cpu().numpy()


WORKLOADS = {
    "disc2d": lambda: I.make_workload("disc2d"),              # periodic in x and y
    "disc2d_open": lambda: I.make_workload("disc2d_open"),
    "deform20": lambda: I.make_workload("deform3d", n=20),
    "tet7": lambda: I.make_workload("vortex_tet", n=7),
    "shear_per": lambda: I.make_workload("shear_periodic", n=12),  # jittered, periodic in x, y, z
}
_cache = {}


def workload(name):
    if name not in _cache:
        _cache[name] = WORKLOADS[name]()
    return _cache[name]


def contexts(torch, O, name, precision=0):
    from paper_1305_3417_gb300 import vof
    w = workload(name)
    key = (name, precision)
    if key not in _cache:
        _cache[key] = (vof.VofContext(w.mesh, precision=precision), O.OracleMesh(w.mesh))
    _cache[key][0].status()  # start from a clear status word
    return w, _cache[key][0], _cache[key][1]


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_geometry(torch, O, name):
    w, ctx, om = contexts(torch, O, name)
    cc, vc, cf, sf = (H(x) for x in ctx.geometry())
    occ, ovc, ocf, osf = om.geometry()
    assert np.abs(cc - occ).max() < 1e-14
    assert np.abs(vc - ovc).max() < 1e-14 * ovc.max()
    assert np.abs(cf - ocf).max() < 1e-14
    assert np.abs(sf - osf).max() < 1e-14 * np.abs(osf).max()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_point_velocity(torch, O, name):
    w, ctx, om = contexts(torch, O, name)
    F, U, dt = w.step_inputs(3)
    Up = H(ctx.point_velocity(T(torch, U))).reshape(3, -1)
    oUp = om.point_velocity(U)
    assert np.abs(Up - oUp).max() < 1e-14 * max(np.abs(oUp).max(), 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_reconstruct(torch, O, name, precision):
    w, ctx, om = contexts(torch, O, name, precision=precision)
    a = w.alpha0
    n, d, fl, it = (H(x) for x in ctx.reconstruct(T(torch, a)))
    n = n.reshape(3, -1)
    on, od, ofl, oit, ost = om.reconstruct(a)
    assert np.array_equal(fl, ofl)
    cells = np.flatnonzero(fl & O.ORIENTED)
    assert cells.size > 10
    assert np.abs(n[:, cells] - on[:, cells]).max() < 1e-11
    _, vc, _, _ = om.geometry()
    # the plane the GPU placed holds alpha*V of the cell, by the oracle's clipper
    for c in cells:
        g = om.cut_volume(c, n[:, c], d[c]) / vc[c] - a[c]
        assert abs(g) <= 3e-13, (c, g)
    assert it[cells].max() <= 100


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_flux_polyhedra(torch, O, name):
    w, ctx, om = contexts(torch, O, name)
    F, U, dt = w.step_inputs(0)
    oUp = om.point_velocity(U)
    rng = np.random.default_rng(5)
    lam = rng.uniform(0.2, 1.8, w.mesh.n_faces)
    lam[::13] = -1.0
    V = H(ctx.flux_polyhedra(T(torch, oUp), dt, T(torch, lam), T(torch, F)))
    faces = np.arange(0, w.mesh.n_faces, max(1, w.mesh.n_faces // 3000))
    oV = np.array([om.swept_volume(f, oUp, dt, lam[f], F[f]) for f in faces])
    scale = np.abs(oV).max()
    assert np.abs(V[faces] - oV).max() < 1e-13 * scale


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_correct_flux(torch, O, name):
    w, ctx, om = contexts(torch, O, name)
    F, U, dt = w.step_inputs(1)
    oUp = om.point_velocity(U)
    lam, it = (H(x) for x in ctx.correct_flux(T(torch, oUp), T(torch, F), dt))
    olam, oit, ost = om.correct_flux(oUp, F, dt)
    assert ost == 0
    fb, ofb = lam < 0, olam < 0
    assert np.array_equal(fb, ofb)
    ok = ~fb
    assert np.abs(lam[ok] - olam[ok]).max() < 1e-10
    # the corrected polyhedra hold the flux volume
    V = H(ctx.flux_polyhedra(T(torch, oUp), dt, T(torch, lam), T(torch, F)))
    assert np.abs(V - F * dt).max() <= 1e-12 * np.abs(F * dt).max()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_phase_flux_on_oracle_inputs(torch, O, name):
    w, ctx, om = contexts(torch, O, name)
    F, U, dt = w.step_inputs(2)
    a = w.alpha0
    on, od, ofl, _, _ = om.reconstruct(a)
    oUp = om.point_velocity(U)
    olam, _, _ = om.correct_flux(oUp, F, dt)
    oVa, ost = om.phase_flux(a, on, od, ofl, oUp, F, olam, dt)
    assert ost == 0
    Va = H(ctx.phase_flux(T(torch, a), T(torch, on), T(torch, od), T(torch, ofl, torch.uint8),
                          T(torch, oUp), T(torch, F), T(torch, olam), dt))
    _, vc, _, _ = om.geometry()
    assert np.abs(Va - oVa).max() < 1e-12 * vc.max()
    assert ctx.status() == 0


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_update(torch, O, name):
    w, ctx, om = contexts(torch, O, name)
    rng = np.random.default_rng(3)
    _, vc, _, _ = om.geometry()
    Va = rng.normal(size=w.mesh.n_faces) * 1e-3 * vc.mean()
    a = np.clip(w.alpha0 + 0.0, 0, 1)
    ta = T(torch, a)
    stats = H(ctx.update(ta, T(torch, Va)))
    oa, ost_arr, ost = om.update(a, Va, bound=True)
    assert np.abs(H(ta) - oa).max() < 1e-14
    assert stats[0] == pytest.approx(ost_arr[0], rel=1e-13)
    assert stats[1] == pytest.approx(ost_arr[1], rel=1e-13)
    assert stats[2] == pytest.approx(ost_arr[2], abs=1e-15)
    assert stats[5] == pytest.approx(ost_arr[5], abs=1e-14)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_advect_step_replay(torch, O, name):
    """Full step A1-A7: from the GPU's own state at several steps, one step on
    both sides agrees cell by cell (replay parity)."""
    w, ctx, om = contexts(torch, O, name)
    _, vc, _, _ = om.geometry()
    ta = T(torch, w.alpha0)
    for k in range(6):
        F, U, dt = w.step_inputs(k)
        a_in = H(ta).copy()
        stats = H(ctx.advect(ta, T(torch, U), T(torch, F), dt))
        oa, ost, st = om.advect(a_in, U, F, dt)
        assert st == 0 and ctx.status() == 0
        assert np.abs(H(ta) - oa).max() < 1e-11, k
        assert stats[6] == ost[6] and stats[7] == ost[7]
        drift = abs(stats[1] + stats[10] - stats[0]) / stats[0]
        assert drift < 1e-12
        assert stats[4] >= -1e-12 and stats[5] <= 1 + 1e-12


def test_exact_shift_gpu(torch, O):
    from paper_1305_3417_gb300 import vof
    nx = 7
    m = I.hex_mesh((nx, 5, 4), open_sides=("x-", "x+"))
    rng = np.random.default_rng(14)
    a = rng.uniform(0, 1, m.n_cells)
    a[rng.uniform(size=m.n_cells) < 0.2] = 0.0
    a[rng.uniform(size=m.n_cells) < 0.2] = 1.0
    fld = I.translation_field((1.0, 0.0, 0.0))
    F = I.face_flux_stokes(m, fld.A)
    Uc = I.cell_velocity(m, fld.u)
    ctx = vof.VofContext(m, bound=False)
    ta = T(torch, a)
    ctx.advect(ta, T(torch, Uc), T(torch, F), m.h)
    A0, A1 = a.reshape(4, 5, nx), H(ta).reshape(4, 5, nx)
    assert np.abs(A1[:, :, 1:] - A0[:, :, :-1]).max() < 1e-12
    assert np.abs(A1[:, :, 0]).max() < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_exact_shift_across_the_period_gpu(torch, O, axis, precision):
    """Periodic in x, y, z, U along one axis, dt = h: alpha rolls by one cell,
    across the seam too; a whole period of steps brings it back."""
    from paper_1305_3417_gb300 import vof
    shape = (5, 4, 3)
    m = I.hex_mesh(shape, (1.0, 0.8, 0.6), periodic="xyz")
    rng = np.random.default_rng(40 + axis)
    a = rng.uniform(0, 1, m.n_cells)
    a[rng.uniform(size=m.n_cells) < 0.2] = 0.0
    a[rng.uniform(size=m.n_cells) < 0.2] = 1.0
    U = np.zeros(3)
    U[axis] = 1.0
    fld = I.translation_field(U)
    F = I.face_flux_stokes(m, fld.A)
    Uc = I.cell_velocity(m, fld.u)
    ctx = vof.VofContext(m, precision=precision, bound=False)
    ta = T(torch, a)
    stats = H(ctx.advect(ta, T(torch, Uc), T(torch, F), m.h))
    A0, A1 = a.reshape(shape[::-1]), H(ta).reshape(shape[::-1])
    tol = 1e-12 if precision == 0 else 2e-5
    assert np.abs(A1 - np.roll(A0, 1, axis=2 - axis)).max() < tol
    assert stats[10] == 0.0  # nothing leaves: no boundary flux
    for _ in range(shape[axis] - 1):
        ctx.advect(ta, T(torch, Uc), T(torch, F), m.h)
    assert np.abs(H(ta) - a).max() < 10 * tol
    assert ctx.status() == 0
    ctx.close()


def test_periodic_mesh_errors(torch, O):
    """Periodic data that do not fit are rejected; a batch takes no periodic mesh."""
    from paper_1305_3417_gb300 import vof
    import copy
    m = I.hex_mesh((4, 4, 3), periodic="xy")
    bad = copy.deepcopy(m)
    bad.face_image[np.flatnonzero(bad.face_image >= 0)[0]] = 0       # a copy of the wrong face
    with pytest.raises(vof.VofError):
        vof.VofContext(bad)
    bad = copy.deepcopy(m)
    bad.point_image[np.flatnonzero(bad.point_image[:, 0])[0], 0] = 2  # two periods away
    with pytest.raises(vof.VofError):
        vof.VofContext(bad)
    one = I.hex_mesh((1, 4, 3), periodic="x")                        # a cell at two images of a point
    with pytest.raises(vof.VofError):
        vof.VofContext(one)
    with pytest.raises(vof.VofError):
        vof.vof_batch_create(m, np.array([0, m.n_cells], np.int32))


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_courant(torch, O, name):
    """The step's Courant number on the device equals the oracle's."""
    w, ctx, om = contexts(torch, O, name)
    F, U, dt = w.step_inputs(1)
    co = ctx.courant(T(torch, F), dt)
    assert co > 0.0
    assert co == pytest.approx(om.courant(F, dt), rel=1e-13)


def test_edge_cases(torch, O):
    w, ctx, om = contexts(torch, O, "deform20")
    F, U, dt = w.step_inputs(0)
    nc = w.mesh.n_cells
    for val in (0.0, 1.0):
        ta = T(torch, np.full(nc, val))
        stats = H(ctx.advect(ta, T(torch, U), T(torch, F), dt))
        assert stats[7] == 0  # no band face
        assert np.abs(H(ta) - val).max() < 1e-13
    # no flux at all: alpha unchanged
    ta = T(torch, w.alpha0)
    ctx.advect(ta, T(torch, U), T(torch, np.zeros_like(F)), dt)
    assert np.array_equal(H(ta), w.alpha0)
    # one mixed cell in an empty domain (unoriented: zero gradient by symmetry is not
    # guaranteed on a jittered mesh, so compare with the oracle)
    a = np.zeros(nc)
    a[nc // 2 + 10] = 0.5
    ta = T(torch, a)
    ctx.advect(ta, T(torch, U), T(torch, F), dt)
    oa, _, _ = om.advect(a, U, F, dt)
    assert np.abs(H(ta) - oa).max() < 1e-12
    assert ctx.status() == 0


def test_invalid_arguments(torch, O):
    from paper_1305_3417_gb300 import vof
    w, ctx, om = contexts(torch, O, "disc2d_open")
    L = vof.lib()
    F, U, dt = w.step_inputs(0)
    tF, tU, ta = T(torch, F), T(torch, U), T(torch, w.alpha0)
    s = vof._stream(None)
    import ctypes
    assert L.vof_advect(ctx.h, None, vof._ptr(tU), vof._ptr(tF), dt, None, s) == -1
    assert L.vof_advect(ctx.h, vof._ptr(ta), vof._ptr(tU), vof._ptr(tF), -1.0, None, s) == -1
    assert L.vof_advect(ctx.h, vof._ptr(ta), vof._ptr(tU), vof._ptr(tF), float("nan"), None, s) == -1
    assert L.vof_advect(None, vof._ptr(ta), vof._ptr(tU), vof._ptr(tF), dt, None, s) == -1
    # a mesh with an out-of-range point index is rejected
    m = workload("disc2d_open").mesh
    bad = I.Mesh(m.points, m.face_ptr, m.face_pts.copy(), m.owner, m.neighbour, m.n_cells, m.cell_verts,
                 m.h, m.dim, m.kind, m.shape, m.wall)
    bad.face_pts[5] = m.n_points + 3
    with pytest.raises(vof.VofError):
        vof.VofContext(bad)
    # inverted cells are rejected
    inv = I.Mesh(m.points * np.array([1.0, 1.0, -1.0]), m.face_ptr, m.face_pts, m.owner, m.neighbour,
                 m.n_cells, m.cell_verts, m.h, m.dim, m.kind, m.shape, m.wall)
    with pytest.raises(vof.VofError):
        vof.VofContext(inv)
    assert ctypes is not None


def test_determinism(torch, O):
    w, ctx, om = contexts(torch, O, "deform20")
    F, U, dt = w.step_inputs(4)
    outs = []
    for _ in range(2):
        ta = T(torch, w.alpha0)
        st = ctx.advect(ta, T(torch, U), T(torch, F), dt)
        outs.append((H(ta), H(st)))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_advect_host_matches_device(torch, O):
    from paper_1305_3417_gb300 import vof
    w, ctx, om = contexts(torch, O, "deform20")
    F, U, dt = w.step_inputs(1)
    ta = T(torch, w.alpha0)
    ctx.advect(ta, T(torch, U), T(torch, F), dt)
    ha = torch.from_numpy(w.alpha0.copy()).pin_memory()
    hU = torch.from_numpy(np.ascontiguousarray(U).reshape(-1).copy()).pin_memory()
    hF = torch.from_numpy(F.copy()).pin_memory()
    hs = torch.zeros(vof.S_LEN, dtype=torch.float64).pin_memory()
    vof.vof_advect_host(ctx.h, ha, hU, hF, dt, hs)
    torch.cuda.synchronize()
    assert np.array_equal(ha.numpy(), H(ta))


def test_grid_barrier_wait_runs_out(torch, O):
    """The cooperative bounding kernel's grid barrier: with every block arriving
    nothing is flagged; with one block leaving at once the others' bounded
    waits run out, set VOF_ST_TIMEOUT and leave (no hang), and the context
    still steps correctly afterwards."""
    from paper_1305_3417_gb300 import vof
    w, ctx, om = contexts(torch, O, "deform20")
    vof.vof_probe_barrier(ctx.h, -1)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    vof.vof_probe_barrier(ctx.h, 0)
    torch.cuda.synchronize()
    assert ctx.status() & 64
    assert ctx.status() == 0           # reading clears the word
    F, U, dt = w.step_inputs(0)
    ta = T(torch, w.alpha0)
    ctx.advect(ta, T(torch, U), T(torch, F), dt)
    oa, _, st = om.advect(w.alpha0.copy(), U, F, dt)
    assert st == 0 and ctx.status() == 0
    assert np.abs(H(ta) - oa).max() < 1e-11


def test_advect_host_pageable_buffers(torch, O):
    """Host arrays that are not pinned (staged copies, synchronous with respect
    to the host): the same step bit for bit."""
    from paper_1305_3417_gb300 import vof
    w, ctx, om = contexts(torch, O, "deform20")
    F, U, dt = w.step_inputs(2)
    ta = T(torch, w.alpha0)
    st = ctx.advect(ta, T(torch, U), T(torch, F), dt)
    ha = torch.from_numpy(w.alpha0.copy())
    assert not ha.is_pinned()
    hs = torch.zeros(vof.S_LEN, dtype=torch.float64)
    vof.vof_advect_host(ctx.h, ha, torch.from_numpy(np.ascontiguousarray(U).reshape(-1).copy()),
                        torch.from_numpy(F.copy()), dt, hs)
    torch.cuda.synchronize()
    assert np.array_equal(ha.numpy(), H(ta))
    assert np.array_equal(hs.numpy(), H(st))


def test_advect_host_steps_queued(torch, O):
    """Five host-buffer steps queued back to back (pinned U read in place by the
    kernels over the host link, F and pageable U copied through two
    alternating device buffer pairs that overlap the previous step) give the
    same fields and statistics, bit for bit, as the device-buffer steps one by
    one."""
    from paper_1305_3417_gb300 import vof
    w, ctx, om = contexts(torch, O, "deform20")
    steps = [w.step_inputs(k) for k in range(5)]
    ta = T(torch, w.alpha0)
    for F, U, dt in steps:
        st = ctx.advect(ta, T(torch, U), T(torch, F), dt)
    ha = torch.from_numpy(w.alpha0.copy()).pin_memory()
    hU = [torch.from_numpy(np.ascontiguousarray(U).reshape(-1).copy()).pin_memory() for _, U, _ in steps]
    hF = [torch.from_numpy(F.copy()).pin_memory() for F, _, _ in steps]
    hs = torch.zeros(vof.S_LEN, dtype=torch.float64).pin_memory()
    for k, (_, _, dt) in enumerate(steps):
        vof.vof_advect_host(ctx.h, ha, hU[k], hF[k], dt, hs)
    torch.cuda.synchronize()
    assert np.array_equal(ha.numpy(), H(ta))
    assert np.array_equal(hs.numpy(), H(st))
    # pageable U and F (the copy path), alpha pinned, queued the same way
    ha = torch.from_numpy(w.alpha0.copy()).pin_memory()
    pU = [u.clone() for u in hU]
    pF = [f.clone() for f in hF]
    assert not pU[0].is_pinned()
    for k, (_, _, dt) in enumerate(steps):
        vof.vof_advect_host(ctx.h, ha, pU[k], pF[k], dt, hs)
    torch.cuda.synchronize()
    assert np.array_equal(ha.numpy(), H(ta))
    assert np.array_equal(hs.numpy(), H(st))


_FULL = {}


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5)])
def test_full_size_sampled(torch, O, precision, tol):
    """128^3 jittered hex, deformation field: one GPU step in the benchmark's
    launch configuration (FP64 and the benchmarked mixed form), compared with
    the oracle on sampled cells (the oracle reconstructs the stencil cells and
    corrects and fluxes the faces it needs)."""
    from paper_1305_3417_gb300 import vof
    if "w" not in _FULL:
        _FULL["w"] = I.make_workload("deform3d")
    w = _FULL["w"]
    m = w.mesh
    ctx = vof.VofContext(m, precision=precision, bound=False)
    om = O.OracleMesh(m)
    F, U, dt = w.step_inputs(0)
    ta = T(torch, w.alpha0)
    stats = H(ctx.advect(ta, T(torch, U), T(torch, F), dt))
    assert ctx.status() == 0
    a1 = H(ta)
    rng = np.random.default_rng(21)
    cls = om.classify_faces(w.alpha0)
    band = np.flatnonzero((cls == 2) & (F != 0))
    assert stats[7] == band.size
    # sample cells touching band faces plus random cells
    band_cells = np.unique(np.concatenate([m.owner[band], m.neighbour[band[band < m.n_internal]]]))
    cells = np.unique(np.concatenate([rng.choice(band_cells, 60, replace=False),
                                      rng.choice(m.n_cells, 40, replace=False)]))
    faces = np.unique(np.concatenate([np.flatnonzero(m.owner == c) for c in cells] +
                                     [np.flatnonzero(m.neighbour == c) for c in cells]))
    sten = np.unique(np.concatenate([om.stencil(f) for f in faces]))
    on, od, ofl, _, _ = om.reconstruct(w.alpha0, sel=sten)
    oUp = om.point_velocity(U)
    olam, _, _ = om.correct_flux(oUp, F, dt, sel=faces)
    oVa, ost = om.phase_flux(w.alpha0, on, od, ofl, oUp, F, olam, dt, sel=faces)
    _, vc, _, _ = om.geometry()
    for c in cells:
        s = 0.0
        for f in np.flatnonzero(m.owner == c):
            s += oVa[f]
        for f in np.flatnonzero(m.neighbour == c):
            s -= oVa[f]
        pre = w.alpha0[c] - s / vc[c]
        assert abs(a1[c] - pre) < tol, (c, a1[c], pre)
    assert abs(stats[1] - stats[0]) / stats[0] < 1e-12
    ctx.close()
    # the same step with the bounding pass keeps alpha in [0, 1]
    ctxb = vof.VofContext(m, precision=precision, bound=True)
    tb = T(torch, w.alpha0)
    sb = H(ctxb.advect(tb, T(torch, U), T(torch, F), dt))
    assert ctxb.status() == 0
    assert sb[4] >= -1e-12 and sb[5] <= 1 + 1e-12
    assert abs(sb[1] - sb[0]) / sb[0] < 1e-12
    ctxb.close()


# ------------------------------------------------------------ mixed precision
# FP32 clipping in a face-centred frame: each piece carries a relative rounding
# of a few 1e-7 of its own volume, so the phase volume of a face is within
# ~1e-6 of the face's swept volume; tolerances are stated against the cell
# volume.
MIXED_VA_TOL = 2e-6     # |dVa| / max V_c
MIXED_ALPHA_TOL = 2e-5  # |d alpha| after one full step


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_phase_flux_mixed_on_oracle_inputs(torch, O, name):
    w, ctx, om = contexts(torch, O, name, precision=1)
    F, U, dt = w.step_inputs(2)
    a = w.alpha0
    on, od, ofl, _, _ = om.reconstruct(a)
    oUp = om.point_velocity(U)
    olam, _, _ = om.correct_flux(oUp, F, dt)
    oVa, ost = om.phase_flux(a, on, od, ofl, oUp, F, olam, dt)
    Va = H(ctx.phase_flux(T(torch, a), T(torch, on), T(torch, od), T(torch, ofl, torch.uint8),
                          T(torch, oUp), T(torch, F), T(torch, olam), dt))
    _, vc, _, _ = om.geometry()
    err = np.abs(Va - oVa).max() / vc.max()
    print(f"mixed phase flux {name}: max |dVa|/V = {err:.3e}")
    assert err < MIXED_VA_TOL
    assert ctx.status() == 0


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_advect_mixed_replay(torch, O, name):
    w, ctx, om = contexts(torch, O, name, precision=1)
    ta = T(torch, w.alpha0)
    worst = 0.0
    for k in range(6):
        F, U, dt = w.step_inputs(k)
        a_in = H(ta).copy()
        stats = H(ctx.advect(ta, T(torch, U), T(torch, F), dt))
        oa, ost, st = om.advect(a_in, U, F, dt)
        assert st == 0 and ctx.status() == 0
        worst = max(worst, np.abs(H(ta) - oa).max())
        drift = abs(stats[1] + stats[10] - stats[0]) / stats[0]
        assert drift < 1e-12
        assert stats[4] >= -1e-12 and stats[5] <= 1 + 1e-12
    print(f"mixed advect {name}: max |d alpha| = {worst:.3e}")
    assert worst < MIXED_ALPHA_TOL


def test_tuner_keeps_the_state_and_the_step(torch, O):
    """vof_tune times every phase-flux launch shape and staging depth on a copy
    of the state and keeps the fastest.  The step it then runs equals the
    default launch's bit for bit when the staging depth is the default's (a
    face's pieces then fall to the same lanes in the same order), and to the
    rounding of the compensated sums otherwise."""
    from paper_1305_3417_gb300 import vof
    w, ctx, om = contexts(torch, O, "deform20", precision=1)
    F, U, dt = w.step_inputs(3)
    tU, tF = T(torch, U), T(torch, F)
    ref = T(torch, w.alpha0)
    ctx.advect(ref, tU, tF, dt)
    a = T(torch, w.alpha0)
    keep = a.clone()
    cfg, ms = vof.vof_tune(ctx.h, a, tU, tF, dt)
    torch.cuda.synchronize()
    assert torch.equal(a, keep) and ms > 0
    assert cfg in {256 * st + 16 * wp + m for st in (0, 1) for wp in (1, 2, 3) for m in (1, 2, 4)}
    ctx.advect(a, tU, tF, dt)
    if cfg // 256 == 0:
        assert torch.equal(a, ref)
    else:
        assert (a - ref).abs().max().item() < 1e-13
    assert ctx.status() == 0
