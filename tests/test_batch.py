"""Batched form: cases joined into one mesh, each case's time step folded into
its F and U, one graph launch per step.

CPU: the joined mesh is the disjoint union of the cases (offsets, internal
faces first, no face between cases, discretely divergence-free F dt per cell).
GPU: one batched step equals, case by case, one oracle step on the case's own
mesh with its own dt (FP64 to the replay tolerance, mixed to the mixed one);
the graph replay equals direct launches bit for bit; the tuner leaves alpha
alone and every launch shape gives the same step bit for bit (each face's
flux is one warp's work whatever the launch); per-case masses match the host.
"""
import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

MIXED_ALPHA_TOL = 2e-5


@pytest.fixture(scope="module")
def batch():
    return I.make_batch(6, seed=1304, hex_range=(5, 8), tet_range=(4, 6), steps=3)


def test_joined_mesh(batch):
    m, off = batch.mesh, batch.cell_off
    assert off[0] == 0 and off[-1] == m.n_cells
    assert m.n_internal == sum(c.n_internal for c in batch.meshes)
    assert m.n_faces == sum(c.n_faces for c in batch.meshes)
    case_of = np.repeat(np.arange(len(batch.cases)), np.diff(off))
    # internal faces join cells of one case only
    assert np.array_equal(case_of[m.owner[:m.n_internal]], case_of[m.neighbour])
    assert np.all(m.owner[:m.n_internal] < m.neighbour)
    # F dt is divergence-free cell by cell
    div = np.zeros(m.n_cells)
    np.add.at(div, m.owner, batch.F_dt)
    np.add.at(div, m.neighbour, -batch.F_dt[:m.n_internal])
    assert np.abs(div).max() < 1e-15
    # case data matches the case's own arrays
    for i, c in enumerate(batch.cases):
        assert np.array_equal(batch.alpha0[off[i]:off[i + 1]], batch.alpha_case[i])
        np.testing.assert_allclose(batch.U_dt[:, off[i]:off[i + 1]], batch.U_case[i] * c.dt, rtol=0, atol=0)
        assert 0.3 <= c.co <= 0.8
    assert {c.kind for c in batch.cases} == {"hex", "tet"}


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3417_gb300 import build
    build.build()
    return torch


def _dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1).copy()).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, MIXED_ALPHA_TOL)])
def test_batch_step_matches_cases(torch, oracle_lib, batch, precision, tol):
    from paper_1305_3417_gb300 import vof
    b = vof.VofBatch(batch, precision=precision)
    a = _dev(torch, batch.alpha0)
    U, F = _dev(torch, batch.U_dt), _dev(torch, batch.F_dt)
    b.advect(a, U, F)
    got = a.cpu().numpy()
    assert vof.vof_status(b.context()) == 0
    off = batch.cell_off
    for i, c in enumerate(batch.cases):
        om = oracle_lib.OracleMesh(batch.meshes[i])
        oa, _, st = om.advect(batch.alpha_case[i].copy(), batch.U_case[i], batch.F_case[i], c.dt)
        assert st == 0
        err = np.abs(got[off[i]:off[i + 1]] - oa).max()
        assert err < tol, (i, c.kind, c.interface, err)


@pytest.mark.gpu
def test_batch_graph_equals_direct(torch, batch):
    from paper_1305_3417_gb300 import vof
    b = vof.VofBatch(batch, precision=1)
    ctx = b.context()
    U, F = _dev(torch, batch.U_dt), _dev(torch, batch.F_dt)
    a1, a2 = _dev(torch, batch.alpha0), _dev(torch, batch.alpha0)
    for _ in range(3):
        b.advect(a1, U, F)
        vof.vof_advect(ctx, a2, U, F, 1.0)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2)


@pytest.mark.gpu
def test_batch_tuner(torch, batch):
    from paper_1305_3417_gb300 import vof
    b = vof.VofBatch(batch, precision=1)
    U, F = _dev(torch, batch.U_dt), _dev(torch, batch.F_dt)
    a0 = _dev(torch, batch.alpha0)
    ref = a0.clone()
    b.advect(ref, U, F)                     # default launch shape
    keep = a0.clone()
    cfg, ms = b.tune(a0, U, F)
    torch.cuda.synchronize()
    assert torch.equal(a0, keep)            # the tuner steps on a copy
    assert cfg in {256 * st + 16 * w + m for st in (0, 1) for w in (1, 2, 3) for m in (1, 2, 4)} and ms > 0
    tuned = a0.clone()
    b.advect(tuned, U, F)                   # tuned launch shape (new graph)
    torch.cuda.synchronize()
    if cfg // 256 == 0:                     # the default staging depth: bit for bit
        assert torch.equal(tuned, ref)
    else:                                   # the other depth: to the sums' rounding
        assert (tuned - ref).abs().max().item() < 1e-13


@pytest.mark.gpu
def test_batch_case_mass(torch, oracle_lib, batch):
    from paper_1305_3417_gb300 import vof
    b = vof.VofBatch(batch, precision=1)
    U, F = _dev(torch, batch.U_dt), _dev(torch, batch.F_dt)
    a = _dev(torch, batch.alpha0)
    mass = torch.zeros(len(batch.cases), dtype=torch.float64, device="cuda")
    b.advect(a, U, F, case_mass=mass)
    got, mass = a.cpu().numpy(), mass.cpu().numpy()
    off = batch.cell_off
    for i in range(len(batch.cases)):
        om = oracle_lib.OracleMesh(batch.meshes[i])
        _, vc, _, _ = om.geometry()
        want = float(np.dot(vc, got[off[i]:off[i + 1]]))
        assert mass[i] == pytest.approx(want, rel=1e-13, abs=1e-300)
