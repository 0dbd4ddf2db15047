"""Whole cases on the GPU against the oracle: the L1 shape error target.

Every form (plain FP64, mixed precision, mixed with the learned initial
guess) runs a whole case through vof_advect; the oracle runs the same inputs
on the host.  The L1 shape error is Sec. 5's E_g read as
L1 = sum_c V_c |alpha_c(T) - alpha_c^exact(T)| (reading R12), the exact state
being the translated disc (2D disc: periodic, the wrapped disc; open sides:
the disc clipped to the domain) or the initial field (the deformation and
single-vortex fields reverse at t = T, the periodic diagonal translation
returns the sphere to the centre).  The target: |L1_gpu - L1_oracle| <= 1e-6, conservation
per step, alpha within [0, 1] to 1e-12.

Also here: the redistribution of over/undershoots (reading R10) through
vof_update against amounts computed by hand, and one step of the 96^3 Kuhn
tetrahedral mesh (5.3 M cells) in the benchmark's launch configuration on
sampled cells.
"""
import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L1_TOL = 1e-6


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3417_gb300 import build
    build.build()
    return torch


def T(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1).copy()).cuda()


CASES = {
    "disc2d": lambda: I.make_workload("disc2d"),
    "disc2d_open": lambda: I.make_workload("disc2d_open"),
    "translate3d_16": lambda: I.make_workload("translate3d", n=16),
    "shear_periodic_12": lambda: I.make_workload("shear_periodic", n=12),
    "shear3d_16": lambda: I.make_workload("shear3d", n=16),
    "deform3d_24": lambda: I.make_workload("deform3d", n=24),
    "vortex_tet_10": lambda: I.make_workload("vortex_tet", n=10),
}
_cache = {}


def case(name):
    if name not in _cache:
        _cache[name] = CASES[name]()
    return _cache[name]


def schedule(w):
    """(step index, dt) of the whole case; the last step is trimmed to t_end."""
    if w.name.startswith("disc2d"):
        return [(k, w.dt) for k in range(w.n_steps)]
    out, t, k = [], 0.0, 0
    while t < w.t_end - 1e-12:
        d = min(w.dt, w.t_end - t)
        out.append((k, d))
        t += d
        k += 1
    return out


def exact(w):
    if w.name.startswith("disc2d"):
        return w.exact(w.n_steps * w.dt)
    return w.alpha0


def oracle_run(O, name):
    key = ("oracle", name)
    if key not in _cache:
        w = case(name)
        om = O.OracleMesh(w.mesh)
        _, vc, _, _ = om.geometry()
        a = w.alpha0.copy()
        flagged = 0
        for k, d in schedule(w):
            F, U, dt = w.step_inputs(k, d)
            a, st, s = om.advect(a, U, F, dt)
            flagged += s != 0
        _cache[key] = (a, vc, flagged)
    return _cache[key]


def trained_guess(torch, name):
    """A network trained on random spheres and planes on the case's mesh
    (targets from the FP64 reconstruction), as the learned form uses it."""
    from paper_1305_3417_gb300 import mlp, vof
    key = ("net", name)
    if key not in _cache:
        w = case(name)
        c64 = vof.VofContext(w.mesh, precision=vof.FP64)
        X, Y = mlp.samples(c64, w.mesh, mlp.random_fields(w.mesh, 6, seed=51))
        c64.close()
        net = vof.Mlp(mlp.init_params(52), max_batch=1 << 15)
        hist = mlp.train(net, X, Y, epochs=20, batch=min(1024, X.shape[0] // 2), lr=3e-3)
        assert hist[-1] < hist[0]
        _cache[key] = net
    return _cache[key]


@pytest.mark.parametrize("form", ["fp64", "mixed", "mixed_guess"])
@pytest.mark.parametrize("name", list(CASES))
def test_whole_case_l1_matches_oracle(torch, oracle_lib, name, form):
    from paper_1305_3417_gb300 import vof
    w = case(name)
    oa, vc, flagged = oracle_run(oracle_lib, name)
    assert flagged == 0
    ex = exact(w)
    prec = vof.FP64 if form == "fp64" else vof.MIXED
    ctx = vof.VofContext(w.mesh, precision=prec)
    if form == "mixed_guess":
        vof.vof_set_guess(ctx.h, trained_guess(torch, name))
    ta = T(torch, w.alpha0)
    stats = torch.zeros(vof.S_LEN, dtype=torch.float64, device="cuda")
    worst_drift, lo, hi = 0.0, 1.0, 0.0
    for k, d in schedule(w):
        F, U, dt = w.step_inputs(k, d)
        ctx.advect(ta, T(torch, U), T(torch, F), dt, stats)
        s = stats.cpu().numpy()
        # volume leaving through open boundary faces is the boundary outflow
        worst_drift = max(worst_drift, abs(s[1] + s[10] - s[0]) / s[0])
        lo, hi = min(lo, s[4]), max(hi, s[5])
        assert ctx.status() == 0, k
    a = ta.cpu().numpy()
    ctx.close()
    l1_gpu = float((vc * np.abs(a - ex)).sum())
    l1_orc = float((vc * np.abs(oa - ex)).sum())
    print(f"{name} {form}: L1 gpu {l1_gpu:.9e} oracle {l1_orc:.9e} |diff| {abs(l1_gpu - l1_orc):.2e}"
          f" drift {worst_drift:.1e} alpha [{lo:.2e}, {1 - hi:.2e} below 1]")
    assert worst_drift <= 1e-12
    assert lo >= -1e-12 and hi <= 1 + 1e-12
    assert abs(l1_gpu - l1_orc) <= L1_TOL


def test_disc2d_against_the_recorded_oracle_fields(torch):
    """The plain FP64 form through the 2D disc case against the oracle's
    recorded fields after 20 steps (tests/golden, written by the oracle)."""
    import os
    from paper_1305_3417_gb300 import vof
    w = case("disc2d")
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    a_ref = np.loadtxt(os.path.join(here, "disc2d_oracle_alpha20.txt"))
    with open(os.path.join(here, "disc2d_oracle.txt")) as f:
        l1_ref = float([ln for ln in f if ln.startswith("# L1")][0].split(":")[1])
    ctx = vof.VofContext(w.mesh, precision=vof.FP64)
    ta = T(torch, w.alpha0)
    for k, d in schedule(w):
        F, U, dt = w.step_inputs(k, d)
        ctx.advect(ta, T(torch, U), T(torch, F), dt)
    a = ta.cpu().numpy()
    vc = ctx.geometry()[1].cpu().numpy()
    ctx.close()
    assert np.abs(a - a_ref).max() < 1e-11
    l1 = float((vc * np.abs(a - w.exact(w.n_steps * w.dt))).sum())
    assert abs(l1 - l1_ref) <= 1e-12


# ----------------------------------------------------------- redistribution

ROWS = [
    # (alpha, expected after the redistribution, passes, global fallback / V)
    ([0.3, 1.2, 0.9, 0.5, -0.05, 0.0, 0.0], [0.44, 1.0, 0.96, 0.45, 0.0, 0.0, 0.0], 1, 0.0),
    ([1.2, 0.6, 1.3, 0.0, 0.5, 0.5, 0.5, 0.5], [1.0, 1.0, 1.0, 0.0, 0.525, 0.525, 0.525, 0.525], 1, 0.10),
    ([0.95, 1.5, 0.2, 0.0, 0.0], [1.0, 1.0, 0.65, 0.0, 0.0], 2, 0.0),
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("row", range(len(ROWS)))
def test_redistribution_amounts(torch, row, precision):
    """Reading R10 through vof_update with zero fluxes on a row of cells:
    amounts computed by hand (the oracle's pins use the same rows)."""
    from paper_1305_3417_gb300 import vof
    alpha, want, passes, gvol = ROWS[row]
    n = len(alpha)
    m = I.hex_mesh((n, 1, 1), length=(1.0, 1.0 / n, 1.0 / n))
    ctx = vof.VofContext(m, precision=precision)
    V = float(ctx.geometry()[1].cpu().numpy()[0])
    ta = T(torch, np.array(alpha, float))
    st = ctx.update(ta, torch.zeros(m.n_faces, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert ctx.status() == 0
    np.testing.assert_allclose(ta.cpu().numpy(), want, rtol=0, atol=1e-14)
    S = vof.S
    assert st[S["bound_passes"]] == passes
    assert st[S["bound_global"]] == pytest.approx(gvol * V, rel=1e-12, abs=1e-300)
    ctx.close()


# -------------------------------------------- 96^3 Kuhn tetrahedra, full size

def test_tet96_full_size_sampled(torch, oracle_lib):
    """One mixed-precision step of the 96^3 Kuhn tetrahedral single-vortex
    workload (5.3 M cells) in the benchmark's launch configuration, compared
    with the oracle on sampled cells: the oracle reconstructs the stencil
    cells and corrects and fluxes the faces it needs."""
    from paper_1305_3417_gb300 import vof
    O = oracle_lib
    w = I.make_workload("vortex_tet")
    m = w.mesh
    ctx = vof.VofContext(m, precision=vof.MIXED, bound=False)
    om = O.OracleMesh(m)
    F, U, dt = w.step_inputs(0)
    ta = T(torch, w.alpha0)
    stats = ctx.advect(ta, T(torch, U), T(torch, F), dt).cpu().numpy()
    assert ctx.status() == 0
    a1 = ta.cpu().numpy()
    rng = np.random.default_rng(23)
    cls = om.classify_faces(w.alpha0)
    band = np.flatnonzero((cls == 2) & (F != 0))
    assert stats[7] == band.size
    band_cells = np.unique(np.concatenate([m.owner[band], m.neighbour[band[band < m.n_internal]]]))
    cells = np.unique(np.concatenate([rng.choice(band_cells, 60, replace=False),
                                      rng.choice(m.n_cells, 30, replace=False)]))
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
    print(f"96^3 tets, mixed, one step: max |d alpha| on {cells.size} sampled cells = {worst:.2e}")
    assert worst < 2e-5
    assert abs(stats[1] - stats[0]) / stats[0] < 1e-12
    ctx.close()
