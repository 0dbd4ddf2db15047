"""vof_reconstruct_static -- the reconstruction for callers that cannot allocate
device memory when they call it (a host framework that owns all device
allocations, a real-time loop that forbids cudaMalloc after start-up) --
gives the same normals, plane offsets and flags as vof_reconstruct, on two
calls in a row (the second call finds the shared static list left over from
the first and must clear it).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["fp64", "mixed", "mixed_guess"])
def test_reconstruct_static_matches_reconstruct(form):
    """Every form of the reconstruction over the static list: plain FP64,
    mixed precision, and mixed with a learned initial guess (whose guesses
    are indexed by position in the static list)."""
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1305_3417_gb300 import build, mlp, vof
    build.build()
    L = vof.lib()
    fn = L.vof_reconstruct_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 6
    w = I.make_workload("deform3d", n=20)
    ctx = vof.VofContext(w.mesh, precision=vof.FP64 if form == "fp64" else vof.MIXED)
    net = None
    if form == "mixed_guess":
        net = vof.Mlp(mlp.init_params(61), max_batch=1 << 14)
        vof.vof_set_guess(ctx.h, net)
    nc = w.mesh.n_cells
    fields = [w.alpha0, np.clip(w.alpha0 + 0.3 * np.sin(np.arange(nc)), 0.0, 1.0)]
    for a in fields:  # two calls in a row, different fields
        ta = torch.from_numpy(a.copy()).cuda()
        n_ref, d_ref, fl_ref, _ = ctx.reconstruct(ta)
        n = torch.full((3 * nc,), 7.0, dtype=torch.float64, device="cuda")
        d = torch.full((nc,), 7.0, dtype=torch.float64, device="cuda")
        fl = torch.full((nc,), 99, dtype=torch.uint8, device="cuda")
        rc = fn(ctx.h, vof._ptr(ta), vof._ptr(n), vof._ptr(d), vof._ptr(fl), vof._stream(None))
        assert rc == 0, vof.vof_error_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(fl, fl_ref)
        assert (n - n_ref).abs().max().item() < 1e-12
        assert (d - d_ref).abs().max().item() < 1e-12
        assert int((fl & vof.ORIENTED).count_nonzero()) > 10
    assert ctx.status() == 0
    # argument errors come back as codes, not faults
    assert fn(None, vof._ptr(ta), vof._ptr(n), vof._ptr(d), vof._ptr(fl), vof._stream(None)) == -1
    if net is not None:
        vof.vof_set_guess(ctx.h, None)
        net.close()
    ctx.close()
