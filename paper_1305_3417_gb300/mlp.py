"""Training data and training loop of the initial-guess network.

Samples are interface cells of seeded synthetic fields (random spheres and
planes) on a mesh; features come from vof_mlp_features, targets from the
FP64 reconstruction of the same context (the NAG normal and the offset s = (d -
d_min)/(d_max - d_min) over the cell's points).  Training runs on the GPU with
the library's forward, backward and Adam kernels.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I
from . import vof


def init_params(seed: int = 1306) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, flat layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, IN, OUT = vof.MLP_HID, vof.MLP_IN, vof.MLP_OUT
    parts = []
    for shape in [(IN, H), (H,), (H, H), (H,), (H, OUT), (OUT,)]:
        if len(shape) == 2:
            lim = np.sqrt(6.0 / shape[0])
            parts.append(rng.uniform(-lim, lim, shape))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def random_fields(mesh, n_fields: int, seed: int = 1306):
    """Volume fractions of random spheres (R in [0.08, 0.3]) and planes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_fields):
        if rng.random() < 0.6:
            R = float(rng.uniform(0.08, 0.3))
            c = rng.uniform(0.2, 0.8, 3)
            out.append(I.sampled_fraction(mesh, I.sphere_sdf(tuple(c), R), m=6))
        else:
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            x0 = rng.uniform(0.3, 0.7, 3)
            out.append(I.sampled_fraction(mesh, lambda x, _n=nrm, _x=x0: (x - _x) @ _n, m=6))
    return out


def random_fields_device(ctx, mesh, n_fields: int, seed: int = 1306, levels: int = 3):
    """As random_fields, with the volume fractions computed on the device by
    vof_evsd (the ball's volume in each cell, R19): spheres directly, planes
    as the boundary of a ball of radius 1e3 whose surface passes through the
    plane's point (its pieces are cut by the tangent plane there)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    vc = ctx.geometry()[1]
    out = []
    buf = torch.zeros(mesh.n_cells, dtype=torch.float64, device=vc.device)
    for _ in range(n_fields):
        if rng.random() < 0.6:
            R = float(rng.uniform(0.08, 0.3))
            c = rng.uniform(0.2, 0.8, 3)
            ball = (float(c[0]), float(c[1]), float(c[2]), R)
        else:
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            x0 = rng.uniform(0.3, 0.7, 3)
            c = x0 - 1e3 * nrm
            ball = (float(c[0]), float(c[1]), float(c[2]), 1e3)
        vof.vof_evsd(ctx.h, None, None, None, ball, levels, buf)
        out.append(torch.clamp(buf / vc, 0.0, 1.0).cpu().numpy())
    return out


def samples(ctx, mesh, fields):
    """(features [n x 33], targets [n x 4]) on the device for the oriented
    interface cells of every field, targets from the context's reconstruction."""
    import torch
    pts = mesh.points
    feats, targs = [], []
    for a in fields:
        ta = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        n, d, fl, _ = ctx.reconstruct(ta)
        fl = fl.cpu().numpy()
        cells = np.flatnonzero(fl & 2).astype(np.int32)
        if cells.size == 0:
            continue
        nn = n.view(3, -1).cpu().numpy()[:, cells].T
        dd = d.cpu().numpy()[cells]
        proj = np.einsum("ckd,cd->ck", pts[mesh.cell_verts[cells]], nn)
        lo, hi = proj.min(1), proj.max(1)
        s = (dd - lo) / (hi - lo)
        tc = torch.from_numpy(cells).cuda()
        f = torch.empty((cells.size, vof.MLP_IN), dtype=torch.float32, device="cuda")
        vof.vof_mlp_features(ctx.h, ta, tc, cells.size, f)
        feats.append(f)
        targs.append(torch.from_numpy(np.concatenate([nn, s[:, None]], 1).astype(np.float32)).cuda())
    return torch.cat(feats), torch.cat(targs)


def train(net, feat, targ, epochs: int = 30, batch: int = 4096, lr: float = 2e-3, seed: int = 1306):
    """Adam over shuffled mini-batches; returns the mean loss of each epoch."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = feat.shape[0]
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot, cnt = 0.0, 0
        for o in range(0, n - batch + 1, batch):
            idx = perm[o:o + batch]
            tot += net.train_step(feat[idx].contiguous(), targ[idx].contiguous(), lr) * batch
            cnt += batch
        hist.append(tot / max(cnt, 1))
    return hist
