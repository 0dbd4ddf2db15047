"""Local adaptive refinement of the octree meshes and the geometric mapping of
the volume fraction onto the new mesh (Sec. 3, Alg. 2).

The refinement cycle (host): the cells of the current octree mesh whose
volume fraction marks them as interface cells are stamped on the finest
lattice, a distance field to them is taken, and a new octree of the same
lattice is built that splits every cell lying within `band` of its own sizes
of them (then 2:1 face-balanced).  Alg. 2's absolute cell map is then the set
of (new cell, old cell) pairs that share volume -- on one lattice every such
pair is nested, the new cell inside the old one (refined or kept) or the old
one inside the new (un-refined) -- which vof_remap turns into volume
fractions on the device: the new cell's part of the old cell's PLIC
polyhedron (kernels of libvof).  The host side here only decides where to
refine and lists the pairs.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


def interface_voxels(mesh, alpha, eps: float = 1e-9) -> np.ndarray:
    """(N, N, N) mask of the finest-lattice voxels of interface cells."""
    cm = mesh.octree["cmap"]
    a = np.asarray(alpha)
    return ((a > eps) & (a < 1.0 - eps))[cm]


def refine_near_interface(mesh, alpha, band: float = 3.0, eps: float = 1e-9):
    """A new octree on the lattice of `mesh` refined (to the same number of
    levels) wherever a cell's centre lies within band * (its size) of the
    centre of an interface voxel of the current field."""
    from scipy import ndimage
    ot = mesh.octree
    N, levels, n0 = ot["N"], ot["levels"], ot["n0"]
    mark = interface_voxels(mesh, alpha, eps)
    if not mark.any():
        dist = np.full(mark.shape, np.inf, np.float32)
    else:
        dist = ndimage.distance_transform_edt(~mark).astype(np.float32)

    def refine(L, i, j, k, s):
        c = np.minimum(np.stack([i, j, k], 1) * s + s // 2, N - 1)
        return dist[c[:, 0], c[:, 1], c[:, 2]] <= band * s

    return I.octree_mesh(n0, levels, refine=refine)


def cell_pairs(dst, src):
    """Alg. 2's cell map as a CSR over the destination cells: (ptr, src cell),
    every source cell sharing volume with each destination cell (ascending)."""
    a = dst.octree["cmap"].ravel().astype(np.int64)
    b = src.octree["cmap"].ravel().astype(np.int64)
    key = np.unique(a * src.n_cells + b)
    d, s = key // src.n_cells, key % src.n_cells
    ptr = np.zeros(dst.n_cells + 1, np.int64)
    np.add.at(ptr, d + 1, 1)
    ptr = np.cumsum(ptr)
    return ptr.astype(np.int32), s.astype(np.int32)


class AmrCase:
    """The deformation case on a dynamically refined octree: steps through a
    VofContext, re-refining every `every` steps around the current interface
    and mapping the volume fraction geometrically (vof_remap) onto the new
    mesh.  The step inputs of each mesh come from the seeded generator."""

    def __init__(self, n0: int = 16, levels: int = 2, band: float = 3.0, co: float = 0.5, precision: int = 0,
                 every: int = 4, device: int = 0, center=(0.35, 0.35, 0.35), R: float = 0.15):
        import torch
        from . import vof
        self.torch, self.vof = torch, vof
        self.band, self.every, self.precision, self.device = band, every, precision, device
        self.field = I.deformation_field(3.0)
        self.mesh = I.octree_mesh(n0, levels, center, R, band)
        a0 = I.sampled_fraction(self.mesh, I.sphere_sdf(center, R))
        umax = float(np.sqrt((I.cell_velocity(self.mesh, self.field.u) ** 2).sum(0)).max())
        self.dt = co * self.mesh.h / umax
        self.center, self.R = center, R
        self._setup(self.mesh)
        self.alpha = torch.from_numpy(a0).cuda(device)
        self.t, self.steps, self.remaps = 0.0, 0, 0
        self.mass_change = []   # relative volume change of each remap

    def _setup(self, mesh):
        vof, torch = self.vof, self.torch
        self.ctx = vof.VofContext(mesh, precision=self.precision, device=self.device)
        self.Fs = torch.from_numpy(I.face_flux_stokes(mesh, self.field.A)).cuda(self.device)
        self.Us = torch.from_numpy(np.ascontiguousarray(I.cell_velocity(mesh, self.field.u)).reshape(-1)).cuda(
            self.device)
        self.vc = self.ctx.geometry()[1]

    def volume(self) -> float:
        return float((self.vc * self.alpha).sum())

    def step(self, t_end: float, stats=None):
        f = self.field
        dt = min(self.dt, t_end - self.t)
        tf = (f.tau_int(self.t + dt) - f.tau_int(self.t)) / dt
        self.ctx.advect(self.alpha, self.Us * f.tau(self.t + 0.5 * dt), self.Fs * tf, dt, stats)
        self.t += dt
        self.steps += 1

    def remap(self):
        """One refinement cycle: the new mesh around the current interface and
        the volume fraction mapped onto it by Alg. 2 (on the device)."""
        vof, torch = self.vof, self.torch
        n, d, fl, _ = self.ctx.reconstruct(self.alpha)
        a_host = self.alpha.cpu().numpy()
        new = refine_near_interface(self.mesh, a_host, self.band)
        ptr, src = cell_pairs(new, self.mesh)
        old_ctx, old_mesh, old_alpha, v0 = self.ctx, self.mesh, self.alpha, self.volume()
        self.mesh = new
        self._setup(new)
        self.alpha = torch.zeros(new.n_cells, dtype=torch.float64, device=old_alpha.device)
        vof.vof_remap(self.ctx.h, old_ctx.h, old_alpha, n, d, fl, torch.from_numpy(ptr).cuda(self.device),
                      torch.from_numpy(src).cuda(self.device), self.alpha)
        torch.cuda.synchronize()
        old_ctx.close()
        self.remaps += 1
        self.mass_change.append(self.volume() / v0 - 1.0)
        return old_mesh

    def run(self, t_end: float, stats=None):
        while self.t < t_end - 1e-12:
            if self.steps and self.steps % self.every == 0:
                self.remap()
            self.step(t_end, stats)
