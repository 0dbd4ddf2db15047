"""Seeded synthetic inputs for the geometric VoF advection step.

This module builds the data that the method consumes; it computes no step of
the method itself.  Both the CUDA path and the CPU oracle receive the arrays
made here, and neither is imported by this module.

* Meshes in the unstructured face-based form the paper describes (Sec. 2: points
  stored once, a face is an ordered list of point indices whose right-hand
  normal points from the owner to the neighbour, owner/neighbour per face,
  internal faces first, then boundary faces with outward normals):
  uniform and jittered hexahedral boxes, and the Kuhn six-tetrahedra split of
  a hexahedral lattice.
* Initial volume fractions: exact disc/rectangle areas on uniform 2D meshes,
  otherwise a Jacobian-weighted midpoint rule over each cell's trilinear
  (hexahedron) or affine (tetrahedron) parametrisation.
* Volumetric face fluxes that are discretely divergence-free (Eq.
  discretedivergence) by construction: F_f is the circulation of a vector
  potential around the face's edge loop (Stokes), with one Gauss-Legendre
  integral per unique edge, so that every edge term enters its two faces with
  opposite signs.
* Cell-centred velocities of the analytic fields of the paper's test cases
  (Sec. 5.2: translation, deformation Eq. deformation-test-case) and of the
  2D single vortex and solid-body rotation.

Random numbers come from numpy's PCG64 generator seeded per workload.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

__all__ = [
    "Mesh", "hex_mesh", "kuhn_tet_mesh", "disc_rect_area", "disc_fraction_2d",
    "sampled_fraction", "sphere_sdf", "cylinder_sdf", "Field", "translation_field", "diagonal_shuttle_field", "periodic_shear_field", "shear_field",
    "deformation_field", "single_vortex_field", "rotation_field",
    "face_flux_stokes", "cell_velocity", "Workload", "make_workload",
    "concat_meshes", "BatchCase", "Batch", "make_batch",
]


@dataclasses.dataclass
class Mesh:
    points: np.ndarray      # (n_points, 3) float64
    face_ptr: np.ndarray    # (n_faces + 1,) int32
    face_pts: np.ndarray    # (face_ptr[-1],) int32
    owner: np.ndarray       # (n_faces,) int32
    neighbour: np.ndarray   # (n_internal,) int32
    n_cells: int
    cell_verts: np.ndarray  # (n_cells, 8 or 4) int32 -- generator's own record
    h: float                # nominal lattice spacing
    dim: int
    kind: str
    shape: tuple = ()
    wall: np.ndarray | None = None   # (n_faces - n_internal,) uint8: 1 = wall (no normal flow)
    octree: dict | None = None       # octree meshes: lattice size N, levels, per cell level / origin /
                                     # size in finest units, and the finest-lattice cell map
    # periodic meshes: period vectors (3, 3) as rows; per point the master point
    # it is an image of and the periods between them (P = P_master + image @
    # period); per boundary face the periodic internal face it is the
    # neighbour's copy of, or -1
    period: np.ndarray | None = None
    point_master: np.ndarray | None = None   # (n_points,) int32
    point_image: np.ndarray | None = None    # (n_points, 3) int8
    face_image: np.ndarray | None = None     # (n_faces - n_internal,) int32

    @property
    def n_points(self) -> int:
        return int(self.points.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.owner.shape[0])

    @property
    def n_internal(self) -> int:
        return int(self.neighbour.shape[0])

    def wall_flags(self) -> np.ndarray:
        if self.wall is None:
            return np.ones(self.n_faces - self.n_internal, np.uint8)
        return np.ascontiguousarray(self.wall, np.uint8)

    def soa_points(self):
        p = np.ascontiguousarray(self.points.T)
        return p[0].copy(), p[1].copy(), p[2].copy()


# --------------------------------------------------------------------------
# Hexahedral boxes
# --------------------------------------------------------------------------

def hex_mesh(n, length=(1.0, 1.0, 1.0), jitter: float = 0.0, seed: int | None = None,
             dim: int = 3, open_sides: tuple = (), periodic: str = "") -> Mesh:
    """Box [0,lx]x[0,ly]x[0,lz] split into nx*ny*nz hexahedra.

    Boundary faces are walls (no normal flow) except on the sides listed in
    ``open_sides`` (any of "x-", "x+", "y-", "y+", "z-", "z+").

    ``periodic`` (any of "x", "y", "z") joins the two sides normal to each
    listed axis: the points of the high side are images of the low side's
    (one period along the axis), a face of the high side becomes an internal
    face from its owner to the low side's cell across the period, and the low
    side's face is that cell's copy of it (``face_image``).

    ``jitter`` moves every point that lies on no boundary plane by an
    independent uniform offset in [-jitter*h, jitter*h] per coordinate
    (h = lx/nx), drawn from PCG64(seed); on a periodic axis the low side's
    points are moved too and the high side's images follow them.  With dim=2
    the mesh is one cell thick and only x, y of points off the x/y boundary
    planes are moved.
    """
    nx, ny, nz = (int(v) for v in n)
    lx, ly, lz = (float(v) for v in length)
    h = lx / nx
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    zs = np.linspace(0.0, lz, nz + 1)
    # point id p(i,j,k) = i + (nx+1)*(j + (ny+1)*k)
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    pid = (I + (nx + 1) * (J + (ny + 1) * K)).astype(np.int64)
    npts = (nx + 1) * (ny + 1) * (nz + 1)
    pts = np.empty((npts, 3))
    pts[pid.ravel(), 0] = xs[I.ravel()]
    pts[pid.ravel(), 1] = ys[J.ravel()]
    pts[pid.ravel(), 2] = zs[K.ravel()]
    per = [ax in periodic for ax in "xyz"]
    if dim == 2 and per[2]:
        raise ValueError("a one-cell-thick mesh is not periodic across its thickness")
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))

        def free(L, n_, p_):
            return (L < n_) if p_ else ((L > 0) & (L < n_))
        if dim == 3:
            inner = free(I, nx, per[0]) & free(J, ny, per[1]) & free(K, nz, per[2])
            ids = np.sort(pid[inner])
            pts[ids] += rng.uniform(-jitter * h, jitter * h, size=(ids.size, 3))
        else:
            inner = free(I, nx, per[0]) & free(J, ny, per[1])
            ids = np.sort(pid[inner])
            pts[ids, :2] += rng.uniform(-jitter * h, jitter * h, size=(ids.size, 2))
    period = np.diag([lx, ly, lz]) * np.array(per, float)[:, None]
    img = np.stack([(I == nx) & per[0], (J == ny) & per[1], (K == nz) & per[2]], -1).astype(np.int8)
    mI, mJ, mK = np.where(img[..., 0] > 0, 0, I), np.where(img[..., 1] > 0, 0, J), np.where(img[..., 2] > 0, 0, K)
    master = (mI + (nx + 1) * (mJ + (ny + 1) * mK)).astype(np.int64)
    point_master = np.empty(npts, np.int32)
    point_image = np.zeros((npts, 3), np.int8)
    point_master[pid.ravel()] = master.ravel()
    point_image[pid.ravel()] = img.reshape(-1, 3)
    if any(per):
        # images sit one period from their masters (jitter included)
        pts[:] = pts[point_master] + point_image.astype(float) @ period

    def P(i, j, k):
        return (i + (nx + 1) * (j + (ny + 1) * k)).astype(np.int64)

    def C(i, j, k):
        return (i + nx * (j + ny * k)).astype(np.int64)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()

    def xface(i, j, k):      # +x normal at x-plane index i
        return np.stack([P(i, j, k), P(i, j + 1, k), P(i, j + 1, k + 1), P(i, j, k + 1)], 1)

    def yface(i, j, k):      # +y normal at y-plane index j
        return np.stack([P(i, j, k), P(i, j, k + 1), P(i + 1, j, k + 1), P(i + 1, j, k)], 1)

    def zface(i, j, k):      # +z normal at z-plane index k
        return np.stack([P(i, j, k), P(i + 1, j, k), P(i + 1, j + 1, k), P(i, j + 1, k)], 1)

    own, nei, fps = [], [], []
    m = ci < nx - 1
    own.append(C(ci[m], cj[m], ck[m])); nei.append(C(ci[m] + 1, cj[m], ck[m]))
    fps.append(xface(ci[m] + 1, cj[m], ck[m]))
    m = cj < ny - 1
    own.append(C(ci[m], cj[m], ck[m])); nei.append(C(ci[m], cj[m] + 1, ck[m]))
    fps.append(yface(ci[m], cj[m] + 1, ck[m]))
    m = ck < nz - 1
    own.append(C(ci[m], cj[m], ck[m])); nei.append(C(ci[m], cj[m], ck[m] + 1))
    fps.append(zface(ci[m], cj[m], ck[m] + 1))
    own_i = np.concatenate(own); nei_i = np.concatenate(nei); fp_i = np.concatenate(fps)
    order = np.lexsort((nei_i, own_i))          # upper-triangular (owner, neighbour) order
    own_i, nei_i, fp_i = own_i[order], nei_i[order], fp_i[order]
    # periodic internal faces: each high side face, from its owner to the low
    # side's cell across the period, after the others (owner order per axis)
    per_block = {}
    pown, pnei, pfp = [], [], []
    nxt = own_i.size
    for ax in range(3):
        if not per[ax]:
            continue
        m = (ci, cj, ck)[ax] == (nx, ny, nz)[ax] - 1
        lo = [ci[m], cj[m], ck[m]]
        lo[ax] = np.zeros_like(lo[ax])
        hi_idx = [ci[m], cj[m], ck[m]]
        hi_idx[ax] = hi_idx[ax] + 1
        pown.append(C(ci[m], cj[m], ck[m])); pnei.append(C(*lo))
        pfp.append((xface, yface, zface)[ax](*hi_idx))
        per_block[ax] = (nxt, pnei[-1])           # first face index, neighbours in order
        nxt += int(m.sum())
    if pown:
        own_i = np.concatenate([own_i] + pown); nei_i = np.concatenate([nei_i] + pnei)
        fp_i = np.concatenate([fp_i] + pfp)

    bown, bfp = [], []
    # x-, x+, y-, y+, z-, z+ ; reversed point order gives the outward normal on the low side
    m = ci == 0
    bown.append(C(ci[m], cj[m], ck[m])); bfp.append(xface(ci[m], cj[m], ck[m])[:, ::-1])
    m = ci == nx - 1
    bown.append(C(ci[m], cj[m], ck[m])); bfp.append(xface(ci[m] + 1, cj[m], ck[m]))
    m = cj == 0
    bown.append(C(ci[m], cj[m], ck[m])); bfp.append(yface(ci[m], cj[m], ck[m])[:, ::-1])
    m = cj == ny - 1
    bown.append(C(ci[m], cj[m], ck[m])); bfp.append(yface(ci[m], cj[m] + 1, ck[m]))
    m = ck == 0
    bown.append(C(ci[m], cj[m], ck[m])); bfp.append(zface(ci[m], cj[m], ck[m])[:, ::-1])
    m = ck == nz - 1
    bown.append(C(ci[m], cj[m], ck[m])); bfp.append(zface(ci[m], cj[m], ck[m] + 1))
    bsorted = []
    wall = []
    fimg = []
    for side, o, f in zip(("x-", "x+", "y-", "y+", "z-", "z+"), bown, bfp):
        ax = "xyz".index(side[0])
        if per[ax] and side[1] == "+":
            continue                              # now the periodic internal faces
        s = np.argsort(o, kind="stable")
        bsorted.append((o[s], f[s]))
        wall.append(np.full(o.size, 0 if (side in open_sides or per[ax]) else 1, np.uint8))
        if per[ax]:
            # the low side's face of cell o is the neighbour's copy of the
            # periodic face whose neighbour is o
            f0, nb = per_block[ax]
            where = np.full(nx * ny * nz, -1, np.int64)
            where[nb] = f0 + np.arange(nb.size)
            fimg.append(where[o[s]])
        else:
            fimg.append(np.full(o.size, -1, np.int64))
    b_own = np.concatenate([b[0] for b in bsorted])
    b_fp = np.concatenate([b[1] for b in bsorted])

    owner = np.concatenate([own_i, b_own]).astype(np.int32)
    face_pts = np.concatenate([fp_i, b_fp]).reshape(-1).astype(np.int32)
    face_ptr = (4 * np.arange(owner.size + 1)).astype(np.int32)
    cell_ids = C(ci, cj, ck)
    cv = np.empty((nx * ny * nz, 8), np.int64)
    for t, (a, b, c) in enumerate([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                                   (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]):
        cv[cell_ids, t] = P(ci + a, cj + b, ck + c)
    mesh = Mesh(pts, face_ptr, face_pts, owner, nei_i.astype(np.int32), nx * ny * nz,
                cv.astype(np.int32), h, dim, "hex", (nx, ny, nz), np.concatenate(wall))
    if any(per):
        mesh.period = period
        mesh.point_master = point_master
        mesh.point_image = point_image
        mesh.face_image = np.concatenate(fimg).astype(np.int32)
    return mesh


# --------------------------------------------------------------------------
# Static octree: a cubic base lattice refined near a sphere, 2:1 face-balanced
# --------------------------------------------------------------------------

def octree_mesh(n0: int = 64, levels: int = 2, center=(0.35, 0.35, 0.35), R: float = 0.15,
                band: float = 3.0, refine=None) -> Mesh:
    """Unit cube: an n0^3 lattice whose cells are split into 8 wherever the cell
    centre lies within band * (the cell's size) of the sphere |x - center| = R,
    level by level down to `levels` splits, then split further until every
    two face neighbours differ by at most one level (2:1 face balance).

    The result is a conforming polyhedral mesh: every cell is an axis-aligned
    box; a side facing four finer cells is four faces (one per finer cell); a
    face gets the midpoints of its edges that are corners of smaller cells
    (hanging points) as extra polygon points, so faces have 4 to 8 points.  A
    face is listed once, owned by the cell whose side it is (the finer of the
    two, or the lower one across +x/+y/+z between equal cells), with its points
    counter-clockwise about the owner's outward normal.  Boundary faces are
    walls.  cell_verts holds each box's 8 corners in the hex corner order.
    Integer lattice coordinates are in units of the finest size 1/(n0 2^levels).

    ``refine(L, i, j, k, s)``, if given, replaces the sphere criterion: a mask
    of the level-L cells (integer coordinates i, j, k at that level, size s in
    finest units) to split.  The returned mesh carries ``octree``: the lattice
    size N, the levels, per cell its level and origin and size (finest units),
    and the (N, N, N) map from finest-lattice voxels to cells.
    """
    N = n0 << levels
    cen = np.asarray(center, float)

    def near(L, i, j, k):
        s = 1 << (levels - L)
        if refine is not None:
            return np.asarray(refine(L, i, j, k, s), bool)
        c = (np.stack([i, j, k], 1) * s + 0.5 * s) / N
        d = np.abs(np.sqrt(((c - cen) ** 2).sum(1)) - R)
        return d <= band * s / N

    g = np.arange(n0)
    I, J, K = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
    leaves = {0: (I, J, K)}
    for L in range(levels):
        leaves.setdefault(L + 1, (np.zeros(0, np.int64),) * 3)
    kids = np.array([(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)])

    def split(L, m):
        i, j, k = leaves[L]
        ci, cj, ck = i[m], j[m], k[m]
        leaves[L] = (i[~m], j[~m], k[~m])
        ni = (2 * ci[:, None] + kids[None, :, 0]).ravel()
        nj = (2 * cj[:, None] + kids[None, :, 1]).ravel()
        nk = (2 * ck[:, None] + kids[None, :, 2]).ravel()
        pi, pj, pk = leaves[L + 1]
        leaves[L + 1] = (np.concatenate([pi, ni]), np.concatenate([pj, nj]), np.concatenate([pk, nk]))

    for L in range(levels):
        i, j, k = leaves[L]
        split(L, near(L, i, j, k))

    def level_map():
        lm = np.zeros((N, N, N), np.int8)
        for L in range(levels + 1):
            i, j, k = leaves[L]
            if i.size == 0:
                continue
            s = 1 << (levels - L)
            nL = N // s
            v = lm.reshape(nL, s, nL, s, nL, s).transpose(0, 2, 4, 1, 3, 5)
            v[i, j, k] = L
        return lm

    while True:                                   # 2:1 face balance
        lm = level_map()
        nb = np.zeros_like(lm)
        nb[1:] = np.maximum(nb[1:], lm[:-1]); nb[:-1] = np.maximum(nb[:-1], lm[1:])
        nb[:, 1:] = np.maximum(nb[:, 1:], lm[:, :-1]); nb[:, :-1] = np.maximum(nb[:, :-1], lm[:, 1:])
        nb[:, :, 1:] = np.maximum(nb[:, :, 1:], lm[:, :, :-1]); nb[:, :, :-1] = np.maximum(nb[:, :, :-1], lm[:, :, 1:])
        changed = False
        for L in range(levels - 1):
            i, j, k = leaves[L]
            if i.size == 0:
                continue
            s = 1 << (levels - L)
            nL = N // s
            bm = nb.reshape(nL, s, nL, s, nL, s).max(axis=(1, 3, 5))
            m = bm[i, j, k] >= L + 2
            if m.any():
                split(L, m)
                changed = True
        if not changed:
            break
    lm = level_map()

    # cells: every leaf, ordered by its origin (z, y, x)
    lv, ox, oy, oz, sz = [], [], [], [], []
    for L in range(levels + 1):
        i, j, k = leaves[L]
        s = 1 << (levels - L)
        lv.append(np.full(i.size, L)); ox.append(i * s); oy.append(j * s); oz.append(k * s)
        sz.append(np.full(i.size, s))
    lv, ox, oy, oz, sz = (np.concatenate(a).astype(np.int64) for a in (lv, ox, oy, oz, sz))
    order = np.lexsort((ox, oy, oz))
    lv, ox, oy, oz, sz = lv[order], ox[order], oy[order], oz[order], sz[order]
    nc = lv.size
    cmap = np.empty((N, N, N), np.int32)
    for L in range(levels + 1):
        sel = np.flatnonzero(lv == L)
        if sel.size == 0:
            continue
        s = 1 << (levels - L)
        nL = N // s
        v = cmap.reshape(nL, s, nL, s, nL, s).transpose(0, 2, 4, 1, 3, 5)
        v[ox[sel] // s, oy[sel] // s, oz[sel] // s] = sel[:, None, None, None]

    # points: the corners of the cells
    M = N + 1
    corner = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)])
    cx = ox[:, None] + corner[None, :, 0] * sz[:, None]
    cy = oy[:, None] + corner[None, :, 1] * sz[:, None]
    cz = oz[:, None] + corner[None, :, 2] * sz[:, None]
    key = (cx + M * (cy + M * cz)).ravel()
    uk, inv = np.unique(key, return_inverse=True)
    pmap = np.full(M * M * M, -1, np.int64)
    pmap[uk] = np.arange(uk.size)
    pts = np.stack([uk % M, (uk // M) % M, uk // (M * M)], 1).astype(float) / N
    cell_verts = inv.reshape(nc, 8).astype(np.int32)

    def pid(x, y, z):
        return pmap[x + M * (y + M * z)]

    # the six sides: (axis, +1/-1); the 4 corners of a side counter-clockwise
    # about the outward normal, as in hex_mesh's x/y/z faces
    def side_corners(ax, sgn, x0, y0, z0, s):
        if ax == 0:
            x = x0 + (s if sgn > 0 else 0)
            c = [(x, y0, z0), (x, y0 + s, z0), (x, y0 + s, z0 + s), (x, y0, z0 + s)]
        elif ax == 1:
            y = y0 + (s if sgn > 0 else 0)
            c = [(x0, y, z0), (x0, y, z0 + s), (x0 + s, y, z0 + s), (x0 + s, y, z0)]
        else:
            z = z0 + (s if sgn > 0 else 0)
            c = [(x0, y0, z), (x0 + s, y0, z), (x0 + s, y0 + s, z), (x0, y0 + s, z)]
        if sgn < 0:
            c = c[::-1]
        return [tuple(np.asarray(v) for v in p) for p in c]

    int_own, int_nei, int_pts, bnd_own, bnd_pts = [], [], [], [], []
    cells = np.arange(nc)
    for ax in range(3):
        for sgn in (1, -1):
            lo = (ox, oy, oz)[ax]
            if sgn > 0:
                edge = lo + sz >= N
                adj = lo + sz                     # first finest index beyond the side
            else:
                edge = lo == 0
                adj = lo - 1
            # the finest cell just outside the side, at the side's low corner
            ax_ = [ox, oy, oz]
            q = [a.copy() for a in ax_]
            q[ax] = np.where(edge, 0, adj)
            nlev = lm[q[0], q[1], q[2]].astype(np.int64)
            nidx = cmap[q[0], q[1], q[2]].astype(np.int64)
            emit_int = ~edge & ((nlev < lv) | ((nlev == lv) & (sgn > 0)))
            for sel, is_b in ((np.flatnonzero(edge), True), (np.flatnonzero(emit_int), False)):
                if sel.size == 0:
                    continue
                c4 = side_corners(ax, sgn, ox[sel], oy[sel], oz[sel], sz[sel])
                ids = []
                for t in range(4):
                    a, b = c4[t], c4[(t + 1) % 4]
                    ids.append(pid(*a))
                    half = (sz[sel] % 2 == 0)
                    mx, my, mz = ((a[0] + b[0]) // 2, (a[1] + b[1]) // 2, (a[2] + b[2]) // 2)
                    mid = np.where(half, pid(mx, my, mz), -1)
                    ids.append(mid)
                F = np.stack(ids, 1)              # (f, 8): corner, midpoint or -1, ...
                if is_b:
                    bnd_own.append(cells[sel]); bnd_pts.append(F)
                else:
                    int_own.append(cells[sel]); int_nei.append(nidx[sel]); int_pts.append(F)
    own_i = np.concatenate(int_own); nei_i = np.concatenate(int_nei); F_i = np.concatenate(int_pts)
    o = np.lexsort((nei_i, own_i))
    own_i, nei_i, F_i = own_i[o], nei_i[o], F_i[o]
    own_b = np.concatenate(bnd_own); F_b = np.concatenate(bnd_pts)
    o = np.argsort(own_b, kind="stable")
    own_b, F_b = own_b[o], F_b[o]
    Fall = np.concatenate([F_i, F_b])
    cnt = (Fall >= 0).sum(1)
    face_ptr = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    face_pts = Fall[Fall >= 0].astype(np.int32)          # row-major: each face's points in order
    owner = np.concatenate([own_i, own_b]).astype(np.int32)
    octree = {"N": N, "levels": levels, "n0": n0, "level": lv, "origin": np.stack([ox, oy, oz], 1),
              "size": sz, "cmap": cmap}
    return Mesh(pts, face_ptr, face_pts, owner, nei_i.astype(np.int32), nc, cell_verts, 1.0 / N, 3, "octree",
                (n0, n0, n0), np.ones(own_b.size, np.uint8), octree)


# --------------------------------------------------------------------------
# Kuhn split of a hexahedral lattice into tetrahedra
# --------------------------------------------------------------------------

def _tet_signed6(p, t):
    a, b, c, d = (p[t[:, i]] for i in range(4))
    return np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a))


def kuhn_tet_mesh(n, length=(1.0, 1.0, 1.0), jitter: float = 0.0,
                  seed: int | None = None) -> Mesh:
    """Each hexahedron of an n^3 lattice split into the six tetrahedra that share
    its (0,0,0)-(1,1,1) diagonal; the split is conforming across hexahedra.
    Interior points are jittered as in :func:`hex_mesh`."""
    base = hex_mesh(n, length, jitter, seed, dim=3)
    nx, ny, nz = base.shape
    pts = base.points
    cv = base.cell_verts.astype(np.int64)       # corners (000,100,110,010,001,101,111,011)
    corner = {(0, 0, 0): 0, (1, 0, 0): 1, (1, 1, 0): 2, (0, 1, 0): 3,
              (0, 0, 1): 4, (1, 0, 1): 5, (1, 1, 1): 6, (0, 1, 1): 7}
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for pa in perms:
        v = [0, 0, 0]
        path = [corner[tuple(v)]]
        for ax in pa:
            v[ax] = 1
            path.append(corner[tuple(v)])
        tets.append(cv[:, path])
    tet = np.stack(tets, 1).reshape(-1, 4)      # hexahedron-major, then permutation
    vol6 = _tet_signed6(pts, tet)
    neg = vol6 < 0
    tet[neg] = tet[neg][:, [0, 2, 1, 3]]
    if np.any(np.abs(vol6) <= 0):
        raise ValueError("degenerate tetrahedron in Kuhn split")
    nt = tet.shape[0]
    # outward faces of a positively oriented tet (a,b,c,d)
    loc = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
    inst = tet[:, loc].reshape(-1, 3)           # (4*nt, 3)
    cell_of = np.repeat(np.arange(nt, dtype=np.int64), 4)
    s = np.sort(inst, axis=1)
    N = np.int64(pts.shape[0])
    key = s[:, 0] + N * (s[:, 1] + N * s[:, 2])
    order = np.argsort(key, kind="stable")
    ks = key[order]
    start = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    cnt = np.diff(np.r_[start, ks.size])
    if np.any(cnt > 2):
        raise ValueError("non-manifold face in tetrahedral mesh")
    pair = start[cnt == 2]
    i0, i1 = order[pair], order[pair + 1]
    c0, c1 = cell_of[i0], cell_of[i1]
    own_inst = np.where(c0 < c1, i0, i1)
    own = np.minimum(c0, c1)
    nei = np.maximum(c0, c1)
    o = np.lexsort((nei, own))
    own, nei, own_inst = own[o], nei[o], own_inst[o]
    single = order[start[cnt == 1]]
    b_own = cell_of[single]
    o = np.argsort(b_own, kind="stable")
    single, b_own = single[o], b_own[o]
    owner = np.concatenate([own, b_own]).astype(np.int32)
    face_pts = np.concatenate([inst[own_inst], inst[single]]).reshape(-1).astype(np.int32)
    face_ptr = (3 * np.arange(owner.size + 1)).astype(np.int32)
    return Mesh(pts, face_ptr, face_pts, owner, nei.astype(np.int32), nt,
                tet.astype(np.int32), base.h, 3, "tet", base.shape)


# --------------------------------------------------------------------------
# Initial volume fractions
# --------------------------------------------------------------------------

def _circle_prim(x, R):
    """Antiderivative of sqrt(R^2 - x^2) on [-R, R]."""
    x = np.clip(x, -R, R)
    return 0.5 * (x * np.sqrt(np.maximum(R * R - x * x, 0.0)) + R * R * np.arcsin(x / R))


def disc_rect_area(cx, cy, R, x0, x1, y0, y1):
    """Exact area of disc((cx,cy),R) intersected with [x0,x1]x[y0,y1].

    The chord length L(X) = |[y0,y1] ^ [cy-s, cy+s]|, s = sqrt(R^2-(X-cx)^2), is a
    piecewise combination of constants and +-s between the abscissae where
    cy +- s crosses y0 or y1; each piece is integrated with the circle's
    antiderivative.  Scalar arguments."""
    a, b = max(x0, cx - R), min(x1, cx + R)
    if b <= a or y1 <= cy - R or y0 >= cy + R:
        return 0.0
    br = [a, b]
    for y in (y0, y1):
        dy = abs(y - cy)
        if dy < R:
            xb = math.sqrt(R * R - dy * dy)
            for xv in (cx - xb, cx + xb):
                if a < xv < b:
                    br.append(xv)
    br = sorted(br)
    area = 0.0
    for u, v in zip(br[:-1], br[1:]):
        if v <= u:
            continue
        xm = 0.5 * (u + v) - cx
        sm = math.sqrt(max(R * R - xm * xm, 0.0))
        top_is_circle = (cy + sm) < y1
        bot_is_circle = (cy - sm) > y0
        if (min(y1, cy + sm) - max(y0, cy - sm)) <= 0.0:
            continue
        S = float(_circle_prim(v - cx, R) - _circle_prim(u - cx, R))
        w = v - u
        top = S + cy * w if top_is_circle else y1 * w
        bot = (cy * w - S) if bot_is_circle else y0 * w
        area += top - bot
    return area


def disc_fraction_2d(mesh: Mesh, cx: float, cy: float, R: float) -> np.ndarray:
    """Exact cell fractions of a disc on a uniform one-cell-thick hex mesh; on a
    mesh periodic in x and y the disc is wrapped (the sum over its images one
    period away; a disc narrower than the box meets each cell in at most one)."""
    nx, ny, _ = mesh.shape
    h = mesh.h
    out = np.zeros(mesh.n_cells)
    if mesh.period is not None:
        Lx, Ly = mesh.period[0, 0], mesh.period[1, 1]
        cx, cy = cx % Lx if Lx else cx, cy % Ly if Ly else cy
        shifts = [(a * Lx, b * Ly) for a in ((-1, 0, 1) if Lx else (0,)) for b in ((-1, 0, 1) if Ly else (0,))]
    else:
        shifts = [(0.0, 0.0)]
    for j in range(ny):
        for i in range(nx):
            out[i + nx * j] = sum(disc_rect_area(cx + sx, cy + sy, R, i * h, (i + 1) * h, j * h, (j + 1) * h)
                                  for sx, sy in shifts) / (h * h)
    return out


def _wrapped_sphere_sdf(c, R):
    """Signed distance to a sphere on the periodic unit box (nearest image)."""
    c = np.asarray(c, float)

    def f(x):
        d = x - c
        d -= np.round(d)
        return np.sqrt((d ** 2).sum(-1)) - R
    return f


def sphere_sdf(c, R):
    c = np.asarray(c, float)
    return lambda x: np.sqrt(((x - c) ** 2).sum(-1)) - R


def cylinder_sdf(cx, cy, R):
    return lambda x: np.sqrt((x[..., 0] - cx) ** 2 + (x[..., 1] - cy) ** 2) - R


def _hex_shape(xi):
    """Trilinear shape functions and their derivatives at reference points xi (m,3),
    corner order (000,100,110,010,001,101,111,011)."""
    u, v, w = xi[:, 0], xi[:, 1], xi[:, 2]
    cs = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                   [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    fu = np.where(cs[None, :, 0] == 1, u[:, None], 1 - u[:, None])
    fv = np.where(cs[None, :, 1] == 1, v[:, None], 1 - v[:, None])
    fw = np.where(cs[None, :, 2] == 1, w[:, None], 1 - w[:, None])
    du = np.where(cs[None, :, 0] == 1, 1.0, -1.0)
    dv = np.where(cs[None, :, 1] == 1, 1.0, -1.0)
    dw = np.where(cs[None, :, 2] == 1, 1.0, -1.0)
    N = fu * fv * fw
    dN = np.stack([du * fv * fw, fu * dv * fw, fu * fv * dw], -1)   # (m,8,3)
    return N, dN


def sampled_fraction(mesh: Mesh, sdf: Callable, m: int = 8, chunk: int = 4096) -> np.ndarray:
    """Initial fraction by a midpoint rule: m^3 reference points per cell mapped
    through the cell's trilinear (hex) or affine (tet) parametrisation, each
    weighted by the map's Jacobian; a point counts if sdf < 0.  Cells whose
    centroid is farther from the surface than their circumradius are set to 0/1
    without sampling."""
    P = mesh.points
    cv = mesh.cell_verts
    X = P[cv]                                    # (nc, k, 3)
    cen = X.mean(1)
    rad = np.sqrt(((X - cen[:, None, :]) ** 2).sum(-1)).max(1)
    dc = sdf(cen)
    out = np.where(dc < 0, 1.0, 0.0)
    near = np.flatnonzero(np.abs(dc) <= rad * 1.0001)
    g = (np.arange(m) + 0.5) / m
    xi = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if cv.shape[1] == 8:                          # hexahedra and octree boxes
        N, dN = _hex_shape(xi)
        for s in range(0, near.size, chunk):
            ids = near[s:s + chunk]
            Xc = X[ids]                              # (b,8,3)
            x = np.einsum("qk,bkd->bqd", N, Xc)
            Jm = np.einsum("qke,bkd->bqde", dN, Xc)   # (b,q,3,3)
            det = np.linalg.det(Jm)
            ins = (sdf(x) < 0).astype(float)
            out[ids] = (det * ins).sum(1) / det.sum(1)
    else:
        srt = -np.sort(-xi, axis=1)                  # s1 >= s2 >= s3 in the unit simplex
        lam = np.stack([1 - srt[:, 0], srt[:, 0] - srt[:, 1], srt[:, 1] - srt[:, 2], srt[:, 2]], 1)
        for s in range(0, near.size, chunk):
            ids = near[s:s + chunk]
            x = np.einsum("qk,bkd->bqd", lam, X[ids])
            out[ids] = (sdf(x) < 0).mean(1)
    return out


# --------------------------------------------------------------------------
# Velocity fields with vector potentials (u = curl A)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Field:
    name: str
    u: Callable            # x (...,3) -> (...,3), spatial part
    A: Callable            # x (...,3) -> (...,3), vector potential of u
    tau: Callable          # time factor tau(t)
    tau_int: Callable      # antiderivative of tau


def translation_field(U):
    U = np.asarray(U, float)
    return Field("translation", lambda x: np.broadcast_to(U, x.shape).copy(),
                 lambda x: 0.5 * np.cross(np.broadcast_to(U, x.shape), x),
                 lambda t: 1.0, lambda t: t)


def deformation_field(T: float = 3.0):
    """Eq. deformation-test-case; A = (0, -(1/pi) s2x sin2y s2z, (1/pi) s2x s2y sin2z)."""
    pi = math.pi

    def u(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([2 * np.sin(pi * X) ** 2 * np.sin(2 * pi * Y) * np.sin(2 * pi * Z),
                         -np.sin(2 * pi * X) * np.sin(pi * Y) ** 2 * np.sin(2 * pi * Z),
                         -np.sin(2 * pi * X) * np.sin(2 * pi * Y) * np.sin(pi * Z) ** 2], -1)

    def A(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        s2x = np.sin(pi * X) ** 2
        return np.stack([np.zeros_like(X),
                         -(1 / pi) * s2x * np.sin(2 * pi * Y) * np.sin(pi * Z) ** 2,
                         (1 / pi) * s2x * np.sin(pi * Y) ** 2 * np.sin(2 * pi * Z)], -1)

    return Field("deformation", u, A, lambda t: math.cos(pi * t / T),
                 lambda t: (T / pi) * math.sin(pi * t / T))


def single_vortex_field(T: float = 8.0):
    pi = math.pi

    def u(x):
        X, Y = x[..., 0], x[..., 1]
        return np.stack([-np.sin(pi * X) ** 2 * np.sin(2 * pi * Y),
                         np.sin(2 * pi * X) * np.sin(pi * Y) ** 2, np.zeros_like(X)], -1)

    def A(x):
        X, Y = x[..., 0], x[..., 1]
        return np.stack([np.zeros_like(X), np.zeros_like(X),
                         -(1 / pi) * np.sin(pi * X) ** 2 * np.sin(pi * Y) ** 2], -1)

    return Field("single_vortex", u, A, lambda t: math.cos(pi * t / T),
                 lambda t: (T / pi) * math.sin(pi * t / T))


def diagonal_shuttle_field():
    """Uniform velocity (1,1,1) s(t) with s = +1 on [0, 1/2), -1 on [1/2, 3/2),
    +1 from 3/2: over [0, 2] a body at the centre of the unit box goes to the
    corner (1,1,1), back through the centre to (0,0,0) and returns to the
    centre (reading R21 of the paper's periodic translation case)."""
    U = np.array([1.0, 1.0, 1.0])

    def tau(t):
        return 1.0 if (t < 0.5 or t >= 1.5) else -1.0

    def tau_int(t):
        return t if t < 0.5 else (1.0 - t if t < 1.5 else t - 2.0)

    return Field("diagonal_shuttle", lambda x: np.broadcast_to(U, x.shape).copy(),
                 lambda x: 0.5 * np.cross(np.broadcast_to(U, x.shape), x), tau, tau_int)


def periodic_shear_field(T: float = 2.0):
    """u = (sin 2 pi y, sin 2 pi z, sin 2 pi x) cos(pi t / T): divergence-free
    and periodic on the unit box, with the periodic potential
    A = -(cos 2 pi z, cos 2 pi x, cos 2 pi y) / (2 pi)."""
    pi = math.pi

    def u(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([np.sin(2 * pi * Y), np.sin(2 * pi * Z), np.sin(2 * pi * X)], -1)

    def A(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return -np.stack([np.cos(2 * pi * Z), np.cos(2 * pi * X), np.cos(2 * pi * Y)], -1) / (2 * pi)

    return Field("periodic_shear", u, A, lambda t: math.cos(pi * t / T),
                 lambda t: (T / pi) * math.sin(pi * t / T))


def shear_field(T: float = 3.0, umax: float = 1.0, R: float = 0.5):
    """The shear test case (Sec. 4.2, Eq. shear-test-case, after Liovic et al.):
    the single vortex in x, y reversed, sin(2 pi y) sin^2(pi x) and
    -sin(2 pi x) sin^2(pi y), with the axial component umax (1 - r/R)^2 about
    the box's vertical axis (r the distance from x = y = 1/2), all times
    cos(pi t / T) (reading R22 of the garbled time factor of the third
    component).  Potential: A_z = sin^2(pi x) sin^2(pi y) / pi for the x, y
    part; A_x = -int_{1/2}^{y} umax (1 - r/R)^2 dy' in closed form for the
    axial part (with sqrt(a^2 + t^2) integrated as (t s + a^2 asinh(t/|a|))/2)."""
    pi = math.pi

    def u(x):
        X, Y = x[..., 0], x[..., 1]
        r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
        return np.stack([np.sin(2 * pi * Y) * np.sin(pi * X) ** 2,
                         -np.sin(2 * pi * X) * np.sin(pi * Y) ** 2,
                         umax * (1.0 - r / R) ** 2], -1)

    def A(x):
        X, Y = x[..., 0], x[..., 1]
        a, t = X - 0.5, Y - 0.5
        sq = np.sqrt(a * a + t * t)
        aa = np.abs(a)
        lg = np.where(aa > 0.0, a * a * np.arcsinh(t / np.where(aa > 0.0, aa, 1.0)), 0.0)
        G = 0.5 * (t * sq + lg)                       # int_0^t sqrt(a^2 + s^2) ds
        Iw = t - (2.0 / R) * G + (a * a * t + t ** 3 / 3.0) / (R * R)
        return np.stack([-umax * Iw, np.zeros_like(X),
                         (1 / pi) * np.sin(pi * X) ** 2 * np.sin(pi * Y) ** 2], -1)

    return Field("shear", u, A, lambda t: math.cos(pi * t / T),
                 lambda t: (T / pi) * math.sin(pi * t / T))


def rotation_field(omega, x0=(0.5, 0.5, 0.5)):
    om = np.asarray(omega, float)
    c = np.asarray(x0, float)
    return Field("rotation", lambda x: np.cross(np.broadcast_to(om, x.shape), x - c),
                 lambda x: -0.5 * ((x - c) ** 2).sum(-1)[..., None] * om,
                 lambda t: 1.0, lambda t: t)


_GL_X, _GL_W = np.polynomial.legendre.leggauss(8)
_GL_X = 0.5 * (_GL_X + 1.0)
_GL_W = 0.5 * _GL_W


def face_flux_stokes(mesh: Mesh, A: Callable, chunk: int = 1 << 20) -> np.ndarray:
    """F_f = circulation of A around face f (Stokes), signed along the face normal.
    One 8-point Gauss-Legendre integral per unique edge (low -> high point id);
    each face sums its edges with +-1, so per-cell sums cancel to round-off."""
    ptr = mesh.face_ptr.astype(np.int64)
    fp = mesh.face_pts.astype(np.int64)
    nf = mesh.n_faces
    cnt = np.diff(ptr)
    face_of = np.repeat(np.arange(nf), cnt)
    nxt = np.arange(fp.size) + 1
    nxt[ptr[1:] - 1] = ptr[:-1]
    a, b = fp, fp[nxt]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    sign = np.where(a < b, 1.0, -1.0)
    N = np.int64(mesh.n_points)
    key = lo * N + hi
    uk, inv = np.unique(key, return_inverse=True)
    e0, e1 = uk // N, uk % N
    P = mesh.points
    I = np.empty(uk.size)
    for s in range(0, uk.size, chunk):
        x0 = P[e0[s:s + chunk]]
        dx = P[e1[s:s + chunk]] - x0
        acc = np.zeros(x0.shape[0])
        for t, w in zip(_GL_X, _GL_W):
            acc += w * np.einsum("ij,ij->i", A(x0 + t * dx), dx)
        I[s:s + chunk] = acc
    return np.bincount(face_of, weights=sign * I[inv.reshape(-1)], minlength=nf)


def cell_velocity(mesh: Mesh, u: Callable) -> np.ndarray:
    """Analytic velocity at the mean of each cell's vertices, SoA (3, n_cells)."""
    cen = mesh.points[mesh.cell_verts].mean(1)
    return np.ascontiguousarray(u(cen).T)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    alpha0: np.ndarray
    field: Field
    F_spatial: np.ndarray      # circulation of the spatial potential per face
    U_spatial: np.ndarray      # (3, n_cells)
    dt: float
    n_steps: int
    t_end: float
    exact: Callable | None = None   # t -> exact fractions (if known)

    def step_inputs(self, n: int, dt: float | None = None):
        """(F, U_c, dt) for step n: F averaged over [t_n, t_n+dt] (exact time
        integral of the field's time factor), U_c at the step midpoint."""
        dt = self.dt if dt is None else dt
        t0 = n * self.dt
        f = self.field
        tf = (f.tau_int(t0 + dt) - f.tau_int(t0)) / dt
        return self.F_spatial * tf, self.U_spatial * f.tau(t0 + 0.5 * dt), dt


def make_workload(name: str, n: int | None = None, co: float = 0.5, seed: int | None = None) -> Workload:
    """Named workloads.

    disc2d:       uniform 32x32x1 hex on [0,1]^2 x [0,1/32], disc R=0.15 at (0.5,0.75),
                  exact fractions, translation (1,1,0), Co 0.5, 20 steps; periodic in
                  x and y (the disc crosses y = 1 and comes back at y = 0), front/back
                  walls.
    disc2d_open:  the same with the four sides open (empty inflow, geometric outflow).
    shear3d:      uniform n^3 hex (n=16) periodic in z (the axial flow leaves
                  through z = 1 and comes back at z = 0), walls in x, y; sphere
                  R=0.15 at (0.5,0.75,0.25); the shear field (T=3, umax=1,
                  R=0.5, R22), Co 0.5 on the speed, to t=3.
    shear_periodic: jittered (+-0.2h, seed 1304) n^3 hex (n=12) periodic in x, y, z,
                  a sphere R=0.25 at (0.9,0.15,0.5) wrapped across two seams, the
                  periodic shear field (sin 2 pi y, sin 2 pi z, sin 2 pi x)
                  cos(pi t / 2), Co 0.5 to t=2 (the field reverses).
    translate3d:  periodic uniform n^3 hex (n=16), sphere R=0.15 at the centre,
                  translation along the diagonal (1,1,1) reversed at t = 1/2 and
                  3/2, to t = 2: the sphere reaches the corner (1,1,1), then
                  (0,0,0), then comes back (the paper's periodic translation case,
                  R21); Co 0.5.
    deform3d:     jittered (+-0.2h, seed 1302) n^3 hex (n=128), sphere R=0.15 at
                  (0.35,0.35,0.35), deformation field T=3, Co 0.5 to t=3.
    vortex_tet:   jittered (+-0.15h, seed 1303) Kuhn split of n^3 (n=96), cylinder
                  R=0.15 at (0.5,0.75), single vortex T=8, Co 0.5 to t=8.
    octree:       static octree, base n^3 (n=64) split twice (finest h = 1/(4n))
                  within 3 cell sizes of the sphere R=0.15 at (0.35,0.35,0.35),
                  2:1 face-balanced; deformation field T=3, Co 0.5 on the finest
                  cells, to t=0.5 (the interface leaves the refined band later).
    """
    if name in ("disc2d", "disc2d_open"):
        n = 32 if n is None else n
        if name == "disc2d":
            mesh = hex_mesh((n, n, 1), (1.0, 1.0, 1.0 / n), dim=2, periodic="xy")
        else:
            mesh = hex_mesh((n, n, 1), (1.0, 1.0, 1.0 / n), dim=2, open_sides=("x-", "x+", "y-", "y+"))
        a0 = disc_fraction_2d(mesh, 0.5, 0.75, 0.15)
        fld = translation_field((1.0, 1.0, 0.0))
        steps = 20
    elif name == "translate3d":
        n = 16 if n is None else n
        mesh = hex_mesh((n, n, n), periodic="xyz")
        a0 = sampled_fraction(mesh, sphere_sdf((0.5, 0.5, 0.5), 0.15))
        fld = diagonal_shuttle_field()
        steps = None
    elif name == "shear3d":
        n = 16 if n is None else n
        mesh = hex_mesh((n, n, n), periodic="z")
        a0 = sampled_fraction(mesh, sphere_sdf((0.5, 0.75, 0.25), 0.15))
        fld = shear_field(3.0)
        steps = None
    elif name == "shear_periodic":
        n = 12 if n is None else n
        mesh = hex_mesh((n, n, n), jitter=0.2, seed=1304 if seed is None else seed, periodic="xyz")
        a0 = sampled_fraction(mesh, _wrapped_sphere_sdf((0.9, 0.15, 0.5), 0.25))
        fld = periodic_shear_field(2.0)
        steps = None
    elif name == "deform3d":
        n = 128 if n is None else n
        mesh = hex_mesh((n, n, n), jitter=0.2, seed=1302 if seed is None else seed)
        a0 = sampled_fraction(mesh, sphere_sdf((0.35, 0.35, 0.35), 0.15))
        fld = deformation_field(3.0)
        steps = None
    elif name == "vortex_tet":
        n = 96 if n is None else n
        mesh = kuhn_tet_mesh((n, n, n), jitter=0.15, seed=1303 if seed is None else seed)
        a0 = sampled_fraction(mesh, cylinder_sdf(0.5, 0.75, 0.15))
        fld = single_vortex_field(8.0)
        steps = None
    elif name == "octree":
        n = 64 if n is None else n
        mesh = octree_mesh(n, 2, (0.35, 0.35, 0.35), 0.15)
        a0 = sampled_fraction(mesh, sphere_sdf((0.35, 0.35, 0.35), 0.15))
        fld = deformation_field(3.0)
        steps = None
    else:
        raise ValueError(name)
    Us = cell_velocity(mesh, fld.u)
    umax = float(np.sqrt((Us ** 2).sum(0)).max())
    # Courant number on the cell size h_c = V_c^(1/3) of the nominal lattice cell
    # (2D: the in-plane spacing); a Kuhn tetrahedron has a sixth of the hexahedron
    # (octree: the finest cells)
    hc = mesh.h if mesh.kind in ("hex", "octree") else mesh.h / 6.0 ** (1.0 / 3.0)
    dt = co * hc / umax
    Fs = face_flux_stokes(mesh, fld.A)
    t_end = {"disc2d": steps * dt if steps else None, "disc2d_open": steps * dt if steps else None,
             "translate3d": 2.0, "shear3d": 3.0, "shear_periodic": 2.0, "deform3d": 3.0, "vortex_tet": 8.0, "octree": 0.5}[name]
    if steps is None:
        steps = int(math.ceil(t_end / dt - 1e-12))
    exact = None
    if name in ("disc2d", "disc2d_open"):
        def exact(t, _m=mesh):
            return disc_fraction_2d(_m, 0.5 + t, 0.75 + t, 0.15)
    return Workload(name, mesh, a0, fld, Fs, Us, dt, steps, t_end, exact)


# --------------------------------------------------------------------------
# Batches of independent cases
# --------------------------------------------------------------------------

def concat_meshes(meshes) -> tuple[Mesh, np.ndarray, np.ndarray]:
    """Disjoint union of meshes as one mesh in the same form: points and cells
    of case i follow those of case i-1, the internal faces of every case come
    first (case order), then the boundary faces.  Returns (mesh, cell offsets
    (n+1,), point offsets (n+1,))."""
    cpo = np.zeros(len(meshes) + 1, np.int64)
    ppo = np.zeros(len(meshes) + 1, np.int64)
    for i, m in enumerate(meshes):
        cpo[i + 1] = cpo[i] + m.n_cells
        ppo[i + 1] = ppo[i] + m.n_points
    pts = np.concatenate([m.points for m in meshes])

    def faces(sel):
        ptrs, fps, owns = [], [], []
        for i, m in enumerate(meshes):
            f0, f1 = sel(m)
            a, b = int(m.face_ptr[f0]), int(m.face_ptr[f1])
            ptrs.append(np.diff(m.face_ptr[f0:f1 + 1]).astype(np.int64))
            fps.append(m.face_pts[a:b].astype(np.int64) + ppo[i])
            owns.append(m.owner[f0:f1].astype(np.int64) + cpo[i])
        return np.concatenate(ptrs), np.concatenate(fps), np.concatenate(owns)

    ci, pi_, oi = faces(lambda m: (0, m.n_internal))
    cb, pb, ob = faces(lambda m: (m.n_internal, m.n_faces))
    nei = np.concatenate([m.neighbour.astype(np.int64) + cpo[i] for i, m in enumerate(meshes)])
    counts = np.concatenate([ci, cb])
    face_ptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=face_ptr[1:])
    wall = np.concatenate([m.wall_flags() for m in meshes]).astype(np.uint8)
    kinds = {m.kind for m in meshes}
    cv = None
    if len({m.cell_verts.shape[1] for m in meshes}) == 1:
        cv = np.concatenate([m.cell_verts.astype(np.int64) + ppo[i] for i, m in enumerate(meshes)]).astype(np.int32)
    mesh = Mesh(pts, face_ptr.astype(np.int32), np.concatenate([pi_, pb]).astype(np.int32),
                np.concatenate([oi, ob]).astype(np.int32), nei.astype(np.int32), int(cpo[-1]),
                cv, min(m.h for m in meshes), 3, kinds.pop() if len(kinds) == 1 else "mixed", (), wall)
    return mesh, cpo, ppo


@dataclasses.dataclass
class BatchCase:
    kind: str            # "hex" or "tet"
    n: int               # lattice cells per side
    interface: str       # "sphere" or "plane"
    centre: np.ndarray
    radius: float        # sphere radius (plane: 0)
    normal: np.ndarray   # plane normal (sphere: 0)
    axis: np.ndarray     # rotation axis (unit)
    omega: float         # rotation rate (max |U| over the box = 1)
    co: float
    dt: float


@dataclasses.dataclass
class Batch:
    cases: list
    mesh: Mesh                 # disjoint union of the cases' meshes
    cell_off: np.ndarray       # (n_cases+1,)
    alpha0: np.ndarray
    F_dt: np.ndarray           # F_f dt_case per face (steady fields: every step)
    U_dt: np.ndarray           # (3, n_cells) U_c dt_case
    meshes: list               # the cases' own meshes (for per-case checks)
    F_case: list               # per case: F_f (spatial, unscaled)
    U_case: list               # per case: (3, n_cells_case)
    alpha_case: list
    n_steps: int


def make_batch(n_cases: int = 256, seed: int = 1304, hex_range=(16, 64), tet_range=(16, 48),
               steps: int = 50) -> Batch:
    """Independent cases of uneven size: half uniform hexahedral boxes with
    n^3 cells (n uniform on hex_range), half Kuhn-split n^3 lattices (n on
    tet_range), on [0,1]^3 with open boundaries; each with a sphere (R uniform
    in [0.1, 0.25], centre within 0.5 - R - 2h of the box centre) or a plane
    through the box centre, under a solid-body rotation about an axis through
    the centre (random for a sphere, the plane normal for a plane) scaled so
    that max |U| over the box is 1, at a Courant number uniform in [0.3, 0.8].

    The step uses a field only through F dt and U dt, so F_dt and U_dt carry
    each case's own time step and the batch advances with dt = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cases, meshes, alphas, Fc, Uc = [], [], [], [], []
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
    for ci in range(n_cases):
        kind = "hex" if ci % 2 == 0 else "tet"
        lo, hi = hex_range if kind == "hex" else tet_range
        n = int(rng.integers(lo, hi + 1))
        h = 1.0 / n
        iface = "sphere" if rng.random() < 0.5 else "plane"
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if iface == "sphere":
            R = float(rng.uniform(0.1, 0.25))
            reach = max(0.5 - R - 2.0 * h, 0.0)
            off = rng.uniform(-1.0, 1.0, 3) * reach
            centre = 0.5 + off
            axis = rng.normal(size=3)
            axis /= np.linalg.norm(axis)
            sdf = sphere_sdf(tuple(centre), R)
            normal = np.zeros(3)
        else:
            R = 0.0
            centre = np.full(3, 0.5)
            normal = v
            axis = v

            def sdf(x, _n=normal):
                return (x - 0.5) @ _n
        # max |omega x (x - c)| over the box is at a corner
        r = corners - 0.5
        dist = np.sqrt(np.maximum((r * r).sum(1) - (r @ axis) ** 2, 0.0)).max()
        omega = 1.0 / dist
        fld = rotation_field(omega * axis)
        co = float(rng.uniform(0.3, 0.8))
        hc = h if kind == "hex" else h / 6.0 ** (1.0 / 3.0)
        dt = co * hc / 1.0
        if kind == "hex":
            m = hex_mesh((n, n, n), open_sides=("x-", "x+", "y-", "y+", "z-", "z+"))
        else:
            m = kuhn_tet_mesh((n, n, n))
            m.wall = np.zeros(m.n_faces - m.n_internal, np.uint8)
        a0 = sampled_fraction(m, sdf)
        F = face_flux_stokes(m, fld.A)
        U = cell_velocity(m, fld.u)
        cases.append(BatchCase(kind, n, iface, centre, R, normal, axis, omega, co, dt))
        meshes.append(m)
        alphas.append(a0)
        Fc.append(F)
        Uc.append(U)
    mesh, cpo, _ = concat_meshes(meshes)
    nif = [m.n_internal for m in meshes]
    F_int = np.concatenate([Fc[i][:nif[i]] * cases[i].dt for i in range(n_cases)])
    F_bnd = np.concatenate([Fc[i][nif[i]:] * cases[i].dt for i in range(n_cases)])
    U_dt = np.concatenate([Uc[i] * cases[i].dt for i in range(n_cases)], axis=1)
    return Batch(cases, mesh, cpo, np.concatenate(alphas), np.concatenate([F_int, F_bnd]),
                 np.ascontiguousarray(U_dt), meshes, Fc, Uc, alphas, steps)
