"""ctypes wrapper of the FP64 CPU oracle (vof_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "vof_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

INTERFACE, ORIENTED, FULL = 1, 2, 4
S = dict(mass_before=0, mass_after=1, min_pre=2, max_pre=3, min_post=4, max_post=5,
         n_interface=6, n_band=7, max_pos_it=8, max_corr_it=9, boundary_out=10, status=11,
         bound_passes=12, bound_global=13)
S_LEN = 14
EPS = 1e-9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fused multiply-add, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "vof_oracle.h"))):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
        sig = {
            "vo_mesh_create": (P, [I, I, I, I, P, P, P, P, P, P, P, P]),
            "vo_mesh_create_periodic": (P, [I, I, I, I, P, P, P, P, P, P, P, P, P, P, P, P]),
            "vo_stencil_codes": (I, [P, I, P, P, I]),
            "vo_courant": (D, [P, P, D]),
            "vo_mesh_destroy": (V, [P]),
            "vo_set_threads": (I, [I]),
            "vo_geometry": (V, [P, P, P, P, P]),
            "vo_stencil": (I, [P, I, P, I]),
            "vo_point_interp": (V, [P, P, P]),
            "vo_nag_gradient": (V, [P, P, I, P, P]),
            "vo_cut_volume": (D, [P, I, P, D]),
            "vo_reconstruct": (I, [P, P, D, I, P, P, P, P, P]),
            "vo_position": (I, [P, I, D, P, P]),
            "vo_reconstruct_grad": (I, [P, P, P, D, I, P, P, P, P, P]),
            "vo_lsq_gradient": (V, [P, P, I, P, P]),
            "vo_evsd": (V, [P, P, P, P, P, I, I, P, P]),
            "vo_remap": (I, [P, P, P, P, P, P, P, P, P]),
            "vo_point_velocity": (V, [P, P, P]),
            "vo_swept_volume": (D, [P, I, P, D, D, D]),
            "vo_correct_flux": (I, [P, P, P, D, I, P, P, P]),
            "vo_phase_flux": (I, [P, P, D, P, P, P, P, P, P, D, I, P, P]),
            "vo_stencil_coverage": (D, [P, I, P, D, D, D]),
            "vo_update": (I, [P, P, P, I, P]),
            "vo_advect": (I, [P, P, P, P, D, D, I, P]),
            "vo_classify_faces": (V, [P, P, D, P]),
            "vo_tet_clip_volume": (D, [P, I, P]),
            "vo_signed_tet_volume": (D, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(n: int) -> int:
    return lib().vo_set_threads(int(n))


def tet_clip_volume(tet, planes) -> float:
    """|tet ^ {x: n_k.x <= d_k}|; tet (4,3), planes (m,4) rows (nx, ny, nz, d)."""
    t = _f64(tet).reshape(12)
    pl = _f64(planes).reshape(-1)
    return lib().vo_tet_clip_volume(_p(t), int(pl.size // 4), _p(pl))


def signed_tet_volume(tet) -> float:
    t = _f64(tet).reshape(12)
    return lib().vo_signed_tet_volume(_p(t))


class OracleMesh:
    """Oracle view of a face-based mesh (see vof_oracle.h for conventions)."""

    def __init__(self, mesh):
        L = lib()
        self.mesh = mesh
        self.nc, self.nf, self.ni, self.np_ = mesh.n_cells, mesh.n_faces, mesh.n_internal, mesh.n_points
        px, py, pz = (np.ascontiguousarray(v) for v in mesh.soa_points())
        self._keep = [px, py, pz, _i32(mesh.face_ptr), _i32(mesh.face_pts), _i32(mesh.owner),
                      _i32(mesh.neighbour), np.ascontiguousarray(mesh.wall_flags(), np.uint8)]
        k = self._keep
        if getattr(mesh, "point_master", None) is not None:
            per = np.ascontiguousarray(mesh.period, np.float64).reshape(9)
            pm = _i32(mesh.point_master)
            pi = np.ascontiguousarray(mesh.point_image, np.int8).reshape(-1)
            fi = _i32(mesh.face_image)
            self._keep += [per, pm, pi, fi]
            self.h = L.vo_mesh_create_periodic(self.np_, self.nf, self.ni, self.nc, _p(k[0]), _p(k[1]), _p(k[2]),
                                               _p(k[3]), _p(k[4]), _p(k[5]), _p(k[6]), _p(k[7]), _p(per),
                                               _p(pm), _p(pi), _p(fi))
        else:
            self.h = L.vo_mesh_create(self.np_, self.nf, self.ni, self.nc, _p(k[0]), _p(k[1]), _p(k[2]),
                                      _p(k[3]), _p(k[4]), _p(k[5]), _p(k[6]), _p(k[7]))
        if not self.h:
            raise RuntimeError("oracle mesh creation failed")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().vo_mesh_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # geometry -------------------------------------------------------------
    def geometry(self):
        cc = np.zeros(3 * self.nc); vc = np.zeros(self.nc)
        cf = np.zeros(3 * self.nf); sf = np.zeros(3 * self.nf)
        lib().vo_geometry(self.h, _p(cc), _p(vc), _p(cf), _p(sf))
        return cc.reshape(3, -1), vc, cf.reshape(3, -1), sf.reshape(3, -1)

    def stencil(self, f):
        out = np.zeros(2048, np.int32)
        n = lib().vo_stencil(self.h, int(f), _p(out), 2048)
        return out[:n].copy()

    def courant(self, F, dt):
        F = _f64(F)
        return lib().vo_courant(self.h, _p(F), float(dt))

    def stencil_codes(self, f):
        """(cells, translation codes) of the face stencil (periodic meshes)."""
        out = np.zeros(2048, np.int32)
        cod = np.zeros(2048, np.int32)
        n = lib().vo_stencil_codes(self.h, int(f), _p(out), _p(cod), 2048)
        return out[:n].copy(), cod[:n].copy()

    # A1 --------------------------------------------------------------------
    def point_interp(self, phi_c):
        phi_c = _f64(phi_c); out = np.zeros(self.np_)
        lib().vo_point_interp(self.h, _p(phi_c), _p(out))
        return out

    def nag_gradient(self, alpha, sel=None):
        alpha = _f64(alpha); g = np.zeros(3 * self.nc)
        s = None if sel is None else _i32(sel)
        lib().vo_nag_gradient(self.h, _p(alpha), 0 if s is None else s.size, _p(s), _p(g))
        return g.reshape(3, -1)

    # A2/A3 -----------------------------------------------------------------
    def cut_volume(self, cell, n, d):
        n = _f64(n)
        return lib().vo_cut_volume(self.h, int(cell), _p(n), float(d))

    def position(self, cell, alpha, n):
        """Alg. 1 for one cell and a given unit normal: (d, iterations)."""
        n = _f64(n); d = np.zeros(1)
        it = lib().vo_position(self.h, int(cell), float(alpha), _p(n), _p(d))
        return float(d[0]), int(it)

    def reconstruct(self, alpha, eps=EPS, sel=None):
        alpha = _f64(alpha)
        n = np.zeros(3 * self.nc); d = np.zeros(self.nc)
        fl = np.zeros(self.nc, np.uint8); it = np.zeros(self.nc, np.int32)
        s = None if sel is None else _i32(sel)
        st = lib().vo_reconstruct(self.h, _p(alpha), eps, 0 if s is None else s.size, _p(s),
                                  _p(n), _p(d), _p(fl), _p(it))
        return n.reshape(3, -1), d, fl, it, st

    def lsq_gradient(self, phi, sel=None):
        """Generalised least-squares gradient (Sec. 2.2.1), (3, nc)."""
        phi = _f64(phi); g = np.zeros(3 * self.nc)
        s = None if sel is None else _i32(sel)
        lib().vo_lsq_gradient(self.h, _p(phi), 0 if s is None else s.size, _p(s), _p(g))
        return g.reshape(3, -1)

    def reconstruct_grad(self, alpha, grad, eps=EPS, sel=None):
        """Reconstruction with the normal of a given gradient (3, nc)."""
        alpha = _f64(alpha); grad = _f64(grad).reshape(-1)
        n = np.zeros(3 * self.nc); d = np.zeros(self.nc)
        fl = np.zeros(self.nc, np.uint8); it = np.zeros(self.nc, np.int32)
        s = None if sel is None else _i32(sel)
        st = lib().vo_reconstruct_grad(self.h, _p(alpha), _p(grad), eps, 0 if s is None else s.size, _p(s),
                                       _p(n), _p(d), _p(fl), _p(it))
        return n.reshape(3, -1), d, fl, it, st

    def evsd(self, flags, n, d, ball, levels, sel=None):
        """E_vsd (Sec. 4.1) per cell against a ball (cx, cy, cz, R); flags None:
        the ball's volume in each cell."""
        fl = None if flags is None else np.ascontiguousarray(flags, np.uint8)
        n = None if n is None else _f64(n).reshape(-1)
        d = None if d is None else _f64(d)
        b = _f64(ball); out = np.zeros(self.nc)
        s = None if sel is None else _i32(sel)
        lib().vo_evsd(self.h, _p(fl), _p(n), _p(d), _p(b), int(levels), 0 if s is None else s.size, _p(s), _p(out))
        return out

    def remap_from(self, src, alpha_src, n_src, d_src, flags_src, pair_ptr, pair_src):
        """Alg. 2: this mesh's volume fractions from the planes of `src` (an
        OracleMesh of the same domain) over the cell pairs (CSR)."""
        a = _f64(alpha_src); n = _f64(n_src).reshape(-1); d = _f64(d_src)
        fl = np.ascontiguousarray(flags_src, np.uint8)
        pp, ps = _i32(pair_ptr), _i32(pair_src)
        out = np.zeros(self.nc)
        lib().vo_remap(self.h, src.h, _p(a), _p(n), _p(d), _p(fl), _p(pp), _p(ps), _p(out))
        return out

    # A4/A5 -----------------------------------------------------------------
    def point_velocity(self, Uc):
        Uc = _f64(Uc).reshape(-1); Up = np.zeros(3 * self.np_)
        lib().vo_point_velocity(self.h, _p(Uc), _p(Up))
        return Up.reshape(3, -1)

    def swept_volume(self, f, Up, dt, lam, F=0.0):
        Up = _f64(Up).reshape(-1)
        return lib().vo_swept_volume(self.h, int(f), _p(Up), float(F), float(dt), float(lam))

    def correct_flux(self, Up, F, dt, sel=None):
        Up = _f64(Up).reshape(-1); F = _f64(F)
        lam = np.zeros(self.nf); it = np.zeros(self.nf, np.int32)
        s = None if sel is None else _i32(sel)
        st = lib().vo_correct_flux(self.h, _p(Up), _p(F), float(dt), 0 if s is None else s.size,
                                   _p(s), _p(lam), _p(it))
        return lam, it, st

    # A6/A7 -----------------------------------------------------------------
    def classify_faces(self, alpha, eps=EPS):
        alpha = _f64(alpha); c = np.zeros(self.nf, np.uint8)
        lib().vo_classify_faces(self.h, _p(alpha), eps, _p(c))
        return c

    def phase_flux(self, alpha, n, d, flags, Up, F, lam, dt, eps=EPS, sel=None):
        alpha = _f64(alpha); n = _f64(n).reshape(-1); d = _f64(d)
        flags = np.ascontiguousarray(flags, np.uint8)
        Up = _f64(Up).reshape(-1); F = _f64(F); lam = _f64(lam)
        Va = np.zeros(self.nf)
        s = None if sel is None else _i32(sel)
        st = lib().vo_phase_flux(self.h, _p(alpha), eps, _p(n), _p(d), _p(flags), _p(Up), _p(F),
                                 _p(lam), float(dt), 0 if s is None else s.size, _p(s), _p(Va))
        return Va, st

    def stencil_coverage(self, f, Up, dt, lam, F=0.0):
        Up = _f64(Up).reshape(-1)
        return lib().vo_stencil_coverage(self.h, int(f), _p(Up), float(F), float(dt), float(lam))

    def update(self, alpha, Va, bound=True):
        a = _f64(alpha).copy(); Va = _f64(Va); st_arr = np.zeros(S_LEN)
        st = lib().vo_update(self.h, _p(a), _p(Va), int(bound), _p(st_arr))
        return a, st_arr, st

    def advect(self, alpha, Uc, F, dt, eps=EPS, bound=True):
        a = _f64(alpha).copy(); Uc = _f64(Uc).reshape(-1); F = _f64(F); st_arr = np.zeros(S_LEN)
        st = lib().vo_advect(self.h, _p(a), _p(Uc), _p(F), float(dt), eps, int(bound), _p(st_arr))
        return a, st_arr, st
