"""Thin ctypes binding of libvof (include/vof.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libvof.so.  Per-step arrays are torch CUDA float64 tensors (flags uint8,
counts int32) on the context's device; the stream defaults to torch's current
stream.  There is no CPU fallback: if libvof.so is missing or cannot load,
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvof.so")

VOF_OK = 0
VOF_ERR_BAD_MESH = -3
FP64, MIXED = 0, 1
INTERFACE, ORIENTED, FULL = 1, 2, 4
STATUS_BITS = {1: "POS_NOT_CONVERGED", 2: "CORR_NOT_CONVERGED", 4: "CLIP_OVERFLOW",
               8: "BOUND_RESIDUAL", 16: "INDEX", 32: "CAPACITY", 64: "TIMEOUT"}
S = dict(mass_before=0, mass_after=1, min_pre=2, max_pre=3, min_post=4, max_post=5,
         n_interface=6, n_band=7, max_pos_it=8, max_corr_it=9, boundary_out=10, n_fallback=11,
         n_bound_sources=12, n_bound_left=13, bound_passes=14, bound_global=15)
S_LEN = 16


class VofError(RuntimeError):
    pass


class _Mesh(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int32), ("n_faces", ctypes.c_int32),
                ("n_internal", ctypes.c_int32), ("n_cells", ctypes.c_int32),
                ("px", ctypes.c_void_p), ("py", ctypes.c_void_p), ("pz", ctypes.c_void_p),
                ("face_ptr", ctypes.c_void_p), ("face_pts", ctypes.c_void_p),
                ("owner", ctypes.c_void_p), ("neighbour", ctypes.c_void_p),
                ("wall", ctypes.c_void_p), ("period", ctypes.c_void_p), ("point_master", ctypes.c_void_p),
                ("point_image", ctypes.c_void_p), ("face_image", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("precision", ctypes.c_int),
                ("bound", ctypes.c_int), ("device", ctypes.c_int)]


EXPORTS = ["vof_create", "vof_destroy", "vof_geometry", "vof_point_velocity", "vof_reconstruct",
           "vof_flux_polyhedra", "vof_correct_flux", "vof_phase_flux", "vof_update", "vof_advect",
           "vof_advect_host", "vof_status", "vof_last_launch_count", "vof_error_string",
           "vof_profile_begin", "vof_profile_end", "vof_work_counts", "vof_count_work", "vof_probe_fma", "vof_probe_barrier",
           "vof_batch_create", "vof_batch_destroy", "vof_batch_context", "vof_batch_advect", "vof_batch_tune",
           "vof_mlp_create", "vof_mlp_destroy", "vof_mlp_params", "vof_mlp_features", "vof_mlp_forward",
           "vof_mlp_gradient", "vof_mlp_train_step", "vof_set_guess", "vof_set_gradient", "vof_lsq_gradient",
           "vof_evsd", "vof_remap", "vof_tune", "vof_create_error", "vof_courant"]
GRAD_NAG, GRAD_LSQ = 0, 1
MLP_IN, MLP_HID, MLP_OUT = 33, 64, 4
MLP_NPARAM = MLP_IN * MLP_HID + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID * MLP_OUT + MLP_OUT
PROF_GROUPS = ["classify", "reconstruct", "correct", "phase_flux", "update"]

_lib = None


def lib():
    """Loads libvof.so (built by paper_1305_3417_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise VofError(f"{LIB_PATH} is not built; run paper_1305_3417_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "vof_create": (I, [ctypes.POINTER(_Mesh), ctypes.POINTER(_Options), ctypes.POINTER(P)]),
        "vof_destroy": (None, [P]),
        "vof_geometry": (I, [P, P, P, P, P, P]),
        "vof_point_velocity": (I, [P, P, P, P]),
        "vof_reconstruct": (I, [P, P, P, P, P, P, P]),
        "vof_flux_polyhedra": (I, [P, P, P, P, D, P, P]),
        "vof_correct_flux": (I, [P, P, P, D, P, P, P]),
        "vof_phase_flux": (I, [P, P, P, P, P, P, P, P, D, P, P]),
        "vof_update": (I, [P, P, P, P, P]),
        "vof_advect": (I, [P, P, P, P, D, P, P]),
        "vof_advect_host": (I, [P, P, P, P, D, P, P]),
        "vof_status": (I, [P, ctypes.POINTER(ctypes.c_uint32), P]),
        "vof_last_launch_count": (I, [P]),
        "vof_error_string": (ctypes.c_char_p, [I]),
        "vof_create_error": (ctypes.c_char_p, []),
        "vof_profile_begin": (I, [P, I]),
        "vof_profile_end": (I, [P, P, ctypes.POINTER(ctypes.c_int)]),
        "vof_work_counts": (I, [P, P, I, P]),
        "vof_count_work": (I, [P, I]),
        "vof_probe_fma": (I, [I, I, ctypes.POINTER(ctypes.c_double), P]),
        "vof_probe_barrier": (I, [P, I, P]),
        "vof_batch_create": (I, [ctypes.POINTER(_Mesh), P, I, ctypes.POINTER(_Options), ctypes.POINTER(P)]),
        "vof_batch_destroy": (None, [P]),
        "vof_batch_context": (P, [P]),
        "vof_batch_advect": (I, [P, P, P, P, P, P, P]),
        "vof_batch_tune": (I, [P, P, P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), P]),
        "vof_mlp_create": (I, [I, P, I, ctypes.POINTER(P)]),
        "vof_mlp_destroy": (None, [P]),
        "vof_mlp_params": (I, [P, P]),
        "vof_mlp_features": (I, [P, P, P, I, P, P]),
        "vof_mlp_forward": (I, [P, P, I, P, P]),
        "vof_mlp_gradient": (I, [P, P, P, I, P, ctypes.POINTER(ctypes.c_float), P]),
        "vof_mlp_train_step": (I, [P, P, P, I, ctypes.c_float, ctypes.POINTER(ctypes.c_float), P]),
        "vof_set_guess": (I, [P, P]),
        "vof_set_gradient": (I, [P, I]),
        "vof_lsq_gradient": (I, [P, P, P, P]),
        "vof_evsd": (I, [P, P, P, P, ctypes.POINTER(ctypes.c_double), I, P, P]),
        "vof_remap": (I, [P, P, P, P, P, P, P, P, P, P]),
        "vof_tune": (I, [P, P, P, P, D, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float), P]),
        "vof_courant": (I, [P, P, D, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(code: int, what: str):
    if code != VOF_OK:
        why = ""
        if code == VOF_ERR_BAD_MESH and what in ("vof_create", "vof_batch_create"):
            why = ": " + lib().vof_create_error().decode()
        raise VofError(f"{what}: {lib().vof_error_string(code).decode()}{why} ({code})")


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, numel, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != dtype:
        raise VofError(f"{name}: expected a CUDA {dtype} tensor")
    if not t.is_contiguous() or t.numel() != numel:
        raise VofError(f"{name}: expected {numel} contiguous elements, got {t.numel()}")
    return t


# ------------------------------------------------------------------ C names

def _mesh_struct(mesh):
    """(_Mesh, arrays kept alive) for a paper_1305_3417_gb300.inputs.Mesh."""
    px, py, pz = (np.ascontiguousarray(v, np.float64) for v in mesh.soa_points())
    fptr = np.ascontiguousarray(mesh.face_ptr, np.int32)
    fpts = np.ascontiguousarray(mesh.face_pts, np.int32)
    own = np.ascontiguousarray(mesh.owner, np.int32)
    nei = np.ascontiguousarray(mesh.neighbour, np.int32)
    wall = np.ascontiguousarray(mesh.wall_flags(), np.uint8)
    keep = [px, py, pz, fptr, fpts, own, nei, wall]
    per = [None] * 4
    if getattr(mesh, "point_master", None) is not None:
        arrs = (np.ascontiguousarray(mesh.period, np.float64).reshape(9),
                np.ascontiguousarray(mesh.point_master, np.int32),
                np.ascontiguousarray(mesh.point_image, np.int8).reshape(-1),
                np.ascontiguousarray(np.append(mesh.face_image, -1), np.int32))  # (never empty)
        keep += list(arrs)
        per = [a.ctypes.data for a in arrs]
    m = _Mesh(mesh.n_points, mesh.n_faces, mesh.n_internal, mesh.n_cells,
              px.ctypes.data, py.ctypes.data, pz.ctypes.data, fptr.ctypes.data, fpts.ctypes.data,
              own.ctypes.data, nei.ctypes.data if nei.size else None, wall.ctypes.data if wall.size else None,
              *per)
    return m, tuple(keep)


def vof_batch_create(mesh, case_cell_ptr, precision: int = MIXED, eps: float = 1e-9, bound: bool = True,
                     device: int = 0):
    """mesh: the joined mesh (inputs.concat_meshes); case_cell_ptr: (ncases+1,) cell offsets."""
    m, keep = _mesh_struct(mesh)
    cp = np.ascontiguousarray(case_cell_ptr, np.int32)
    o = _Options(eps, int(precision), int(bool(bound)), int(device))
    h = ctypes.c_void_p()
    _check(lib().vof_batch_create(ctypes.byref(m), cp.ctypes.data, int(cp.size - 1), ctypes.byref(o),
                                  ctypes.byref(h)), "vof_batch_create")
    return h


def vof_batch_destroy(h):
    if h:
        lib().vof_batch_destroy(h)


def vof_batch_context(h):
    return ctypes.c_void_p(lib().vof_batch_context(h))


def vof_batch_advect(h, alpha, U_dt, F_dt, stats=None, case_mass=None, stream=None):
    _check(lib().vof_batch_advect(h, _ptr(alpha), _ptr(U_dt), _ptr(F_dt), _ptr(stats), _ptr(case_mass),
                                  _stream(stream)), "vof_batch_advect")


def vof_batch_tune(h, alpha, U_dt, F_dt, stream=None):
    """Returns (config = 16*warps + multiplier, step ms)."""
    cfg, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    _check(lib().vof_batch_tune(h, _ptr(alpha), _ptr(U_dt), _ptr(F_dt), ctypes.byref(cfg), ctypes.byref(ms),
                                _stream(stream)), "vof_batch_tune")
    return int(cfg.value), float(ms.value)


def vof_create(mesh, precision: int = FP64, eps: float = 1e-9, bound: bool = True, device: int = 0):
    """mesh: paper_1305_3417_gb300.inputs.Mesh (host arrays).  Returns a handle."""
    m, keep = _mesh_struct(mesh)
    o = _Options(eps, int(precision), int(bool(bound)), int(device))
    h = ctypes.c_void_p()
    _check(lib().vof_create(ctypes.byref(m), ctypes.byref(o), ctypes.byref(h)), "vof_create")
    return h


def vof_destroy(h):
    if h:
        lib().vof_destroy(h)


def vof_geometry(h, cc, vc, cf, sf, stream=None):
    _check(lib().vof_geometry(h, _ptr(cc), _ptr(vc), _ptr(cf), _ptr(sf), _stream(stream)), "vof_geometry")


def vof_point_velocity(h, Uc, Up, stream=None):
    _check(lib().vof_point_velocity(h, _ptr(Uc), _ptr(Up), _stream(stream)), "vof_point_velocity")


def vof_reconstruct(h, alpha, n, d, flags, iters=None, stream=None):
    _check(lib().vof_reconstruct(h, _ptr(alpha), _ptr(n), _ptr(d), _ptr(flags), _ptr(iters), _stream(stream)),
           "vof_reconstruct")


def vof_flux_polyhedra(h, Up, F, lam, dt, V, stream=None):
    _check(lib().vof_flux_polyhedra(h, _ptr(Up), _ptr(F), _ptr(lam), float(dt), _ptr(V), _stream(stream)),
           "vof_flux_polyhedra")


def vof_correct_flux(h, Up, F, dt, lam, iters=None, stream=None):
    _check(lib().vof_correct_flux(h, _ptr(Up), _ptr(F), float(dt), _ptr(lam), _ptr(iters), _stream(stream)),
           "vof_correct_flux")


def vof_phase_flux(h, alpha, n, d, flags, Up, F, lam, dt, Va, stream=None):
    _check(lib().vof_phase_flux(h, _ptr(alpha), _ptr(n), _ptr(d), _ptr(flags), _ptr(Up), _ptr(F), _ptr(lam),
                                float(dt), _ptr(Va), _stream(stream)), "vof_phase_flux")


def vof_update(h, alpha, Va, stats=None, stream=None):
    _check(lib().vof_update(h, _ptr(alpha), _ptr(Va), _ptr(stats), _stream(stream)), "vof_update")


def vof_advect(h, alpha, Uc, F, dt, stats=None, stream=None):
    _check(lib().vof_advect(h, _ptr(alpha), _ptr(Uc), _ptr(F), float(dt), _ptr(stats), _stream(stream)),
           "vof_advect")


def vof_courant(h, F, dt, co, stream=None):
    """co: one-element float64 device tensor, written with the step's Courant number."""
    _check(lib().vof_courant(h, _ptr(F), float(dt), _ptr(co), _stream(stream)), "vof_courant")


def vof_advect_host(h, alpha, Uc, F, dt, stats=None, stream=None):
    """Host (preferably pinned) CPU tensors; copies happen inside the call."""
    _check(lib().vof_advect_host(h, _ptr(alpha), _ptr(Uc), _ptr(F), float(dt), _ptr(stats), _stream(stream)),
           "vof_advect_host")


def vof_status(h, stream=None) -> int:
    bits = ctypes.c_uint32(0)
    _check(lib().vof_status(h, ctypes.byref(bits), _stream(stream)), "vof_status")
    return int(bits.value)


def vof_last_launch_count(h) -> int:
    return int(lib().vof_last_launch_count(h))


def vof_error_string(code: int) -> str:
    return lib().vof_error_string(int(code)).decode()


def vof_profile_begin(h, max_steps: int):
    _check(lib().vof_profile_begin(h, int(max_steps)), "vof_profile_begin")


def vof_profile_end(h):
    """Returns ({group: summed ms}, steps)."""
    ms = (ctypes.c_double * len(PROF_GROUPS))()
    n = ctypes.c_int(0)
    _check(lib().vof_profile_end(h, ms, ctypes.byref(n)), "vof_profile_end")
    return dict(zip(PROF_GROUPS, list(ms))), int(n.value)


WORK = ["prism_planes", "piece_tests", "edges", "tet_volumes", "cut_fractions", "plane_shifts", "faces",
        "fill64", "fill32", "cubic_triangles", "cubic_evals", "reserved"]


def vof_set_gradient(h, kind: int):
    """Gradient of the reconstruction: GRAD_NAG (default) or GRAD_LSQ."""
    _check(lib().vof_set_gradient(h, int(kind)), "vof_set_gradient")


def vof_lsq_gradient(h, alpha, grad, stream=None):
    _check(lib().vof_lsq_gradient(h, _ptr(alpha), _ptr(grad), _stream(stream)), "vof_lsq_gradient")


def vof_evsd(h, flags, n, d, ball, levels, out, stream=None):
    """E_vsd per cell against the ball (cx, cy, cz, R); flags None: the ball's
    volume in each cell."""
    b = (ctypes.c_double * 4)(*[float(x) for x in ball])
    _check(lib().vof_evsd(h, _ptr(flags) if flags is not None else None, _ptr(n) if n is not None else None,
                          _ptr(d) if d is not None else None, b, int(levels), _ptr(out), _stream(stream)),
           "vof_evsd")


def vof_remap(dst, src, alpha_src, n_src, d_src, flags_src, pair_ptr, pair_src, alpha_dst, stream=None):
    """Alg. 2: alpha_dst of context dst from src's planes over the cell pairs."""
    _check(lib().vof_remap(dst, src, _ptr(alpha_src), _ptr(n_src), _ptr(d_src), _ptr(flags_src), _ptr(pair_ptr),
                           _ptr(pair_src), _ptr(alpha_dst), _stream(stream)), "vof_remap")


def vof_tune(h, alpha, Uc, F, dt, stream=None):
    """Autotunes the context's mixed phase-flux launch on one step from alpha
    (left unchanged); returns (config, ms)."""
    cfg, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    _check(lib().vof_tune(h, _ptr(alpha), _ptr(Uc), _ptr(F), float(dt), ctypes.byref(cfg), ctypes.byref(ms),
                          _stream(stream)), "vof_tune")
    return int(cfg.value), float(ms.value)


def vof_count_work(h, on: bool = True):
    """Instrumented step kernels (work counting) on or off."""
    _check(lib().vof_count_work(h, int(bool(on))), "vof_count_work")


def vof_work_counts(h, reset: bool = True, stream=None):
    """Counted primitives since the last reset (include/vof.h), by name."""
    c = (ctypes.c_ulonglong * len(WORK))()
    _check(lib().vof_work_counts(h, c, int(bool(reset)), _stream(stream)), "vof_work_counts")
    return {k: int(c[i]) for i, k in enumerate(WORK)}


def vof_probe_barrier(h, skip_block: int = -1, stream=None):
    """Check of the cooperative kernels' grid barrier: block skip_block leaves at
    once and the others' bounded waits run out (VOF_ST_TIMEOUT)."""
    _check(lib().vof_probe_barrier(h, int(skip_block), _stream(stream)), "vof_probe_barrier")


def vof_probe_fma(device: int = 0, precision: int = FP64, stream=None) -> float:
    out = ctypes.c_double(0.0)
    _check(lib().vof_probe_fma(int(device), int(precision), ctypes.byref(out), _stream(stream)),
           "vof_probe_fma")
    return float(out.value)


# -------------------------------------------------------------- convenience

class VofContext:
    """Owns a libvof context and checks tensor shapes before each call."""

    def __init__(self, mesh, precision: int = FP64, eps: float = 1e-9, bound: bool = True, device: int = 0):
        import torch
        self.nc, self.nf, self.np_, self.ni = mesh.n_cells, mesh.n_faces, mesh.n_points, mesh.n_internal
        self.device = torch.device("cuda", device)
        self.h = vof_create(mesh, precision, eps, bound, device)

    def close(self):
        if getattr(self, "h", None):
            vof_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _z(self, n, dtype=None):
        import torch
        return torch.zeros(n, dtype=dtype or torch.float64, device=self.device)

    def courant(self, F, dt) -> float:
        """The step's Courant number (synchronises to read it back)."""
        co = self._z(1)
        vof_courant(self.h, F, dt, co)
        return float(co.item())

    def geometry(self):
        cc, vc, cf, sf = self._z(3 * self.nc), self._z(self.nc), self._z(3 * self.nf), self._z(3 * self.nf)
        vof_geometry(self.h, cc, vc, cf, sf)
        return cc.view(3, -1), vc, cf.view(3, -1), sf.view(3, -1)

    def point_velocity(self, Uc):
        import torch
        _dev(Uc, torch.float64, 3 * self.nc, "Uc")
        Up = self._z(3 * self.np_)
        vof_point_velocity(self.h, Uc, Up)
        return Up

    def reconstruct(self, alpha):
        import torch
        _dev(alpha, torch.float64, self.nc, "alpha")
        n, d = self._z(3 * self.nc), self._z(self.nc)
        fl = self._z(self.nc, torch.uint8)
        it = self._z(self.nc, torch.int32)
        vof_reconstruct(self.h, alpha, n, d, fl, it)
        return n, d, fl, it

    def flux_polyhedra(self, Up, dt, lam=None, F=None):
        import torch
        _dev(Up, torch.float64, 3 * self.np_, "Up")
        V = self._z(self.nf)
        vof_flux_polyhedra(self.h, Up, F, lam, dt, V)
        return V

    def correct_flux(self, Up, F, dt):
        import torch
        _dev(Up, torch.float64, 3 * self.np_, "Up")
        _dev(F, torch.float64, self.nf, "F")
        lam = self._z(self.nf)
        it = self._z(self.nf, torch.int32)
        vof_correct_flux(self.h, Up, F, dt, lam, it)
        return lam, it

    def phase_flux(self, alpha, n, d, flags, Up, F, lam, dt):
        Va = self._z(self.nf)
        vof_phase_flux(self.h, alpha, n, d, flags, Up, F, lam, dt, Va)
        return Va

    def update(self, alpha, Va):
        stats = self._z(S_LEN)
        vof_update(self.h, alpha, Va, stats)
        return stats

    def advect(self, alpha, Uc, F, dt, stats=None):
        import torch
        _dev(alpha, torch.float64, self.nc, "alpha")
        _dev(Uc, torch.float64, 3 * self.nc, "Uc")
        _dev(F, torch.float64, self.nf, "F")
        if stats is None:
            stats = self._z(S_LEN)
        vof_advect(self.h, alpha, Uc, F, dt, stats)
        return stats

    def status(self) -> int:
        return vof_status(self.h)


class VofBatch:
    """A batch of cases (inputs.Batch) advanced as one mesh, one graph launch per step."""

    def __init__(self, batch, precision: int = MIXED, eps: float = 1e-9, bound: bool = True, device: int = 0):
        import torch
        m = batch.mesh
        self.nc, self.nf, self.ncases = m.n_cells, m.n_faces, len(batch.cases)
        self.device = torch.device("cuda", device)
        self.h = vof_batch_create(m, batch.cell_off, precision, eps, bound, device)

    def close(self):
        if getattr(self, "h", None):
            vof_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def context(self):
        return vof_batch_context(self.h)

    def advect(self, alpha, U_dt, F_dt, stats=None, case_mass=None):
        import torch
        _dev(alpha, torch.float64, self.nc, "alpha")
        _dev(U_dt, torch.float64, 3 * self.nc, "U_dt")
        _dev(F_dt, torch.float64, self.nf, "F_dt")
        if case_mass is not None:
            _dev(case_mass, torch.float64, self.ncases, "case_mass")
        vof_batch_advect(self.h, alpha, U_dt, F_dt, stats, case_mass)

    def tune(self, alpha, U_dt, F_dt):
        return vof_batch_tune(self.h, alpha, U_dt, F_dt)


class Mlp:
    """The initial-guess network (BF16 tensor-core forward/backward, Adam)."""

    def __init__(self, params, max_batch: int = 1 << 16, device: int = 0):
        p = np.ascontiguousarray(params, np.float32)
        if p.size != MLP_NPARAM:
            raise VofError(f"expected {MLP_NPARAM} parameters, got {p.size}")
        self.max_batch, self.device = int(max_batch), device
        self.h = ctypes.c_void_p()
        _check(lib().vof_mlp_create(self.max_batch, p.ctypes.data, int(device), ctypes.byref(self.h)),
               "vof_mlp_create")

    def close(self):
        if getattr(self, "h", None):
            lib().vof_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(MLP_NPARAM, np.float32)
        _check(lib().vof_mlp_params(self.h, out.ctypes.data), "vof_mlp_params")
        return out

    def forward(self, feat):
        import torch
        n = feat.shape[0]
        out = torch.empty((n, MLP_OUT), dtype=torch.float32, device=feat.device)
        _check(lib().vof_mlp_forward(self.h, _ptr(feat), int(n), _ptr(out), _stream(None)), "vof_mlp_forward")
        return out

    def gradient(self, feat, target):
        import torch
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=feat.device)
        loss = ctypes.c_float(0.0)
        _check(lib().vof_mlp_gradient(self.h, _ptr(feat), _ptr(target), int(feat.shape[0]), _ptr(g),
                                      ctypes.byref(loss), _stream(None)), "vof_mlp_gradient")
        return float(loss.value), g

    def train_step(self, feat, target, lr: float) -> float:
        loss = ctypes.c_float(0.0)
        _check(lib().vof_mlp_train_step(self.h, _ptr(feat), _ptr(target), int(feat.shape[0]), float(lr),
                                        ctypes.byref(loss), _stream(None)), "vof_mlp_train_step")
        return float(loss.value)


def vof_mlp_features(h, alpha, cells, n, feat, stream=None):
    _check(lib().vof_mlp_features(h, _ptr(alpha), _ptr(cells), int(n), _ptr(feat), _stream(stream)),
           "vof_mlp_features")


def vof_set_guess(h, mlp):
    _check(lib().vof_set_guess(h, mlp.h if mlp is not None else None), "vof_set_guess")
