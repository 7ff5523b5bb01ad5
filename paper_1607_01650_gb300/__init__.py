"""GB300 (sm_103a) hot path of sparse-view dual-energy CT: ADM-TV reconstruction
and PLS two-material decomposition (Li et al., arXiv:1607.01650, Sec. 2).

This module is a thin ctypes binding of ``libdect.so`` (C ABI declared in
``include/dect.h``).  It only marshals arguments: PyTorch supplies device
memory and streams, and every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library or a CUDA device is
missing, calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
from typing import List, Optional, Sequence, Tuple

from . import _build

__all__ = ["Geometry", "Plan", "ConePlan", "project_cone", "backproject_cone", "pls_decompose_cone",
           "pls_edge_mask_cone", "AdmParams", "PlsParams", "AdmReport", "AdmProfile", "DectError",
           "load", "project", "backproject", "project_otf", "backproject_otf", "adm_tv", "adm_tv_batch",
           "pls_decompose", "pls_edge_mask", "kernel_launches",
           "library_path"]


class DectError(RuntimeError):
    pass


class _Geometry(C.Structure):
    _fields_ = [("n", C.c_int), ("pixel_mm", C.c_double), ("n_views", C.c_int),
                ("n_bins", C.c_int), ("pitch_mm", C.c_double), ("sod_mm", C.c_double),
                ("sdd_mm", C.c_double), ("start_rad", C.c_double), ("arc_rad", C.c_double),
                ("det_offset_mm", C.c_double)]


class _PlanInfo(C.Structure):
    _fields_ = [("n_pixels", C.c_int64), ("n_rays", C.c_int64), ("nnz", C.c_int64),
                ("table_bytes", C.c_int64), ("n_grid_aligned", C.c_int64)]


class _ConeGeometry(C.Structure):
    _fields_ = [("n", C.c_int), ("nz", C.c_int), ("pixel_mm", C.c_double), ("slice_mm", C.c_double),
                ("n_views", C.c_int), ("n_rows", C.c_int), ("n_cols", C.c_int),
                ("pitch_u_mm", C.c_double), ("pitch_v_mm", C.c_double), ("sod_mm", C.c_double),
                ("sdd_mm", C.c_double), ("start_rad", C.c_double), ("arc_rad", C.c_double),
                ("offset_u_mm", C.c_double), ("offset_v_mm", C.c_double)]


class _AdmParams(C.Structure):
    _fields_ = [("mu", C.c_double), ("rho", C.c_double), ("xi", C.c_double),
                ("beta", C.c_double * 2), ("step_rule", C.c_int), ("max_iter", C.c_int),
                ("rel_obj_tol", C.c_double), ("check_every", C.c_int), ("warm_start", C.c_int),
                ("nonneg", C.c_int), ("joint_tv", C.c_int)]


class _AdmReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("objective", C.c_double),
                ("rel_change", C.c_double), ("primal_res", C.c_double), ("resid_drift", C.c_double)]


class _AdmProfile(C.Structure):
    _fields_ = [("fwd_ms_total", C.c_double), ("bwd_ms_total", C.c_double),
                ("fwd_launches", C.c_int64), ("bwd_launches", C.c_int64),
                ("table_bytes_fwd", C.c_int64), ("table_bytes_bwd", C.c_int64)]


class _AdmGroup(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("m", C.c_void_p), ("x", C.c_void_p), ("n_slices", C.c_int),
                ("reports", C.c_void_p)]


class _PlsParams(C.Structure):
    _fields_ = [("eta", (C.c_double * 2) * 2), ("gamma", C.c_double), ("edge_tau", C.c_double),
                ("edge_eps", C.c_double), ("max_iter", C.c_int), ("tol", C.c_double)]


class _PlsReport(C.Structure):
    _fields_ = [("iters", C.c_int * 2), ("relres", C.c_double * 2)]


_lib = None

# name: (restype, argtypes) -- every entry point of include/dect.h
_P = C.c_void_p
_SIGS = {
    "dect_plan_create": (C.c_int, [C.POINTER(_Geometry), C.c_int, _P, C.POINTER(_P)]),
    "dect_plan_destroy": (C.c_int, [_P]),
    "dect_plan_create_cone": (C.c_int, [C.POINTER(_ConeGeometry), C.c_int, _P, C.POINTER(_P)]),
    "dect_pls_decompose_cone": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(_PlsParams), _P, _P, _P]),
    "dect_pls_edge_mask_cone": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, _P, _P]),
    "dect_plan_get_info": (C.c_int, [_P, C.POINTER(_PlanInfo)]),
    "dect_plan_copy_table": (C.c_int, [_P, _P, _P, _P, _P]),
    "dect_project": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dect_backproject": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dect_fbp": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dect_adm_tv": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(_AdmParams), _P, _P]),
    "dect_adm_tv_ex": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(_AdmParams), _P, _P, _P]),
    "dect_pls_decompose": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(_PlsParams), _P, _P, _P]),
    "dect_adm_tv_groups": (C.c_int, [C.POINTER(_AdmGroup), C.c_int, C.POINTER(_AdmParams), C.c_int, _P]),
    "dect_pls_decompose_noalloc": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(_PlsParams), _P, _P, _P]),
    "dect_pls_edge_mask": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, _P, _P]),
    "dect_adm_tv_batch": (C.c_int, [C.POINTER(_AdmGroup), C.c_int, C.POINTER(_AdmParams), _P]),
    "dect_adm_tv_batch_ex": (C.c_int, [C.POINTER(_AdmGroup), C.c_int, C.POINTER(_AdmParams), C.c_int, _P]),
    "dect_project_otf": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dect_backproject_otf": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "dect_kernel_launches": (C.c_int64, []),
    "dect_cnn_num_params": (C.c_int64, []),
    "dect_cnn_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(_P)]),
    "dect_cnn_destroy": (C.c_int, [_P]),
    "dect_cnn_set_params": (C.c_int, [_P, _P]),
    "dect_cnn_get_params": (C.c_int, [_P, _P]),
    "dect_cnn_forward": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_float, _P]),
    "dect_cnn_loss_grad": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, C.c_float,
                                     C.POINTER(C.c_float), _P, _P]),
    "dect_cnn_adam_step": (C.c_int, [_P, C.c_float, C.c_float, C.c_float, C.c_float, _P]),
    "dect_cnn_set_conv_path": (C.c_int, [_P, C.c_int]),
    "dect_cnn_get_conv_path": (C.c_int, [_P]),
    "dect_cnn_check": (C.c_int, [_P]),
    "dect_cnn_set_conv_tuning": (C.c_int, [_P, C.c_int]),
    "dect_selftest_bounded_wait": (C.c_int, [C.c_uint, _P]),
    "dect_selftest_index": (C.c_int, [C.c_int, _P]),
    "dect_check_status": (C.c_int, []),
    "dect_checked_build": (C.c_int, []),
    "dect_plan_get_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "dect_plan_set_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "dect_plan_get_fwd_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "dect_plan_set_fwd_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "dect_plan_get_tv_tuning": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "dect_plan_set_tv_tuning": (C.c_int, [_P, C.c_int, C.c_int]),
    "dect_status_string": (C.c_char_p, [C.c_int]),
    "dect_last_error": (C.c_char_p, []),
    "dect_version": (C.c_int, []),
}


def library_path() -> str:
    """libdect.so, or libdect_checked.so (the index-checked build) when the
    environment variable DECT_CHECKED is 1 at import time."""
    return _build.LIB_CHECKED if os.environ.get("DECT_CHECKED") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Load libdect.so (compiling it first when it is missing or stale)."""
    global _lib
    if _lib is None:
        path = library_path()
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise DectError("%s is not built (run __graft_entry__.build())" % os.path.basename(path))
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, what: str):
    if status != 0:
        lib = load()
        raise DectError("%s: %s (%s)" % (what, lib.dect_status_string(status).decode(),
                                         lib.dect_last_error().decode()))


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None, device=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise DectError("tensor must live in CUDA device memory")
    if dtype is not None and t.dtype != dtype:
        raise DectError("expected dtype %s, got %s" % (dtype, t.dtype))
    if not t.is_contiguous():
        raise DectError("tensor must be contiguous")
    if device is not None and t.device.index != device:
        raise DectError("tensor on cuda:%d, plan on cuda:%d" % (t.device.index, device))
    return C.c_void_p(t.data_ptr())


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Fan-beam slice geometry (Sec. 2.1, Fig. 1).  Units mm / rad."""
    n: int
    px: float
    nv: int
    nb: int
    pitch: float
    sod: float
    sdd: float
    start: float = 0.0
    arc: float = 2.0 * math.pi
    det_offset: float = 0.0

    @classmethod
    def of(cls, g) -> "Geometry":
        return cls(g.n, g.px, g.nv, g.nb, g.pitch, g.sod, g.sdd, g.start, g.arc, g.det_offset)

    def _c(self) -> _Geometry:
        return _Geometry(self.n, self.px, self.nv, self.nb, self.pitch, self.sod, self.sdd,
                         self.start, self.arc, self.det_offset)


class Plan:
    """Siddon system matrix of one geometry on one device (dect_plan_*)."""

    def __init__(self, geom, device: int = 0, stream=None):
        import torch
        self.geom = Geometry.of(geom)
        self.device = device
        lib = load()
        h = C.c_void_p()
        with torch.cuda.device(device):
            _check(lib.dect_plan_create(C.byref(self.geom._c()), device, _stream(stream),
                                        C.byref(h)), "dect_plan_create")
        self._h = h
        info = _PlanInfo()
        _check(lib.dect_plan_get_info(h, C.byref(info)), "dect_plan_get_info")
        self.nnz = int(info.nnz)
        self.n_pixels = int(info.n_pixels)
        self.n_rays = int(info.n_rays)
        self.table_bytes = int(info.table_bytes)
        self.n_grid_aligned = int(info.n_grid_aligned)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().dect_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tuning(self, images: int):
        """(chosen A^T variant, [median us of each variant]) for a batch width; see dect.h."""
        ch = C.c_int(-1)
        us = (C.c_float * BWD_VARIANTS)()
        _check(load().dect_plan_get_tuning(self._h, images, C.byref(ch), us), "dect_plan_get_tuning")
        return ch.value, list(us)

    def set_tuning(self, images: int, choice: int):
        """Force the A^T variant for a batch width (-1: re-time on the next ADM call)."""
        _check(load().dect_plan_set_tuning(self._h, images, choice), "dect_plan_set_tuning")

    def fwd_tuning(self, images: int):
        """(chosen A variant, [median us of each variant]) for a batch width; see dect.h."""
        ch = C.c_int(-1)
        us = (C.c_float * FWD_VARIANTS)()
        _check(load().dect_plan_get_fwd_tuning(self._h, images, C.byref(ch), us), "dect_plan_get_fwd_tuning")
        return ch.value, list(us)

    def set_fwd_tuning(self, images: int, choice: int):
        """Force the A variant for a batch width (-1: re-time on the next ADM call)."""
        _check(load().dect_plan_set_fwd_tuning(self._h, images, choice), "dect_plan_set_fwd_tuning")

    def tv_tuning(self, images: int):
        """(chosen TV-step variant, [median us of each variant]) for a batch width; see dect.h."""
        ch = C.c_int(-1)
        us = (C.c_float * TV_VARIANTS)()
        _check(load().dect_plan_get_tv_tuning(self._h, images, C.byref(ch), us), "dect_plan_get_tv_tuning")
        return ch.value, list(us)

    def set_tv_tuning(self, images: int, choice: int):
        """Force the TV-step variant for a batch width (-1: re-time on the next ADM call)."""
        _check(load().dect_plan_set_tv_tuning(self._h, images, choice), "dect_plan_set_tv_tuning")

    def table(self):
        """(rowptr int64 [M+1], pix int32 [nnz], len float32 [nnz]) as numpy arrays."""
        import numpy as np
        M = self.geom.nv * self.geom.nb
        rowptr = np.zeros(M + 1, np.int64)
        pix = np.zeros(max(self.nnz, 1), np.int32)
        ln = np.zeros(max(self.nnz, 1), np.float32)
        _check(load().dect_plan_copy_table(self._h, rowptr.ctypes.data, pix.ctypes.data,
                                           ln.ctypes.data, _stream()), "dect_plan_copy_table")
        return rowptr, pix[:self.nnz], ln[:self.nnz]


class ConePlan(Plan):
    """Cone-beam plan (dect_plan_create_cone): 3-D Siddon table of a
    circular orbit with a flat 2-D detector.  geom: an object with n, nz,
    px, pz, nv, nr, nc, pu, pv, sod, sdd, start, arc, off_u, off_v (mm, rad)."""

    def __init__(self, geom, device: int = 0, stream=None):  # noqa: super-init replaced
        import torch
        self.geom = geom
        self.device = device
        lib = load()
        h = C.c_void_p()
        cg = _ConeGeometry(geom.n, geom.nz, geom.px, geom.pz, geom.nv, geom.nr, geom.nc, geom.pu, geom.pv,
                           geom.sod, geom.sdd, geom.start, geom.arc, geom.off_u, geom.off_v)
        with torch.cuda.device(device):
            _check(lib.dect_plan_create_cone(C.byref(cg), device, _stream(stream), C.byref(h)),
                   "dect_plan_create_cone")
        self._h = h
        info = _PlanInfo()
        _check(lib.dect_plan_get_info(h, C.byref(info)), "dect_plan_get_info")
        self.nnz = int(info.nnz)
        self.n_pixels = int(info.n_pixels)
        self.n_rays = int(info.n_rays)
        self.table_bytes = int(info.table_bytes)
        self.n_grid_aligned = int(info.n_grid_aligned)

    def table(self):
        """(rowptr int64 [M+1], voxel int32 [nnz], len float32 [nnz]) as numpy arrays."""
        import numpy as np
        rowptr = np.zeros(self.n_rays + 1, np.int64)
        pix = np.zeros(max(self.nnz, 1), np.int32)
        ln = np.zeros(max(self.nnz, 1), np.float32)
        _check(load().dect_plan_copy_table(self._h, rowptr.ctypes.data_as(C.c_void_p),
                                           pix.ctypes.data_as(C.c_void_p), ln.ctypes.data_as(C.c_void_p),
                                           _stream()), "dect_plan_copy_table")
        return rowptr, pix[:self.nnz], ln[:self.nnz]


def project_cone(plan: ConePlan, x, y=None, stream=None):
    """y = A x for volumes x [..., nz, n, n] -> y [..., nv, nr, nc] (cone-beam plan)."""
    import torch
    g = plan.geom
    if x.shape[-3:] != (g.nz, g.n, g.n):
        raise DectError("x must end in (nz, n, n)")
    batch = x.numel() // (g.nz * g.n * g.n)
    if y is None:
        y = torch.empty(x.shape[:-3] + (g.nv, g.nr, g.nc), device=x.device, dtype=torch.float32)
    _check(load().dect_project(plan.handle, _ptr(x, torch.float32, plan.device), _ptr(y, torch.float32, plan.device),
                               batch, _stream(stream)), "dect_project")
    return y


def backproject_cone(plan: ConePlan, y, x=None, stream=None):
    """x = A^T y for projections y [..., nv, nr, nc] -> x [..., nz, n, n] (cone-beam plan)."""
    import torch
    g = plan.geom
    if y.shape[-3:] != (g.nv, g.nr, g.nc):
        raise DectError("y must end in (nv, nr, nc)")
    batch = y.numel() // (g.nv * g.nr * g.nc)
    if x is None:
        x = torch.empty(y.shape[:-3] + (g.nz, g.n, g.n), device=y.device, dtype=torch.float32)
    _check(load().dect_backproject(plan.handle, _ptr(y, torch.float32, plan.device),
                                   _ptr(x, torch.float32, plan.device), batch, _stream(stream)), "dect_backproject")
    return x


def project(plan: Plan, x, y=None, stream=None):
    """y = A x for x [..., n, n] float32 CUDA -> y [..., nv, nb] (Eq. (1))."""
    import torch
    g = plan.geom
    batch = x.numel() // (g.n * g.n)
    if x.shape[-2:] != (g.n, g.n):
        raise DectError("x must end in (n, n)")
    if y is None:
        y = torch.empty(x.shape[:-2] + (g.nv, g.nb), device=x.device, dtype=torch.float32)
    _check(load().dect_project(plan.handle, _ptr(x, torch.float32, plan.device),
                               _ptr(y, torch.float32, plan.device), batch, _stream(stream)),
           "dect_project")
    return y


def project_otf(plan: Plan, x, y=None, stream=None):
    """y = A x with the on-the-fly projector (no table read; see dect_project_otf)."""
    import torch
    g = plan.geom
    if x.shape[-2:] != (g.n, g.n):
        raise DectError("x must end in (n, n)")
    batch = x.numel() // (g.n * g.n)
    if y is None:
        y = torch.empty(x.shape[:-2] + (g.nv, g.nb), device=x.device, dtype=torch.float32)
    _check(load().dect_project_otf(plan.handle, _ptr(x, torch.float32, plan.device),
                                   _ptr(y, torch.float32, plan.device), batch, _stream(stream)), "dect_project_otf")
    return y


def backproject_otf(plan: Plan, y, x=None, stream=None):
    """x = A^T y with the on-the-fly projector (see dect_backproject_otf)."""
    import torch
    g = plan.geom
    if y.shape[-2:] != (g.nv, g.nb):
        raise DectError("y must end in (nv, nb)")
    batch = y.numel() // (g.nv * g.nb)
    if x is None:
        x = torch.empty(y.shape[:-2] + (g.n, g.n), device=y.device, dtype=torch.float32)
    _check(load().dect_backproject_otf(plan.handle, _ptr(y, torch.float32, plan.device),
                                       _ptr(x, torch.float32, plan.device), batch, _stream(stream)),
           "dect_backproject_otf")
    return x


def backproject(plan: Plan, y, x=None, stream=None):
    """x = A^T y for y [..., nv, nb] float32 CUDA -> x [..., n, n] (transpose in G_f, Eq. (9))."""
    import torch
    g = plan.geom
    if y.shape[-2:] != (g.nv, g.nb):
        raise DectError("y must end in (nv, nb)")
    batch = y.numel() // (g.nv * g.nb)
    if x is None:
        x = torch.empty(y.shape[:-2] + (g.n, g.n), device=y.device, dtype=torch.float32)
    _check(load().dect_backproject(plan.handle, _ptr(y, torch.float32, plan.device),
                                   _ptr(x, torch.float32, plan.device), batch, _stream(stream)),
           "dect_backproject")
    return x


def fbp(plan: Plan, m, x=None, stream=None):
    """Fan-beam FBP of m [..., nv, nb] float32 CUDA -> x [..., n, n] (1/mm); see dect_fbp.

    The analytic reconstruction of Sec. 2.4 / Sec. 3, used as an initial image
    for adm_tv (warm_start=True).  Needs a plan over a full 360-degree arc."""
    import torch
    g = plan.geom
    if m.shape[-2:] != (g.nv, g.nb):
        raise DectError("m must end in (nv, nb)")
    batch = m.numel() // (g.nv * g.nb)
    if x is None:
        x = torch.empty(m.shape[:-2] + (g.n, g.n), device=m.device, dtype=torch.float32)
    _check(load().dect_fbp(plan.handle, _ptr(m, torch.float32, plan.device),
                           _ptr(x, torch.float32, plan.device), batch, _stream(stream)), "dect_fbp")
    return x


BB1, CAUCHY = 0, 1
BWD_VARIANTS = 8                        # DECT_BWD_VARIANTS in include/dect.h
FWD_VARIANTS = 3                        # DECT_FWD_VARIANTS in include/dect.h
TV_VARIANTS = 2                         # DECT_TV_VARIANTS in include/dect.h


@dataclasses.dataclass
class AdmParams:
    """Parameters of Eq. (3)-(10); see dect_adm_params in include/dect.h."""
    mu: float = 4.0
    rho: float = 256.0
    xi: float = 0.0                     # <= 0: xi = rho
    beta: Tuple[float, float] = (1.0, 0.6)
    step_rule: int = CAUCHY
    max_iter: int = 100
    rel_obj_tol: float = 0.0
    check_every: int = 10
    warm_start: bool = False
    nonneg: bool = False                # project f onto f >= 0 after each f-step
    joint: bool = False                 # one TV over both energies of a slice

    def _c(self) -> _AdmParams:
        b = (C.c_double * 2)(*self.beta)
        return _AdmParams(self.mu, self.rho, self.xi, b, self.step_rule, self.max_iter,
                          self.rel_obj_tol, self.check_every, 1 if self.warm_start else 0,
                          1 if self.nonneg else 0, 1 if self.joint else 0)


@dataclasses.dataclass
class AdmReport:
    iters: int
    converged: bool
    objective: float
    rel_change: float
    primal_res: float = 0.0    # |A f - g| recomputed from the result
    resid_drift: float = 0.0   # |r_carried - (A f - g)|


def _report(r) -> AdmReport:
    return AdmReport(r.iters, bool(r.converged), r.objective, r.rel_change, r.primal_res, r.resid_drift)


@dataclasses.dataclass
class AdmProfile:
    """CUDA-event timing of the two table kernels inside one adm_tv call."""
    fwd_ms_total: float
    bwd_ms_total: float
    fwd_launches: int
    bwd_launches: int
    table_bytes_fwd: int
    table_bytes_bwd: int


def adm_tv(plan: Plan, m, params: AdmParams, x=None, stream=None, profile: bool = False):
    """ADM-TV reconstruction (Eq. (3)-(10)) of slices sharing `plan`.

    m: [S, 2, nv, nb] float32 CUDA (energy 0 = high, 1 = low).  Returns
    (x [S, 2, n, n], reports[S * 2]) and, with profile=True, an AdmProfile.
    """
    import torch
    g = plan.geom
    if m.dim() != 4 or m.shape[1:] != (2, g.nv, g.nb):
        raise DectError("m must be [S, 2, nv, nb]")
    S = m.shape[0]
    if x is None:
        x = torch.zeros((S, 2, g.n, g.n), device=m.device, dtype=torch.float32)
    elif x.shape != (S, 2, g.n, g.n):
        raise DectError("x must be [S, 2, n, n]")
    rep = (_AdmReport * max(2 * S, 1))()
    prof = _AdmProfile() if profile else None
    _check(load().dect_adm_tv_ex(plan.handle, _ptr(m, torch.float32, plan.device),
                                 _ptr(x, torch.float32, plan.device), S, C.byref(params._c()),
                                 C.cast(rep, C.c_void_p),
                                 C.cast(C.pointer(prof), C.c_void_p) if prof is not None else None,
                                 _stream(stream)), "dect_adm_tv")
    reps = [_report(r) for r in rep[:2 * S]]
    if profile:
        return x, reps, AdmProfile(prof.fwd_ms_total, prof.bwd_ms_total, prof.fwd_launches,
                                   prof.bwd_launches, prof.table_bytes_fwd, prof.table_bytes_bwd)
    return x, reps


def adm_tv_groups(groups, params: AdmParams, workers: int = 0, stream=None):
    """ADM-TV of slices of uneven geometry (Eq. (3)-(10)) in one call.

    groups: list of (plan, m [S, 2, nv, nb], x [S, 2, n, n] or None); plans must
    differ.  Groups run concurrently on their own streams.  Returns
    [(x, reports)] in the order given.
    """
    import torch
    cg = (_AdmGroup * max(len(groups), 1))()
    keep = []
    out = []
    for i, (plan, m, x) in enumerate(groups):
        g = plan.geom
        if m.dim() != 4 or m.shape[1:] != (2, g.nv, g.nb):
            raise DectError("group %d: m must be [S, 2, nv, nb]" % i)
        S = m.shape[0]
        if x is None:
            x = torch.zeros((S, 2, g.n, g.n), device=m.device, dtype=torch.float32)
        rep = (_AdmReport * max(2 * S, 1))()
        keep.append(rep)
        cg[i] = _AdmGroup(plan.handle.value, _ptr(m, torch.float32, plan.device).value,
                          _ptr(x, torch.float32, plan.device).value, S, C.cast(rep, C.c_void_p).value)
        out.append((x, rep, S))
    _check(load().dect_adm_tv_groups(cg, len(groups), C.byref(params._c()), workers, _stream(stream)),
           "dect_adm_tv_groups")
    return [(x, [_report(r) for r in rep[:2 * S]]) for x, rep, S in out]


PROJ_TABLE, PROJ_OTF = 0, 1              # DECT_PROJ_* in include/dect.h


def adm_tv_batch(groups, params: AdmParams, stream=None, projector: str = "otf"):
    """ADM-TV (Eq. (3)-(10)) of slices of uneven geometry, all advanced together
    with one launch per ADM phase (dect_adm_tv_batch_ex), the projector
    computed on the fly ("otf") or streamed from the plans' stored tables
    ("table").  groups: list of (plan, m [S, 2, nv, nb], x [S, 2, n, n] or
    None); plans may repeat.  Returns [(x, reports)] in the order given."""
    proj = {"table": PROJ_TABLE, "otf": PROJ_OTF}.get(projector)
    if proj is None:
        raise DectError("projector must be 'table' or 'otf'")
    import torch
    cg = (_AdmGroup * max(len(groups), 1))()
    keep, out = [], []
    for i, (plan, m, x) in enumerate(groups):
        g = plan.geom
        if m.dim() != 4 or m.shape[1:] != (2, g.nv, g.nb):
            raise DectError("group %d: m must be [S, 2, nv, nb]" % i)
        S = m.shape[0]
        if x is None:
            x = torch.zeros((S, 2, g.n, g.n), device=m.device, dtype=torch.float32)
        elif x.shape != (S, 2, g.n, g.n):
            raise DectError("group %d: x must be [S, 2, n, n]" % i)
        rep = (_AdmReport * max(2 * S, 1))()
        keep.append(rep)
        cg[i] = _AdmGroup(plan.handle.value, _ptr(m, torch.float32, plan.device).value,
                          _ptr(x, torch.float32, plan.device).value, S, C.cast(rep, C.c_void_p).value)
        out.append((x, rep, S))
    _check(load().dect_adm_tv_batch_ex(cg, len(groups), C.byref(params._c()), proj, _stream(stream)),
           "dect_adm_tv_batch_ex")
    return [(x, [_report(r) for r in rep[:2 * S]]) for x, rep, S in out]


def check_status():
    """Raise DectError if an index check of the checked build has failed
    since the last call (dect_check_status); no-op in the plain build."""
    _check(load().dect_check_status(), "dect_check_status")


def kernel_launches() -> int:
    """Kernels launched by libdect so far in this process."""
    return int(load().dect_kernel_launches())


@dataclasses.dataclass
class PlsParams:
    """Parameters of Eq. (11)-(15); see dect_pls_params in include/dect.h."""
    eta: Sequence[Sequence[float]] = ((0.0184, 0.0227), (0.0342, 0.0573))
    gamma: float = 0.1
    edge_tau: float = 0.2
    edge_eps: float = 0.05
    max_iter: int = 500
    tol: float = 1e-6

    def _c(self) -> _PlsParams:
        e = ((C.c_double * 2) * 2)()
        for i in range(2):
            for j in range(2):
                e[i][j] = self.eta[i][j]
        return _PlsParams(e, self.gamma, self.edge_tau, self.edge_eps, self.max_iter, self.tol)


def pls_decompose(x, params: PlsParams, u=None, stream=None):
    """PLS decomposition (Eq. (11)-(15)): x [B, 2, n, n] (x_h, x_l) -> u [B, 2, n, n] (u_1, u_2).

    Returns (u, reports) with reports[b] = ((iters_1, iters_2), (relres_1, relres_2)).
    """
    import torch
    if x.dim() != 4 or x.shape[1] != 2 or x.shape[2] != x.shape[3]:
        raise DectError("x must be [B, 2, n, n]")
    n = x.shape[-1]
    batch = x.shape[0]
    if u is None:
        u = torch.empty_like(x)
    dev = x.device.index
    rep = (_PlsReport * max(batch, 1))()
    _check(load().dect_pls_decompose(_ptr(x, torch.float32, dev), n, batch, C.byref(params._c()),
                                     _ptr(u, torch.float32, dev), C.cast(rep, C.c_void_p),
                                     _stream(stream)), "dect_pls_decompose")
    reps = [(tuple(r.iters), tuple(r.relres)) for r in rep[:batch]]
    return u, reps


def pls_edge_mask(x, tau: float, mask=None, stream=None):
    """Edge map of Eq. (14) as the decomposition decides it: x [B, 2, n, n] -> uint8 [B, n, n]."""
    import torch
    if x.dim() != 4 or x.shape[1] != 2 or x.shape[2] != x.shape[3]:
        raise DectError("x must be [B, 2, n, n]")
    n = x.shape[-1]
    batch = x.shape[0]
    dev = x.device.index
    if mask is None:
        mask = torch.empty((batch, n, n), dtype=torch.uint8, device=x.device)
    _check(load().dect_pls_edge_mask(_ptr(x, torch.float32, dev), n, batch, float(tau),
                                     _ptr(mask, torch.uint8, dev), _stream(stream)), "dect_pls_edge_mask")
    return mask


def pls_decompose_cone(x, params: PlsParams, u=None, stream=None):
    """3-D PLS decomposition (6 neighbours): x [B, 2, nz, n, n] -> u [B, 2, nz, n, n]."""
    import torch
    if x.dim() != 5 or x.shape[1] != 2 or x.shape[3] != x.shape[4]:
        raise DectError("x must be [B, 2, nz, n, n]")
    batch, nz, n = x.shape[0], x.shape[2], x.shape[-1]
    if u is None:
        u = torch.empty_like(x)
    dev = x.device.index
    rep = (_PlsReport * max(batch, 1))()
    _check(load().dect_pls_decompose_cone(_ptr(x, torch.float32, dev), n, nz, batch, C.byref(params._c()),
                                          _ptr(u, torch.float32, dev), C.cast(rep, C.c_void_p), _stream(stream)),
           "dect_pls_decompose_cone")
    return u, [(tuple(r.iters), tuple(r.relres)) for r in rep[:batch]]


def pls_edge_mask_cone(x, tau: float, mask=None, stream=None):
    """Edge map of the 3-D decomposition: x [B, 2, nz, n, n] -> uint8 [B, nz, n, n]."""
    import torch
    if x.dim() != 5 or x.shape[1] != 2:
        raise DectError("x must be [B, 2, nz, n, n]")
    batch, nz, n = x.shape[0], x.shape[2], x.shape[-1]
    if mask is None:
        mask = torch.empty((batch, nz, n, n), dtype=torch.uint8, device=x.device)
    _check(load().dect_pls_edge_mask_cone(_ptr(x, torch.float32, x.device.index), n, nz, batch, float(tau),
                                          _ptr(mask, torch.uint8, x.device.index), _stream(stream)),
           "dect_pls_edge_mask_cone")
    return mask


# Limits of the allocation-free decomposition (include/dect.h).
PLS_NOALLOC_MAX_PIXELS = 262144
PLS_NOALLOC_MAX_BATCH = 64


def pls_decompose_noalloc(x, params: PlsParams, u, stream=None):
    """Same as pls_decompose, for callers that cannot allocate device memory.

    The library takes the decomposition's scratch from a fixed array it holds
    on every device (no cudaMalloc, no stream, event or graph creation); `u`
    must be passed in.  Work is limited to batch * n * n <= PLS_NOALLOC_MAX_PIXELS
    and batch <= PLS_NOALLOC_MAX_BATCH.  Calls share that array, so calls that
    could overlap on the GPU must be ordered on one stream.
    """
    import torch
    if x.dim() != 4 or x.shape[1] != 2 or x.shape[2] != x.shape[3]:
        raise DectError("x must be [B, 2, n, n]")
    if u is None or u.shape != x.shape:
        raise DectError("u must be given, with the shape of x")
    n = x.shape[-1]
    batch = x.shape[0]
    dev = x.device.index
    rep = (_PlsReport * max(batch, 1))()
    _check(load().dect_pls_decompose_noalloc(_ptr(x, torch.float32, dev), n, batch,
                                             C.byref(params._c()), _ptr(u, torch.float32, dev),
                                             C.cast(rep, C.c_void_p), _stream(stream)),
           "dect_pls_decompose_noalloc")
    return u, [(tuple(r.iters), tuple(r.relres)) for r in rep[:batch]]


class Cnn:
    """CNN warm start (see dect_cnn_* in include/dect.h): x -> x + s * net(x / s)."""

    def __init__(self, device: int = 0, max_pixels: int = 1 << 20):
        import torch
        self.device = device
        h = C.c_void_p()
        with torch.cuda.device(device):
            _check(load().dect_cnn_create(device, max_pixels, C.byref(h)), "dect_cnn_create")
        self._h = h
        self.max_pixels = int(max_pixels)
        self.num_params = int(load().dect_cnn_num_params())

    def close(self):
        if getattr(self, "_h", None):
            load().dect_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.num_params:
            raise DectError("expected %d parameters" % self.num_params)
        _check(load().dect_cnn_set_params(self._h, p.ctypes.data), "dect_cnn_set_params")

    def get_params(self):
        import numpy as np
        p = np.zeros(self.num_params, np.float32)
        _check(load().dect_cnn_get_params(self._h, p.ctypes.data), "dect_cnn_get_params")
        return p

    # kernels of the 3x3 convolutions (dect_cnn_set_conv_path)
    CONV_TCGEN05 = 0
    CONV_MMA_SYNC = 1

    @property
    def conv_path(self) -> int:
        return int(load().dect_cnn_get_conv_path(self._h))

    @conv_path.setter
    def conv_path(self, path: int):
        _check(load().dect_cnn_set_conv_path(self._h, int(path)), "dect_cnn_set_conv_path")

    def set_conv_tuning(self, blocks_per_sm: int):
        """Resident blocks per SM of the tensor-memory convolution (1 or 2)."""
        _check(load().dect_cnn_set_conv_tuning(self._h, int(blocks_per_sm)), "dect_cnn_set_conv_tuning")

    def check(self):
        """Synchronise and raise if a bounded device wait ran out (dect_cnn_check)."""
        _check(load().dect_cnn_check(self._h), "dect_cnn_check")

    def forward(self, x, scale: float, out=None, stream=None, check: bool = True):
        """x: [B, H, W] float32 CUDA (H, W multiples of 4).  With check (the
        default) the call synchronises and raises if a device wait ran out."""
        import torch
        B, H, W = x.shape
        if out is None:
            out = torch.empty_like(x)
        _check(load().dect_cnn_forward(self._h, _ptr(x, torch.float32, self.device),
                                       _ptr(out, torch.float32, self.device), B, H, W, scale,
                                       _stream(stream)), "dect_cnn_forward")
        if check:
            self.check()
        return out

    def loss_grad(self, x, target, scale: float, want_grad: bool = False, stream=None):
        import numpy as np
        import torch
        B, H, W = x.shape
        loss = C.c_float(0.0)
        g = np.zeros(self.num_params, np.float32) if want_grad else None
        _check(load().dect_cnn_loss_grad(self._h, _ptr(x, torch.float32, self.device),
                                         _ptr(target, torch.float32, self.device), B, H, W, scale,
                                         C.byref(loss), g.ctypes.data if want_grad else None,
                                         _stream(stream)), "dect_cnn_loss_grad")
        return (float(loss.value), g) if want_grad else float(loss.value)

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  stream=None):
        _check(load().dect_cnn_adam_step(self._h, lr, beta1, beta2, eps, _stream(stream)),
               "dect_cnn_adam_step")
