"""ctypes binding of libgbmd.so: the C ABI of include/gbmd.h under the same names.

Argument marshalling only.  Every step of the computation runs in the library's CUDA kernels;
if the library cannot be loaded, ``lib()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MD_FP64, MD_MIXED, MD_FP32 = 0, 1, 2
MD_REBUILD_VMAX, MD_REBUILD_DISP, MD_REBUILD_EVERY = 0, 1, 2
STATUS = {
    0: "MD_OK", -1: "MD_ERR_INVALID_ARG", -2: "MD_ERR_BOX_TOO_SMALL", -3: "MD_ERR_NBR_OVERFLOW",
    -4: "MD_ERR_CELL_OVERFLOW", -5: "MD_ERR_NONFINITE", -6: "MD_ERR_TIMEOUT", -7: "MD_ERR_CUDA",
    -8: "MD_ERR_WORKSPACE",
}
SERIES_COLS = 9

# every symbol include/gbmd.h declares
EXPORTS = (
    "md_workspace_bytes", "md_workspace_bytes_batch", "md_create", "md_create_batch", "md_bin_cells",
    "md_build_neighbours", "md_compute_forces", "md_integrate", "md_reduce_props", "md_get_series",
    "md_clear_series", "md_get_state", "md_set_state", "md_get_cells", "md_get_neighbours", "md_check",
    "md_nrep", "md_natoms", "md_nbr_capacity", "md_cells_per_axis", "md_set_tuning", "md_get_tuning",
    "md_destroy", "md_last_error", "md_set_timing", "md_get_timing", "md_forces_static",
    "md_adjoint_workspace_bytes", "md_adjoint", "md_props_latest", "md_debug_set_error",
    "md_dyn_workspace_bytes", "md_dyn_begin", "md_dyn_sample", "md_dyn_get", "md_set_chains",
)
NPHASE = 6
PHASES = ("step", "bin", "reorder", "build", "props", "other")


class MDError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class md_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("box", ctypes.c_double * 3), ("eps", ctypes.c_double),
                ("sigma", ctypes.c_double), ("mass", ctypes.c_double), ("rc", ctypes.c_double),
                ("skin", ctypes.c_double), ("dt", ctypes.c_double), ("shift_energy", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("reorder_every", ctypes.c_int32),
                ("nbr_capacity", ctypes.c_int32), ("rebuild_rule", ctypes.c_int32),
                ("props_every", ctypes.c_int32), ("cell_block", ctypes.c_int32)]


class md_props(ctypes.Structure):
    _fields_ = [("U", ctypes.c_double), ("K", ctypes.c_double), ("E_per_atom", ctypes.c_double),
                ("virial", ctypes.c_double), ("pressure", ctypes.c_double), ("P", ctypes.c_double * 3),
                ("vmax", ctypes.c_double), ("mean_nbrs", ctypes.c_double), ("step", ctypes.c_int64),
                ("rebuilds", ctypes.c_int64), ("max_cell_occ", ctypes.c_int32), ("max_nbrs", ctypes.c_int32),
                ("reorders", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["P"] = list(self.P)
        return d


class md_tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("nbr_batch", ctypes.c_int32),
                ("build_batch", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("step_kernel", ctypes.c_int32), ("build_stage", ctypes.c_int32),
                ("reorder_every", ctypes.c_int32)]


class md_chains(ctypes.Structure):
    _fields_ = [("length", ctypes.c_int32), ("pad", ctypes.c_int32), ("fene_k", ctypes.c_double),
                ("fene_r0", ctypes.c_double), ("bend_k", ctypes.c_double), ("dihedral_k", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libgbmd.so (building it in-tree if needed).  Raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libgbmd.so not found at {_build.LIB}; run paper_2003_14061_gb300.build")
        L = ctypes.CDLL(_build.LIB)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        P = ctypes.POINTER(md_params)
        sig = {
            "md_workspace_bytes": (sz, [P]),
            "md_workspace_bytes_batch": (sz, [P, i32, vp, vp]),
            "md_create": (ctypes.c_int, [P, vp, sz, vp, vp, vp, ctypes.POINTER(vp)]),
            "md_create_batch": (ctypes.c_int, [P, i32, vp, vp, vp, sz, vp, vp, vp, ctypes.POINTER(vp)]),
            "md_bin_cells": (ctypes.c_int, [vp]),
            "md_build_neighbours": (ctypes.c_int, [vp]),
            "md_compute_forces": (ctypes.c_int, [vp]),
            "md_integrate": (ctypes.c_int, [vp, i32]),
            "md_reduce_props": (ctypes.c_int, [vp, vp]),
            "md_get_series": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32)]),
            "md_clear_series": (ctypes.c_int, [vp]),
            "md_get_state": (ctypes.c_int, [vp, vp, vp, vp]),
            "md_set_state": (ctypes.c_int, [vp, vp, vp]),
            "md_get_cells": (ctypes.c_int, [vp, vp]),
            "md_get_neighbours": (ctypes.c_int, [vp, vp, vp, i32]),
            "md_check": (ctypes.c_int, [vp]),
            "md_nrep": (i32, [vp]),
            "md_natoms": (i64, [vp]),
            "md_nbr_capacity": (i32, [vp]),
            "md_cells_per_axis": (ctypes.c_int, [vp, i32, vp]),
            "md_set_tuning": (ctypes.c_int, [vp, ctypes.POINTER(md_tuning)]),
            "md_get_tuning": (ctypes.c_int, [vp, ctypes.POINTER(md_tuning)]),
            "md_destroy": (ctypes.c_int, [vp]),
            "md_set_timing": (ctypes.c_int, [vp, i32]),
            "md_get_timing": (ctypes.c_int, [vp, vp, vp, vp]),
            "md_last_error": (ctypes.c_char_p, []),
            "md_forces_static": (ctypes.c_int, [P, i64, vp, vp, vp, vp]),
            "md_adjoint_workspace_bytes": (sz, [vp, i32, i32]),
            "md_adjoint": (ctypes.c_int, [vp, vp, sz, i32, i32, vp, vp, vp, vp]),
            "md_props_latest": (ctypes.c_int, [vp, vp]),
            "md_debug_set_error": (ctypes.c_int, [vp, i32]),
            "md_dyn_workspace_bytes": (sz, [vp, i32, i32]),
            "md_dyn_begin": (ctypes.c_int, [vp, vp, sz, i32, i32]),
            "md_dyn_sample": (ctypes.c_int, [vp]),
            "md_dyn_get": (ctypes.c_int, [vp, vp, vp, vp]),
            "md_set_chains": (ctypes.c_int, [vp, ctypes.POINTER(md_chains)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib


def last_error() -> str:
    return lib().md_last_error().decode()


def check(code: int, what: str) -> None:
    if code != 0:
        raise MDError(code, what, last_error())


def call(name: str, *args) -> int:
    """Call an entry point by name and raise MDError on a non-zero status."""
    fn = getattr(lib(), name)
    rc = fn(*args)
    if fn.restype is ctypes.c_int:
        check(rc, name)
    return rc
