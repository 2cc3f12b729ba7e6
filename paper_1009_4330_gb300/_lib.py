"""ctypes declarations of the C ABI in include/md.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import _build

MD_OK, MD_ERR_INVALID, MD_ERR_CUDA, MD_ERR_OOM, MD_ERR_BOX_TOO_SMALL, MD_ERR_LIST_OVERFLOW, \
    MD_ERR_NONFINITE, MD_ERR_TIMEOUT, MD_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["MD_OK", "MD_ERR_INVALID", "MD_ERR_CUDA", "MD_ERR_OOM", "MD_ERR_BOX_TOO_SMALL",
                "MD_ERR_LIST_OVERFLOW", "MD_ERR_NONFINITE", "MD_ERR_TIMEOUT", "MD_ERR_UNSUPPORTED"]
MD_POT_LJ, MD_POT_EAM_FS = 0, 1
MD_PREC_FP64, MD_PREC_MIXED = 0, 1
MD_LIST_AUTO, MD_LIST_FULL, MD_LIST_HALF = 0, 1, 2
MD_MAX_TYPES = 8

# every entry point the header declares (checked by the CPU test suite)
EXPORTS = ("md_create", "md_batch_create", "md_destroy", "md_build_neighbors", "md_compute_forces", "md_step",
           "md_energy_virial", "md_get_state", "md_set_state", "md_set_params", "md_forces_backward",
           "md_autotune", "md_set_kernel", "md_info", "md_get_neighbors", "md_sync_status", "md_last_error",
           "md_time_force", "md_step_eager", "md_neighbors_noalloc", "md_time_gather", "md_set_staging",
           "md_cell_forces", "md_autotune_table", "md_probe_ceilings", "md_probe_fp64_math", "md_halo_pack",
           "md_halo_unpack", "md_vv", "md_create_capacity", "md_reset")
MD_HALO_X, MD_HALO_V, MD_HALO_F, MD_HALO_FP, MD_HALO_EV = 1, 2, 4, 8, 16
MD_VV_DRIFT, MD_VV_DISP, MD_VV_DENSITY, MD_VV_FORCE, MD_VV_KICK = range(5)


class MdConfig(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("n_types", ctypes.c_int32), ("box", ctypes.c_double * 3),
                ("pot", ctypes.c_int), ("params", ctypes.POINTER(ctypes.c_double)), ("n_params", ctypes.c_int32),
                ("cutoff", ctypes.c_double), ("skin", ctypes.c_double), ("dt", ctypes.c_double),
                ("mass", ctypes.POINTER(ctypes.c_double)), ("ftm2v", ctypes.c_double),
                ("energy_shift", ctypes.c_int32), ("prec", ctypes.c_int), ("list", ctypes.c_int),
                ("tpa", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class MdInfo(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("n_rep", ctypes.c_int32), ("tpa", ctypes.c_int32),
                ("list", ctypes.c_int32), ("block", ctypes.c_int32), ("maxneigh", ctypes.c_int32),
                ("vec", ctypes.c_int32), ("max_count", ctypes.c_int32), ("list_entries", ctypes.c_int64), ("rebuilds", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("bins", ctypes.c_int32 * 3), ("tile_atoms", ctypes.c_int32),
                ("tiles_staged", ctypes.c_int32), ("n_tiles_force", ctypes.c_int32)]


class MdTuneRow(ctypes.Structure):
    _fields_ = [("tpa", ctypes.c_int32), ("list", ctypes.c_int32), ("block", ctypes.c_int32), ("vec", ctypes.c_int32),
                ("ms", ctypes.c_double)]


class MdCeilings(ctypes.Structure):
    _fields_ = [("fp32_fma_tflops", ctypes.c_double), ("fp64_fma_tflops", ctypes.c_double),
                ("l2_gather_gps", ctypes.c_double), ("l2_gather_gbs", ctypes.c_double),
                ("index_stream_gbs", ctypes.c_double), ("hbm_copy_gbs", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmd.so (building it first if needed).  Raises if it cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libmd.so not found at {_build.LIB}; run paper_1009_4330_gb300._build.build()")
    lib = ctypes.CDLL(_build.LIB)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "md_create": [P(MdConfig), vp, vp, vp, P(vp)],
        "md_batch_create": [i32, P(MdConfig), P(vp), P(vp), P(vp), P(vp)],
        "md_destroy": [vp],
        "md_build_neighbors": [vp],
        "md_compute_forces": [vp, vp],
        "md_step": [vp, i64],
        "md_energy_virial": [vp, vp],
        "md_get_state": [vp, vp, vp, vp],
        "md_set_state": [vp, vp, vp],
        "md_set_params": [vp, P(d)],
        "md_forces_backward": [vp, vp, vp, vp],
        "md_autotune": [vp, ctypes.c_char_p],
        "md_set_kernel": [vp, i32, ctypes.c_int, i32, i32],
        "md_step_eager": [vp, i64],
        "md_neighbors_noalloc": [i64, vp, P(d), d, vp, vp, i32, vp],
        "md_info": [vp, P(MdInfo)],
        "md_get_neighbors": [vp, vp, vp, i32],
        "md_sync_status": [vp],
        "md_time_force": [vp, i32, i32, P(d), P(d)],
        "md_time_gather": [vp, i32, i32, P(d)],
        "md_set_staging": [vp, i32],
        "md_cell_forces": [vp, vp, i32, P(d)],
        "md_autotune_table": [vp, P(MdTuneRow), i32, P(i32)],
        "md_probe_ceilings": [vp, P(MdCeilings)],
        "md_probe_fp64_math": [i32, i64, vp, vp, vp],
        "md_halo_pack": [vp, vp, i64, i32, P(d), vp],
        "md_halo_unpack": [vp, vp, i64, i32, i32, vp],
        "md_vv": [vp, i32, P(d)],
        "md_create_capacity": [P(MdConfig), i64, vp, vp, vp, P(vp)],
        "md_reset": [vp, i64, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.md_last_error.argtypes = [vp]
    lib.md_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib
