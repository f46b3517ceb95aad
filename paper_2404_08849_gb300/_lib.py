"""ctypes declarations of the C ABI in include/grist.h (argument marshalling
only; every step of the hot path runs in libgrist_gb300.so)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

_P = ctypes.POINTER
_D = ctypes.c_double
_I = ctypes.c_int32
_V = ctypes.c_void_p

GRIST_FP64, GRIST_MIX, GRIST_MIX_DBL_MASS, GRIST_MIX_DF = 0, 1, 2, 3
GRIST_SUM_DRY_MASS, GRIST_SUM_TRACER_MASS, GRIST_SUM_AREA_WEIGHTED = 0, 1, 2
GRIST_FLAG_NONFINITE, GRIST_FLAG_TIMEOUT = 0x1, 0x2
# precision-map rows (grist_dycore_params.emulate_fp32_rows), in the header's order
GRIST_ROWS = {"mass_flux": 0x001, "wind": 0x002, "pv_flux": 0x004, "ke_grad": 0x008, "vadv_u": 0x010,
              "pgf": 0x020, "theta": 0x040, "dpi_pv": 0x080, "eos": 0x100, "nh_adv": 0x200}
GRIST_ROW_ALL = 0x3ff

STATUS = {0: "GRIST_OK", -1: "GRIST_EINVAL", -2: "GRIST_ECUDA", -3: "GRIST_ENOMEM",
          -4: "GRIST_ENUMERIC", -5: "GRIST_ETIMEOUT", -6: "GRIST_EUNSUPPORTED"}


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_cells", _I), ("n_edges", _I), ("n_vertices", _I), ("max_edges", _I), ("radius", _D),
                ("cell_xyz", _P(_D)), ("cell_area", _P(_D)), ("vertex_xyz", _P(_D)), ("vertex_area", _P(_D)),
                ("edge_dc", _P(_D)), ("edge_dv", _P(_D)), ("f_vertex", _P(_D)),
                ("cells_on_edge", _P(_I)), ("vertices_on_edge", _P(_I)), ("n_edges_on_cell", _P(_I)),
                ("edges_on_cell", _P(_I)), ("cells_on_cell", _P(_I)), ("edges_on_vertex", _P(_I)),
                ("cells_on_vertex", _P(_I)), ("edge_sign_on_cell", _P(_D)), ("edge_sign_on_vertex", _P(_D)),
                ("kite_area", _P(_D)), ("n_edges_on_edge", _P(_I)), ("edges_on_edge", _P(_I)),
                ("trisk_weight", _P(_D)), ("d2_stencil", _P(_I)), ("d2_coef", _P(_D)), ("sfc_reorder", _I)]


class TracerMember(ctypes.Structure):
    _fields_ = [("n_levels", _I), ("n_tracers", _I), ("ld", _I), ("q", _V), ("dpi", _V), ("mass_flux", _V),
                ("vmass_flux", _V), ("ld_int", _I)]


class TracerBatch(ctypes.Structure):
    _fields_ = [("n_members", _I), ("members", _P(TracerMember)), ("prec", ctypes.c_int), ("limiter", _I),
                ("beta_upwind", _D), ("vertical_courant_max", _D)]


class TracerTuning(ctypes.Structure):
    _fields_ = [("block", _I), ("tracers_per_thread", _I), ("persistent", _I), ("use_graph", _I), ("fused", _I),
                ("levels_per_thread", _I), ("cell_edges", _I)]


class DycoreParams(ctypes.Structure):
    _fields_ = [("n_levels", _I), ("ld", _I), ("ld_int", _I), ("pi_top", _D), ("p0", _D), ("rd", _D),
                ("cp", _D), ("g", _D), ("offcentre_beta", _D), ("b_interface", _P(_D)), ("phi_surface", _V),
                ("emulate_fp32_rows", ctypes.c_uint32)]


class DycoreState(ctypes.Structure):
    _fields_ = [("u", _V), ("ps", _V), ("dpi_theta", _V), ("w", _V), ("phi", _V), ("mass_flux_accum", _V),
                ("accum_weight", _V), ("dpi_start", _V), ("p_nh", _V), ("p_nh_valid", _I), ("accum_scale", _D),
                ("vmass_flux_accum", _V)]


EXPORTS = {
    "grist_mesh_create": ([_P(MeshDesc), ctypes.c_int, _P(_V)], ctypes.c_int),
    "grist_mesh_destroy": ([_V], ctypes.c_int),
    "grist_mesh_permutation": ([_V, _P(_I), _P(_I), _P(_I)], ctypes.c_int),
    "grist_mesh_counts": ([_V, _P(_I), _P(_I), _P(_I)], ctypes.c_int),
    "grist_mesh_features": ([_V, _P(ctypes.c_uint32)], ctypes.c_int),
    "grist_tracer_step": ([_V, _P(TracerBatch), _D, _V], ctypes.c_int),
    "grist_dycore_step_hydro": ([_V, _P(DycoreState), _P(DycoreParams), ctypes.c_int, _D, _V], ctypes.c_int),
    "grist_dycore_step_nh": ([_V, _P(DycoreState), _P(DycoreParams), ctypes.c_int, _D, _V], ctypes.c_int),
    "grist_global_sums": ([_V, ctypes.c_int, _V, _V, _I, _I, ctypes.c_int, _D, _P(_D), _V], ctypes.c_int),
    "grist_last_step_status": ([_V, _P(ctypes.c_uint32)], ctypes.c_int),
    "grist_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "grist_profile_enable": ([_V, ctypes.c_int], ctypes.c_int),
    "grist_profile_read": ([_V, _I, ctypes.c_char_p, _P(_I), _P(_D), _P(_I)], ctypes.c_int),
    "grist_tracer_set_tuning": ([_V, _P(TracerTuning)], ctypes.c_int),
    "grist_tracer_get_tuning": ([_V, _P(TracerTuning)], ctypes.c_int),
    "grist_tracer_autotune": ([_V, _P(TracerBatch), _D, _I, _V, _P(TracerTuning), _P(_D)], ctypes.c_int),
    "grist_selftest_bounded_wait": ([_V, ctypes.c_int64, _V], ctypes.c_int),
    "grist_weighted_sum_noalloc": ([_V, _V, ctypes.c_int64, _V, _V], ctypes.c_int),
    "grist_bench_fp64_fma": ([ctypes.c_int64, _I, _I, _V, _V], ctypes.c_int),
    "grist_capture_begin": ([_V], ctypes.c_int),
    "grist_capture_end": ([_V, _P(_V)], ctypes.c_int),
    "grist_graph_launch": ([_V, _V], ctypes.c_int),
    "grist_graph_destroy": ([_V], ctypes.c_int),
    "grist_selftest_conversions": ([ctypes.c_uint64, ctypes.c_uint64, _P(ctypes.c_uint64), _P(ctypes.c_uint64)],
                                   ctypes.c_int),
    "grist_selftest_split": ([ctypes.c_uint64, ctypes.c_uint64, _P(ctypes.c_uint64), _P(ctypes.c_uint64)],
                             ctypes.c_int),
    "grist_diag_vorticity": ([_V, _V, ctypes.c_int, _I, _I, _V, _V], ctypes.c_int),
    "grist_selftest_reciprocal": ([ctypes.c_uint64, ctypes.c_uint64, _P(ctypes.c_uint64), _P(ctypes.c_uint64),
                                   _P(ctypes.c_uint64)], ctypes.c_int),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgrist_gb300.so (building it in-tree when missing or stale).
    Raises if the library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libgrist_gb300.so is missing; run paper_2404_08849_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, (args, res) in EXPORTS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class GristError(RuntimeError):
    def __init__(self, func, code):
        super().__init__("%s failed: %s (%d)" % (func, STATUS.get(code, "?"), code))
        self.code = code


def check(func, code):
    if code != 0:
        raise GristError(func, code)
    return code
