"""ctypes binding of the C ABI in include/fe_mf.h (argument marshalling only).

Every function of the header is exposed under the same name.  Loading fails
loudly when libfe_mf.so has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfe_mf.so")

FE_OK = 0
FE_EINVAL = -1
FE_ENOMEM = -2
FE_EPATTERN = -3
FE_ECUDA = -4
FE_EDEVICE = -5
FE_ESTATE = -6
FE_EUNSUPPORTED = -7
FE_F32 = 1
FE_F64 = 2
FORM_SUMFAC = 0      # FE_FORM_SUMFAC
FORM_CELLMAT = 1     # FE_FORM_CELLMAT

_NAMES = {FE_EINVAL: "FE_EINVAL", FE_ENOMEM: "FE_ENOMEM", FE_EPATTERN: "FE_EPATTERN",
          FE_ECUDA: "FE_ECUDA", FE_EDEVICE: "FE_EDEVICE", FE_ESTATE: "FE_ESTATE",
          FE_EUNSUPPORTED: "FE_EUNSUPPORTED"}


class FeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class fe_mesh_info_t(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("p", C.c_int32),
                ("dirichlet", C.c_int32), ("npx", C.c_int32), ("npy", C.c_int32), ("npz", C.c_int32),
                ("lx", C.c_int32), ("ly", C.c_int32), ("lz", C.c_int32), ("n_row_blocks", C.c_int32),
                ("max_rows_per_block", C.c_int32), ("nq1", C.c_int32), ("n_dofs", C.c_int64),
                ("n_cells", C.c_int64), ("n_q", C.c_int64), ("hx", C.c_double), ("hy", C.c_double),
                ("hz", C.c_double)]


class fe_bcsr_info_t(C.Structure):
    _fields_ = [("n_cols", C.c_int32), ("n_col_blocks", C.c_int32), ("n_row_blocks", C.c_int32),
                ("dtype", C.c_int32), ("max_width", C.c_int32), ("pad_", C.c_int32),
                ("nnz_blocks", C.c_int64), ("n_values", C.c_int64), ("stored_entries", C.c_int64),
                ("value_bytes", C.c_size_t), ("table_bytes", C.c_size_t), ("n_tiles", C.c_int64),
                ("active_cell_cols", C.c_int64), ("n_gram_items_py", C.c_int64),
                ("n_gram_items_pp", C.c_int64), ("gram_flops", C.c_double)]


_P = C.c_void_p
_i32, _i64, _sz, _dbl = C.c_int32, C.c_int64, C.c_size_t, C.c_double
_pi32, _pi64, _pdbl = C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)

# name -> argtypes (every function returns int)
SIGNATURES = {
    "fe_version": [],
    "fe_last_error": [C.c_char_p, _sz],
    "fe_mesh_create": [_i32, _i32, _i32, _dbl, _dbl, _dbl, _i32, _i32, C.POINTER(_P)],
    "fe_mesh_destroy": [_P],
    "fe_mesh_get_info": [_P, C.POINTER(fe_mesh_info_t)],
    "fe_mesh_row_blocks": [_P, _P],
    "fe_mesh_patch_coords": [_P, _P],
    "fe_mesh_dof_keys": [_P, _P],
    "fe_mesh_node_coords": [_P, _P],
    "fe_mesh_quad_points": [_P, _P],
    "fe_mesh_workspace_bytes": [_P, C.POINTER(_sz)],
    "fe_mesh_upload": [_P, _P, _sz, _P],
    "fe_mesh_set_potential": [_P, _P, _i32],
    "fe_mesh_check_device": [_P, _P, _pi32],
    "fe_column_blocks": [_P, _i32, _P, _i32, _P, _P],
    "fe_pattern_closed": [_P, _i32, _P, _P, _P, _P, _i64, _pi64],
    "fe_bcsr_create": [_P, _i32, _i32, _P, _P, _P, _i32, C.POINTER(_P)],
    "fe_bcsr_destroy": [_P],
    "fe_bcsr_get_info": [_P, C.POINTER(fe_bcsr_info_t)],
    "fe_bcsr_block_offsets": [_P, _P],
    "fe_bcsr_row_strides": [_P, _P],
    "fe_bcsr_bind": [_P, _P, _P, _P],
    "fe_apply_H": [_P, _P, _P, _P],
    "fe_apply_M": [_P, _P, _P, _P],
    "fe_gram_PtY": [_P, _P, _P, _P],
    "fe_gram_PtY_sym": [_P, _P, _P, _P],
    "fe_gram_PtP": [_P, _P, _P],
    "fe_apply_H_gram": [_P, _P, _P, _P, _P, _P],
    "fe_apply_H_gram_host": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "fe_mmult": [_P, _P, _dbl, _dbl, _dbl, _P, _P],
    "fe_trace_dot": [_P, _P, _P, _P],
    "fe_bcsr_set_launch": [_P, _i32, _i32, _i32],
    "fe_bcsr_set_sm_limit": [_P, _i32],
    "fe_bcsr_get_launch": [_P, _pi32, _pi32, _pi32],
    "fe_bcsr_set_closed": [_P, _i32],
    "fe_bcsr_get_closed": [_P, _pi32],
    "fe_bcsr_set_form": [_P, _i32],
    "fe_bcsr_get_form": [_P, _pi32],
    "fe_graph_create": [_P, _P, _P, _P, _P, _P, C.POINTER(_P)],
    "fe_graph_launch": [_P, _P],
    "fe_graph_destroy": [_P],
    "fe_autotune": [_P, _P, _P, C.c_char_p, _P, _pdbl],
    "fe_probe_fma": [_i32, _i64, _pdbl, _P],
    "fe_probe_fma_static": [_i32, _i64, _pdbl, _P],
}

_lib = None


def load() -> C.CDLL:
    """Load libfe_mf.so from the package directory (build it first with
    `python -m paper_1907_01005_gb300.build`)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -m paper_1907_01005_gb300.build)")
    lib = C.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    _lib = lib
    return lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    load().fe_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(rc: int) -> int:
    if rc != FE_OK:
        raise FeError(rc, last_error())
    return rc


def _wrap(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"Raw C ABI call {name} (returns the int status)."
    return f


for _name in SIGNATURES:
    globals()[_name] = _wrap(_name)
