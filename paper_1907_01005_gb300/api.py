"""Object layer over the C ABI: handles with lifetimes, numpy arrays for host
data and torch tensors for device memory.  Argument marshalling only; every
computation runs in libfe_mf.so."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi as capi
from ._capi import FE_F32, FE_F64, FORM_CELLMAT, FORM_SUMFAC, check


def _hptr(a: np.ndarray) -> C.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


def _dptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(s) -> C.c_void_p:
    if s is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(s, "cuda_stream"):
        return C.c_void_p(s.cuda_stream)
    return C.c_void_p(int(s))


def torch_dtype(dtype: int):
    import torch
    return torch.float64 if dtype == FE_F64 else torch.float32


def np_dtype(dtype: int):
    return np.float64 if dtype == FE_F64 else np.float32


class Mesh:
    """fe_mesh handle: box of Q_p cells, Morton patch order, DoF map."""

    def __init__(self, nx, ny, nz, hx, hy, hz, p, dirichlet=1):
        h = C.c_void_p()
        check(capi.fe_mesh_create(nx, ny, nz, hx, hy, hz, p, dirichlet, C.byref(h)))
        self.h = h
        info = capi.fe_mesh_info_t()
        check(capi.fe_mesh_get_info(h, C.byref(info)))
        self.info = info
        self._ws = None
        self._vq = {}

    def __del__(self):
        if getattr(self, "h", None) is not None and capi._lib is not None:
            capi.fe_mesh_destroy(self.h)
            self.h = None

    @property
    def n_dofs(self) -> int:
        return int(self.info.n_dofs)

    @property
    def n_row_blocks(self) -> int:
        return int(self.info.n_row_blocks)

    def row_blocks(self) -> np.ndarray:
        a = np.empty(self.n_row_blocks + 1, np.int64)
        check(capi.fe_mesh_row_blocks(self.h, _hptr(a)))
        return a

    def patch_coords(self) -> np.ndarray:
        a = np.empty((self.n_row_blocks, 3), np.int32)
        check(capi.fe_mesh_patch_coords(self.h, _hptr(a)))
        return a

    def dof_keys(self) -> np.ndarray:
        a = np.empty((self.n_dofs, 3), np.int32)
        check(capi.fe_mesh_dof_keys(self.h, _hptr(a)))
        return a

    def node_coords(self) -> np.ndarray:
        a = np.empty((self.n_dofs, 3), np.float64)
        check(capi.fe_mesh_node_coords(self.h, _hptr(a)))
        return a

    def quad_points(self) -> np.ndarray:
        a = np.empty((int(self.info.n_q), 3), np.float64)
        check(capi.fe_mesh_quad_points(self.h, _hptr(a)))
        return a

    def column_blocks(self, centres: np.ndarray, n_col_blocks: int):
        c = np.ascontiguousarray(centres, np.float64)
        perm = np.empty(len(c), np.int32)
        cbp = np.empty(n_col_blocks + 1, np.int32)
        check(capi.fe_column_blocks(self.h, len(c), _hptr(c), n_col_blocks, _hptr(perm), _hptr(cbp)))
        return perm, cbp

    def pattern_closed(self, n_col_blocks: int, supp_ptr: np.ndarray, supp_dofs: np.ndarray):
        sp_ = np.ascontiguousarray(supp_ptr, np.int64)
        sd = np.ascontiguousarray(supp_dofs, np.int64)
        row_ptr = np.empty(self.n_row_blocks + 1, np.int64)
        nnz = C.c_int64()
        rc = capi.fe_pattern_closed(self.h, n_col_blocks, _hptr(sp_), _hptr(sd), _hptr(row_ptr),
                                    C.c_void_p(0), 0, C.byref(nnz))
        if rc not in (capi.FE_OK, capi.FE_ENOMEM):
            check(rc)
        col_idx = np.empty(max(1, nnz.value), np.int32)
        check(capi.fe_pattern_closed(self.h, n_col_blocks, _hptr(sp_), _hptr(sd), _hptr(row_ptr),
                                     _hptr(col_idx), nnz.value, C.byref(nnz)))
        return row_ptr, col_idx[:nnz.value]

    # device side ---------------------------------------------------------
    def upload(self, device="cuda", stream=None):
        import torch
        nb = C.c_size_t()
        check(capi.fe_mesh_workspace_bytes(self.h, C.byref(nb)))
        self._ws = torch.empty(max(256, nb.value), dtype=torch.uint8, device=device)
        check(capi.fe_mesh_upload(self.h, _dptr(self._ws), nb.value, _stream(stream)))
        return self

    def set_potential(self, vq, dtype: int):
        """Registers V at the Gauss points (torch tensor on the device, kept alive here)."""
        self._vq[dtype] = vq
        check(capi.fe_mesh_set_potential(self.h, _dptr(vq), dtype))

    def check_device(self, stream=None) -> int:
        code = C.c_int32()
        check(capi.fe_mesh_check_device(self.h, _stream(stream), C.byref(code)))
        return code.value


class BCSR:
    """fe_bcsr handle: block pattern, value layout and device work lists."""

    def __init__(self, mesh: Mesh, cbp, row_ptr, col_idx, dtype: int):
        self.mesh = mesh
        self.cbp = np.ascontiguousarray(cbp, np.int32)
        self.row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, np.int32)
        self.dtype = dtype
        h = C.c_void_p()
        check(capi.fe_bcsr_create(mesh.h, int(self.cbp[-1]), len(self.cbp) - 1, _hptr(self.cbp),
                                  _hptr(self.row_ptr), _hptr(self.col_idx), dtype, C.byref(h)))
        self.h = h
        info = capi.fe_bcsr_info_t()
        check(capi.fe_bcsr_get_info(h, C.byref(info)))
        self.info = info
        self.values = None
        self.tables = None

    def __del__(self):
        if getattr(self, "h", None) is not None and capi._lib is not None:
            capi.fe_bcsr_destroy(self.h)
            self.h = None

    @property
    def n_cols(self) -> int:
        return int(self.info.n_cols)

    def block_offsets(self) -> np.ndarray:
        a = np.empty(max(1, int(self.info.nnz_blocks)), np.int64)
        check(capi.fe_bcsr_block_offsets(self.h, _hptr(a)))
        return a[: int(self.info.nnz_blocks)]

    def row_strides(self) -> np.ndarray:
        a = np.empty(len(self.cbp) - 1, np.int32)
        check(capi.fe_bcsr_row_strides(self.h, _hptr(a)))
        return a

    def alloc(self, device="cuda", with_tables=True):
        import torch
        vals = torch.zeros(int(self.info.n_values), dtype=torch_dtype(self.dtype), device=device)
        tabs = (torch.empty(max(256, int(self.info.table_bytes)), dtype=torch.uint8, device=device)
                if with_tables else None)
        return vals, tabs

    def bind(self, values, tables=None, stream=None):
        self.values, self.tables = values, tables
        check(capi.fe_bcsr_bind(self.h, _dptr(values), _dptr(tables), _stream(stream)))
        return self

    def set_launch(self, persistent: int, ctas_per_sm: int = 4, cells_per_round: int = 0):
        check(capi.fe_bcsr_set_launch(self.h, int(persistent), int(ctas_per_sm), int(cells_per_round)))

    def set_sm_limit(self, max_sms: int):
        """Caps the SMs of the persistent launches reading this multivector (0: all)."""
        check(capi.fe_bcsr_set_sm_limit(self.h, int(max_sms)))

    def set_closed(self, closed: bool):
        """Declares the pattern closed for P's values (P^T Y is then symmetric)."""
        check(capi.fe_bcsr_set_closed(self.h, 1 if closed else 0))

    def get_closed(self) -> bool:
        v = C.c_int32()
        check(capi.fe_bcsr_get_closed(self.h, C.byref(v)))
        return bool(v.value)

    def set_form(self, form: int):
        """Form of the cell operator of fe_apply_H / fe_apply_M with this P as
        source: FORM_SUMFAC (sum factorisation) or FORM_CELLMAT (element
        matrices on the tensor cores; FP32, p <= 2)."""
        check(capi.fe_bcsr_set_form(self.h, int(form)))

    def get_form(self) -> int:
        v = C.c_int32()
        check(capi.fe_bcsr_get_form(self.h, C.byref(v)))
        return v.value

    def get_launch(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        check(capi.fe_bcsr_get_launch(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value


def apply_H(mesh: Mesh, P: BCSR, Y: BCSR, stream=None):
    check(capi.fe_apply_H(mesh.h, P.h, Y.h, _stream(stream)))


def apply_M(mesh: Mesh, P: BCSR, Y: BCSR, stream=None):
    """Y = mask(P) * (M P), the mass operator."""
    check(capi.fe_apply_M(mesh.h, P.h, Y.h, _stream(stream)))


def gram_PtY(P: BCSR, Y: BCSR, G, stream=None):
    """G = P^T Y, every block formed."""
    check(capi.fe_gram_PtY(P.h, Y.h, _dptr(G), _stream(stream)))


def gram_PtY_sym(P: BCSR, Y: BCSR, G, stream=None):
    """G = P^T Y when the caller knows it is symmetric (Y = H P or M P of P's
    current values, P declared closed): upper blocks formed and mirrored."""
    check(capi.fe_gram_PtY_sym(P.h, Y.h, _dptr(G), _stream(stream)))


def gram_PtP(P: BCSR, G, stream=None):
    check(capi.fe_gram_PtP(P.h, _dptr(G), _stream(stream)))


def mmult(A: BCSR, X, C: BCSR, alpha=1.0, gamma=0.0, beta=0.0, stream=None):
    """C = alpha (A X + gamma A) + beta C on C's pattern (X: M x M FP64 on the device)."""
    check(capi.fe_mmult(A.h, _dptr(X), float(alpha), float(gamma), float(beta), C.h, _stream(stream)))


def trace_dot(D: BCSR, G: BCSR, out, stream=None):
    """out[0] = tr(D^T G) (out: one FP64 on the device)."""
    check(capi.fe_trace_dot(D.h, G.h, _dptr(out), _stream(stream)))


def om_gradient(PhiH: BCSR, PhiM: BCSR, Hbar, Mbar, G: BCSR, stream=None):
    """G = -2 Phi_M Hbar + 2 Phi_H (2 I - Mbar) on G's pattern (Sec. 2)."""
    mmult(PhiH, Mbar, G, alpha=-2.0, gamma=-2.0, beta=0.0, stream=stream)
    mmult(PhiM, Hbar, G, alpha=-2.0, gamma=0.0, beta=1.0, stream=stream)


def apply_H_gram(mesh: Mesh, P: BCSR, Y: BCSR, G_PY, G_PP, stream=None):
    check(capi.fe_apply_H_gram(mesh.h, P.h, Y.h, _dptr(G_PY), _dptr(G_PP), _stream(stream)))


def apply_H_gram_host(mesh: Mesh, P: BCSR, Y: BCSR, G_PY, G_PP, P_host, Y_host, G_PY_host,
                      G_PP_host, stream=None):
    """Host-buffer variant: torch CPU tensors (pinned for full bandwidth)."""
    check(capi.fe_apply_H_gram_host(mesh.h, P.h, Y.h, _dptr(G_PY), _dptr(G_PP), _dptr(P_host),
                                    _dptr(Y_host), _dptr(G_PY_host), _dptr(G_PP_host), _stream(stream)))


def autotune(mesh: Mesh, P: BCSR, Y: BCSR, cache_path: str | None = None, stream=None) -> float:
    """Times the launch candidates of fe_apply_H and keeps the fastest on P;
    returns its ms per call (-1 on a cache hit)."""
    ms = C.c_double()
    path = cache_path.encode() if cache_path else None
    check(capi.fe_autotune(mesh.h, P.h, Y.h, path, _stream(stream), C.byref(ms)))
    return ms.value


class StepGraph:
    """CUDA graph of one apply_H_gram step over fixed buffers (fe_graph_*)."""

    def __init__(self, mesh: Mesh, P: BCSR, Y: BCSR, G_PY, G_PP, stream=None):
        self._keep = (mesh, P, Y, G_PY, G_PP)
        h = C.c_void_p()
        check(capi.fe_graph_create(mesh.h, P.h, Y.h, _dptr(G_PY), _dptr(G_PP), _stream(stream), C.byref(h)))
        self.h = h

    def launch(self, stream=None):
        check(capi.fe_graph_launch(self.h, _stream(stream)))

    def __del__(self):
        if getattr(self, "h", None) is not None and capi._lib is not None:
            capi.fe_graph_destroy(self.h)
            self.h = None
