"""Builds a library problem from a synthetic workload.

All finite-element arithmetic (node positions, Gauss points, column blocks,
closed pattern, value layout) comes from the C ABI; this module only
evaluates the synthetic orbital and potential definitions at the points the
library reports and copies numbers into the library's layout.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import api
from ._capi import FE_F32, FE_F64


@dataclass
class Problem:
    cfg: object
    mesh: api.Mesh
    dtype: int
    perm: np.ndarray            # new column j holds orbital perm[j]
    cbp: np.ndarray             # column block pointer
    row_ptr: np.ndarray
    col_idx: np.ndarray
    rb_ptr: np.ndarray
    keys: np.ndarray            # (n_dofs,) lattice key I + lx (J + ly K) of each DoF
    P: api.BCSR
    Y: api.BCSR
    P_host: np.ndarray          # values of P in the BCSR layout (dtype of the path)
    vq: np.ndarray              # potential at the Gauss points, FP64, library layout
    supp_nnz: int
    dev: dict = field(default_factory=dict)

    @property
    def n_cols(self):
        return int(self.cbp[-1])


def _axis_coords(mesh: api.Mesh, xyz: np.ndarray, ijk: np.ndarray):
    out = []
    for d, n in enumerate((mesh.info.lx, mesh.info.ly, mesh.info.lz)):
        c = np.zeros(n)
        c[ijk[:, d]] = xyz[:, d]
        out.append(c)
    return out


def build_problem(cfg, dtype: int = FE_F32, pattern: str = "closed") -> Problem:
    """pattern: "closed" (the library's closed pattern, Y = H P exactly) or
    "support" (only the row blocks that hold support nodes of a column block,
    so that Y = mask(P) * (H P) differs from H P)."""
    from synth import inputs
    mesh = api.Mesh(cfg.nx, cfg.ny, cfg.nz, cfg.hx, cfg.hy, cfg.hz, cfg.p, cfg.dirichlet)
    info = mesh.info
    centres = inputs.orbital_centres(cfg)
    perm, cbp = mesh.column_blocks(centres, cfg.n_col_blocks)
    xyz = mesh.node_coords()
    ijk = mesh.dof_keys().astype(np.int64)
    lx, ly, lz = info.lx, info.ly, info.lz
    keys = ijk[:, 0] + lx * (ijk[:, 1] + ly * ijk[:, 2])
    dof_of_key = np.empty(lx * ly * lz, np.int64)
    dof_of_key[keys] = np.arange(len(keys))
    bnd = np.zeros(len(keys), bool)
    if cfg.dirichlet:
        bnd = ((ijk[:, 0] == 0) | (ijk[:, 0] == lx - 1) | (ijk[:, 1] == 0) | (ijk[:, 1] == ly - 1)
               | (ijk[:, 2] == 0) | (ijk[:, 2] == lz - 1))
    ax = _axis_coords(mesh, xyz, ijk)
    M = len(perm)
    col_dofs, col_vals = [], []
    for j in range(M):
        a = int(perm[j])
        lo, hi = inputs.support_candidates(cfg, a, centres)
        rng = [np.nonzero((ax[d] >= lo[d] - 1e-12) & (ax[d] <= hi[d] + 1e-12))[0] for d in range(3)]
        I, J, K = np.meshgrid(*rng, indexing="ij")
        d = dof_of_key[(I + lx * (J + ly * K)).ravel()]
        d = np.sort(d)
        sup = inputs.orbital_support(cfg, xyz[d], a, centres) & ~bnd[d]
        d = d[sup]
        col_dofs.append(d)
        col_vals.append(inputs.orbital_values(cfg, xyz[d], keys[d], a, centres))
    ncb = len(cbp) - 1
    supp = [np.unique(np.concatenate([col_dofs[j] for j in range(cbp[c], cbp[c + 1])]))
            for c in range(ncb)]
    supp_ptr = np.concatenate([[0], np.cumsum([len(s) for s in supp])]).astype(np.int64)
    supp_dofs = np.concatenate(supp).astype(np.int64) if supp_ptr[-1] else np.zeros(1, np.int64)
    if pattern == "closed":
        row_ptr, col_idx = mesh.pattern_closed(ncb, supp_ptr, supp_dofs)
    else:
        rbp = mesh.row_blocks()
        R = mesh.n_row_blocks
        has = np.zeros((R, ncb), bool)
        for c in range(ncb):
            has[np.searchsorted(rbp, supp[c], side="right") - 1, c] = True
        row_ptr = np.concatenate([[0], np.cumsum(has.sum(1))]).astype(np.int64)
        col_idx = np.nonzero(has)[1].astype(np.int32)
    P = api.BCSR(mesh, cbp, row_ptr, col_idx, dtype)
    Y = api.BCSR(mesh, cbp, row_ptr, col_idx, dtype)
    P.set_closed(pattern == "closed")   # the closed pattern is built from exactly these supports
    rb_ptr = mesh.row_blocks()
    offs = P.block_offsets()
    dense = np.full((mesh.n_row_blocks, ncb), -1, np.int64)
    rows_of_k = np.repeat(np.arange(mesh.n_row_blocks), np.diff(row_ptr))
    dense[rows_of_k, col_idx] = np.arange(len(col_idx))
    vals = np.zeros(int(P.info.n_values), api.np_dtype(dtype))
    ld = P.row_strides()
    for c in range(ncb):
        for j in range(cbp[c], cbp[c + 1]):
            d = col_dofs[j]
            r = np.searchsorted(rb_ptr, d, side="right") - 1
            blk = dense[r, c]
            assert np.all(blk >= 0), "support outside the closed pattern"
            vals[offs[blk] + (d - rb_ptr[r]) * ld[c] + (j - cbp[c])] = col_vals[j]
    qp = mesh.quad_points()
    vq = inputs.potential(cfg, qp)
    return Problem(cfg, mesh, dtype, perm, cbp, row_ptr, col_idx, rb_ptr, keys, P, Y, vals, vq,
                   int(sum(len(x) for x in col_dofs)))


def to_device(pb: Problem, device="cuda", stream=None) -> Problem:
    """Allocates and binds the device buffers (torch) and uploads inputs."""
    import torch
    tdt = api.torch_dtype(pb.dtype)
    pb.mesh.upload(device, stream)
    vq = torch.from_numpy(pb.vq.astype(api.np_dtype(pb.dtype))).to(device)
    pb.mesh.set_potential(vq, pb.dtype)
    pv, pt = pb.P.alloc(device, with_tables=True)
    yv, _ = pb.Y.alloc(device, with_tables=False)
    pv.copy_(torch.from_numpy(pb.P_host))
    pb.P.bind(pv, pt, stream)
    pb.Y.bind(yv, None, stream)
    M = pb.n_cols
    pb.dev = {"vq": vq, "P": pv, "Pt": pt, "Y": yv,
              "G_PY": torch.zeros((M, M), dtype=torch.float64, device=device),
              "G_PP": torch.zeros((M, M), dtype=torch.float64, device=device)}
    return pb


def unpack_entries(pb: Problem, values: np.ndarray):
    """All stored entries of a BCSR value array as (dof, column, value)."""
    offs = pb.P.block_offsets()
    ld = pb.P.row_strides()
    rows_of_k = np.repeat(np.arange(pb.mesh.n_row_blocks), np.diff(pb.row_ptr))
    dofs, cols, vals = [], [], []
    for k in range(len(pb.col_idx)):
        r, c = rows_of_k[k], pb.col_idx[k]
        nr = int(pb.rb_ptr[r + 1] - pb.rb_ptr[r])
        w = int(pb.cbp[c + 1] - pb.cbp[c])
        blk = values[offs[k]: offs[k] + nr * ld[c]].reshape(nr, ld[c])[:, :w]
        d = np.repeat(np.arange(pb.rb_ptr[r], pb.rb_ptr[r + 1]), w)
        cc = np.tile(np.arange(pb.cbp[c], pb.cbp[c + 1]), nr)
        dofs.append(d)
        cols.append(cc)
        vals.append(blk.ravel())
    return np.concatenate(dofs), np.concatenate(cols), np.concatenate(vals)
