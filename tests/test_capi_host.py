"""C ABI library on the host (no GPU): it loads, exports every declared
symbol, and its integer setup work (Alg. 1 blocking, Alg. 2 column blocks,
closed pattern, tile lists) matches the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle import fe_oracle as O
from synth import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1907_01005_gb300 import _capi
    so = _capi.LIB_PATH
    if not os.path.exists(so):
        from paper_1907_01005_gb300 import build
        build.build()
    return _capi.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "fe_mf.h")).read()
    return sorted(set(re.findall(r"^int\s+(fe_\w+)\s*\(", hdr, re.M)))


def test_library_exports_every_declared_symbol(lib):
    from paper_1907_01005_gb300 import _capi
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/fe_mf.h but not exported"
        assert n in _capi.SIGNATURES, f"{n} has no Python binding"
    assert set(_capi.SIGNATURES) == set(names)
    assert lib.fe_version() >= 100


def test_error_reporting(lib):
    from paper_1907_01005_gb300 import FeError, Mesh
    with pytest.raises(FeError) as e:
        Mesh(3, 4, 4, 1, 1, 1, 2)
    assert "even" in str(e.value)
    with pytest.raises(FeError):
        Mesh(4, 4, 4, 1, 1, 1, 9)


def _problem(name):
    from paper_1907_01005_gb300 import harness
    cfg = inputs.get_config(name)
    return cfg, harness.build_problem(cfg)


@pytest.mark.parametrize("name", ["tiny", "small_p2", "small_p4", "small_p1", "small_p3", "narrow_p4", "free_p2",
                                  "free_p4"])
def test_host_setup_matches_oracle(lib, name):
    cfg, pb = _problem(name)
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    info = pb.mesh.info
    assert info.n_dofs == mesh.n_nodes and info.n_row_blocks == blk.n_patches
    # DoF keys are a bijection onto the lattice, and row blocks match the
    # oracle's ownership rule and Morton order
    assert np.array_equal(np.sort(pb.keys), np.arange(mesh.n_nodes))
    rows = np.diff(pb.rb_ptr)
    np.testing.assert_array_equal(rows, blk.rows_per_block())
    own = blk.owner_rank(pb.keys)
    np.testing.assert_array_equal(own, np.repeat(np.arange(blk.n_patches), rows))
    pc = pb.mesh.patch_coords()
    np.testing.assert_array_equal(blk.patch_to_rank[blk.patch_id(pc[:, 0], pc[:, 1], pc[:, 2])],
                                  np.arange(blk.n_patches))
    # node coordinates and Gauss points
    np.testing.assert_allclose(pb.mesh.node_coords(), mesh.node_coords(pb.keys), rtol=0, atol=1e-13)
    qp = pb.mesh.quad_points().reshape(blk.n_patches, 8, -1, 3)
    for r in range(0, blk.n_patches, max(1, blk.n_patches // 7)):
        px, py, pz = pc[r]
        for c in range(8):
            cell = mesh.cell_index(2 * px + (c & 1), 2 * py + ((c >> 1) & 1), 2 * pz + ((c >> 2) & 1))
            np.testing.assert_allclose(qp[r, c], mesh.cell_qpoints([cell])[0], rtol=0, atol=1e-13)
    # Alg. 2 column blocks
    perm, ptr = O.column_blocks(blk, inputs.orbital_centres(cfg), cfg.n_col_blocks)
    np.testing.assert_array_equal(pb.perm, perm)
    np.testing.assert_array_equal(pb.cbp, ptr)
    # closed pattern
    mv = O.build_orbitals(mesh, cfg)
    pat = O.block_pattern(blk, mv, perm, ptr)
    lib_pat = np.zeros_like(pat)
    rr = np.repeat(np.arange(blk.n_patches), np.diff(pb.row_ptr))
    lib_pat[rr, pb.col_idx] = True
    np.testing.assert_array_equal(lib_pat, pat)
    assert pb.supp_nnz == sum(len(k) for k in mv.keys)


@pytest.mark.parametrize("name", ["small_p2", "small_p4"])
def test_tiles_follow_accessor_semantics(lib, name):
    """Tile (patch, c) exists iff one of the up to eight row blocks the patch
    touches stores c (Alg. 4/5: the union of sorted column lists); the tile
    count and the active cell-columns agree with a brute-force count."""
    cfg, pb = _problem(name)
    pc = pb.mesh.patch_coords()
    rank = {tuple(p): r for r, p in enumerate(pc)}
    cols = [set(pb.col_idx[pb.row_ptr[r]:pb.row_ptr[r + 1]].tolist()) for r in range(len(pc))]
    w = np.diff(pb.cbp)
    n_tiles = 0
    active = 0
    for r, (px, py, pz) in enumerate(pc):
        slots = {}
        for s in range(8):
            q = (px - 1 + (s & 1), py - 1 + ((s >> 1) & 1), pz - 1 + ((s >> 2) & 1))
            slots[s] = rank.get(q)
        union = set().union(*[cols[v] for v in slots.values() if v is not None])
        n_tiles += len(union)
        for c in union:
            for cell in range(8):
                cx, cy, cz = cell & 1, (cell >> 1) & 1, (cell >> 2) & 1
                touched = [s for s in range(8) if not ((not (s & 1) and cx) or (not ((s >> 1) & 1) and cy)
                                                       or (not ((s >> 2) & 1) and cz))]
                if any(slots[s] is not None and c in cols[slots[s]] for s in touched):
                    active += w[c]
    assert pb.P.info.n_tiles == n_tiles
    assert pb.P.info.active_cell_cols == active


def test_gram_flop_count(lib):
    cfg, pb = _problem("small_p2")
    rows = np.diff(pb.rb_ptr)
    w = np.diff(pb.cbp)
    f = 0.0
    for r in range(len(rows)):
        cs = pb.col_idx[pb.row_ptr[r]:pb.row_ptr[r + 1]]
        f += 2.0 * rows[r] * w[cs].sum() ** 2
    assert pb.P.info.gram_flops == pytest.approx(f, rel=1e-12)


def test_pattern_rejections(lib):
    from paper_1907_01005_gb300 import BCSR, FeError, Mesh
    m = Mesh(4, 4, 4, 1, 1, 1, 2)
    R = m.n_row_blocks
    cbp = np.array([0, 8, 16], np.int32)
    ok_ptr = np.arange(R + 1, dtype=np.int64)
    with pytest.raises(FeError, match="ascending"):
        rp = ok_ptr.copy(); rp[1:] = 2 * np.arange(1, R + 1)
        BCSR(m, cbp, rp, np.array([1, 0] * R, np.int32), 1)
    with pytest.raises(FeError, match="out of range"):
        BCSR(m, cbp, ok_ptr, np.full(R, 5, np.int32), 1)
    with pytest.raises(FeError, match="width"):
        BCSR(m, np.array([0, 17], np.int32), ok_ptr, np.zeros(R, np.int32), 1)
    b = BCSR(m, cbp, ok_ptr, np.zeros(R, np.int32), 1)
    assert b.info.nnz_blocks == R
    # empty pattern is valid
    e = BCSR(m, cbp, np.zeros(R + 1, np.int64), np.zeros(1, np.int32), 1)
    assert e.info.n_tiles == 0 and e.info.n_values == 0


def test_launch_knobs_validated(lib):
    from paper_1907_01005_gb300 import BCSR, FeError, Mesh
    m = Mesh(4, 4, 4, 1, 1, 1, 2)
    R = m.n_row_blocks
    b = BCSR(m, np.array([0, 8], np.int32), np.arange(R + 1, dtype=np.int64), np.zeros(R, np.int32), 1)
    assert b.get_launch() == (0, 4, 0)
    b.set_launch(1, 6, 2)
    assert b.get_launch() == (1, 6, 2)
    for bad in [(2, 4, 0), (1, 0, 0), (1, 33, 0), (0, 4, -1), (0, 4, 3), (0, 4, 16)]:
        with pytest.raises(FeError, match="fe_bcsr_set_launch"):
            b.set_launch(*bad)
    assert b.get_launch() == (1, 6, 2)


def test_fp32_gram_union_limit(lib):
    """The FP32 Gram packs at most 64 column blocks per row block; a wider row
    block is refused at creation (FP64 has no such limit)."""
    from paper_1907_01005_gb300 import BCSR, FE_EUNSUPPORTED, FeError, Mesh
    m = Mesh(4, 4, 4, 1, 1, 1, 2)
    R = m.n_row_blocks
    ncb = 65
    cbp = np.arange(ncb + 1, dtype=np.int32)
    row_ptr = np.zeros(R + 1, np.int64)
    row_ptr[1:] = ncb
    col_idx = np.arange(ncb, dtype=np.int32)
    with pytest.raises(FeError, match="at most 64") as e:
        BCSR(m, cbp, row_ptr, col_idx, 1)
    assert e.value.code == FE_EUNSUPPORTED
    assert BCSR(m, cbp, row_ptr, col_idx, 2).info.nnz_blocks == ncb


def test_closed_flag(lib):
    from paper_1907_01005_gb300 import BCSR, FeError, Mesh
    m = Mesh(4, 4, 4, 1, 1, 1, 2)
    R = m.n_row_blocks
    b = BCSR(m, np.array([0, 8], np.int32), np.arange(R + 1, dtype=np.int64), np.zeros(R, np.int32), 1)
    assert b.get_closed() is False
    b.set_closed(True)
    assert b.get_closed() is True
    from paper_1907_01005_gb300 import _capi
    assert _capi.fe_bcsr_set_closed(b.h, 2) == _capi.FE_EINVAL


def test_form_knob(lib):
    """The cell-matrix form is accepted for FP32 at p <= 2 only; the mesh
    workspace grows by its constant operand sets (2 sets x 6 npad x 32 floats)."""
    import ctypes as C
    from paper_1907_01005_gb300 import BCSR, FORM_CELLMAT, FORM_SUMFAC, FeError, Mesh, _capi
    for p, npad in [(1, 16), (2, 32)]:
        m = Mesh(4, 4, 4, 1, 1, 1, p)
        nb = C.c_size_t()
        _capi.check(_capi.fe_mesh_workspace_bytes(m.h, C.byref(nb)))
        assert nb.value == 256 + 2 * 6 * npad * 32 * 4
        R = m.n_row_blocks
        b = BCSR(m, np.array([0, 8], np.int32), np.arange(R + 1, dtype=np.int64), np.zeros(R, np.int32), 1)
        assert b.get_form() == FORM_SUMFAC
        b.set_form(FORM_CELLMAT)
        assert b.get_form() == FORM_CELLMAT
        assert _capi.fe_bcsr_set_form(b.h, 2) == _capi.FE_EINVAL
        assert b.get_form() == FORM_CELLMAT
        b64 = BCSR(m, np.array([0, 8], np.int32), np.arange(R + 1, dtype=np.int64), np.zeros(R, np.int32), 2)
        assert _capi.fe_bcsr_set_form(b64.h, FORM_CELLMAT) == _capi.FE_EUNSUPPORTED
    m4 = Mesh(2, 2, 2, 1, 1, 1, 4)
    nb = C.c_size_t()
    _capi.check(_capi.fe_mesh_workspace_bytes(m4.h, C.byref(nb)))
    assert nb.value == 256
    R = m4.n_row_blocks
    b4 = BCSR(m4, np.array([0, 8], np.int32), np.arange(R + 1, dtype=np.int64), np.zeros(R, np.int32), 1)
    with pytest.raises(FeError, match="p <= 2"):
        b4.set_form(FORM_CELLMAT)
