"""Cell-matrix form of the apply (element matrices as dense products per cell,
Sec. 3.2 Eq. fe_matrices_cell_based; FP32, p <= 2, TF32 tensor cores with a
3-term split) through the C ABI against the FP64 oracle, on the tolerances
of the sum-factorised FP32 path: Y 1e-5, P^T Y 1e-6, P^T P 1e-10."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL = dict(Y=1e-5, PY=1e-6, PP=1e-10)
SMALL = ["tiny", "small_p1", "small_p2", "wide_p2", "narrow_p2", "free_p2"]


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _problem(name, pattern="closed"):
    from paper_1907_01005_gb300 import FORM_CELLMAT, harness
    cfg = inputs.get_config(name)
    pb = harness.build_problem(cfg, 1, pattern=pattern)
    harness.to_device(pb)
    pb.P.set_form(FORM_CELLMAT)
    assert pb.P.get_form() == FORM_CELLMAT
    return cfg, pb


@pytest.mark.parametrize("name", SMALL)
def test_cellmat_parity_small(name):
    import torch
    from paper_1907_01005_gb300 import apply_H_gram, harness
    cfg, pb = _problem(name)
    d = pb.dev
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    r = O.run(cfg, fp32_inputs=True)
    dofs, cols, vals = harness.unpack_entries(pb, d["Y"].cpu().numpy())
    keys = pb.keys[dofs]
    ref = np.asarray(r.Y.tocsr()[keys, pb.perm[cols]]).ravel()
    assert _relerr(vals, ref) <= TOL["Y"], _relerr(vals, ref)
    assert np.all(vals[r.mesh.boundary(keys)] == 0)          # Dirichlet rows stay zero
    G_PY, G_PP = d["G_PY"].cpu().numpy(), d["G_PP"].cpu().numpy()
    ref_py = r.G_PY[np.ix_(pb.perm, pb.perm)]
    ref_pp = r.G_PP[np.ix_(pb.perm, pb.perm)]
    assert _relerr(G_PY, ref_py) <= TOL["PY"], _relerr(G_PY, ref_py)
    assert _relerr(G_PP, ref_pp) <= TOL["PP"], _relerr(G_PP, ref_pp)


@pytest.mark.parametrize("name", ["tiny", "small_p1", "small_p2"])
def test_cellmat_mass(name):
    import torch
    from paper_1907_01005_gb300 import apply_M, harness
    cfg, pb = _problem(name)
    apply_M(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    r = O.run(cfg, fp32_inputs=True, H=O.assemble(O.BoxMesh.from_config(cfg), None, mass=True))
    dofs, cols, vals = harness.unpack_entries(pb, pb.dev["Y"].cpu().numpy())
    ref = np.asarray(r.Y.tocsr()[pb.keys[dofs], pb.perm[cols]]).ravel()
    assert _relerr(vals, ref) <= TOL["Y"], _relerr(vals, ref)


def test_cellmat_open_pattern():
    """A pattern that is not closed: Y keeps the masked entries of H P."""
    import torch
    from paper_1907_01005_gb300 import apply_H, harness
    cfg, pb = _problem("small_p2", pattern="support")
    apply_H(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    centres = inputs.orbital_centres(cfg)
    perm, ptr = O.column_blocks(blk, centres, cfg.n_col_blocks)
    mv = O.build_orbitals(mesh, cfg, centres, round_fp32=True)
    Psp = O.sparse_multivector(mesh, mv).tocsc()
    pat = np.zeros((blk.n_patches, len(ptr) - 1), bool)
    for c in range(len(ptr) - 1):
        for j in range(ptr[c], ptr[c + 1]):
            pat[blk.owner_rank(Psp.indices[Psp.indptr[perm[j]]:Psp.indptr[perm[j] + 1]]), c] = True
    Yref = O.apply_masked(O.assemble(mesh, O.potential_fn(cfg, True)), Psp, blk, pat,
                          O.entry_mask(blk, pat, perm, ptr))
    dofs, cols, vals = harness.unpack_entries(pb, pb.dev["Y"].cpu().numpy())
    ref = np.asarray(sp.csr_matrix(Yref)[pb.keys[dofs], pb.perm[cols]]).ravel()
    assert _relerr(vals, ref) <= TOL["Y"], _relerr(vals, ref)


def test_cellmat_empty_pattern():
    import torch
    from paper_1907_01005_gb300 import BCSR, FORM_CELLMAT, Mesh, apply_H
    m = Mesh(4, 4, 4, 0.25, 0.25, 0.25, 2)
    m.upload()
    m.set_potential(torch.zeros(int(m.info.n_q), dtype=torch.float32, device="cuda"), 1)
    R = m.n_row_blocks
    cbp = np.array([0, 8, 16], np.int32)
    P = BCSR(m, cbp, np.zeros(R + 1, np.int64), np.zeros(1, np.int32), 1)
    Y = BCSR(m, cbp, np.zeros(R + 1, np.int64), np.zeros(1, np.int32), 1)
    P.set_form(FORM_CELLMAT)
    pv, pt = P.alloc()
    yv, _ = Y.alloc(with_tables=False)
    P.bind(pv, pt)
    Y.bind(yv, None)
    apply_H(m, P, Y)
    torch.cuda.synchronize()
    assert m.check_device() == 0


def test_cellmat_repeat_and_forms_agree():
    """Two calls in a row agree (Y is re-zeroed; the work counter is reset),
    and the two forms agree within the FP32 tolerance."""
    import torch
    from paper_1907_01005_gb300 import FORM_SUMFAC, apply_H
    cfg, pb = _problem("small_p2")
    apply_H(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    Y1 = pb.dev["Y"].cpu().numpy()
    apply_H(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    Y2 = pb.dev["Y"].cpu().numpy()
    assert _relerr(Y2, Y1) <= 1e-6
    pb.P.set_form(FORM_SUMFAC)
    apply_H(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    Y3 = pb.dev["Y"].cpu().numpy()
    assert _relerr(Y1, Y3) <= TOL["Y"]


@pytest.mark.slow
def test_cellmat_paper_scale_p2():
    """846,369 DoFs x 320 orbitals at p = 2 through fe_apply_H_gram: Y on
    sampled rows (the oracle computes each from the cells around the node)
    and P^T P against the oracle's full FP64 product."""
    import torch
    from paper_1907_01005_gb300 import apply_H_gram
    cfg, pb = _problem("p2")
    d = pb.dev
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    Y = d["Y"].cpu().numpy()
    mesh = O.BoxMesh.from_config(cfg)
    centres = inputs.orbital_centres(cfg)
    mv = O.build_orbitals(mesh, cfg, centres, round_fp32=True)
    Psp = O.sparse_multivector(mesh, mv)
    rng = np.random.default_rng(11)
    ld, offs = pb.P.row_strides(), pb.P.block_offsets()
    stored_rb = np.nonzero(np.diff(pb.row_ptr) > 0)[0]
    dofs = np.unique(np.concatenate([rng.choice(np.arange(pb.rb_ptr[r], pb.rb_ptr[r + 1]), 3, replace=False)
                                     for r in rng.choice(stored_rb, 40, replace=False)]))
    ref_rows = O.apply_rows(mesh, O.potential_fn(cfg, True), Psp, pb.keys[dofs])
    kof = {}
    rows_of_k = np.repeat(np.arange(pb.mesh.n_row_blocks), np.diff(pb.row_ptr))
    for k in range(len(pb.col_idx)):
        kof[(rows_of_k[k], pb.col_idx[k])] = k
    got, ref = [], []
    for i, dof in enumerate(dofs):
        r = int(np.searchsorted(pb.rb_ptr, dof, side="right") - 1)
        for c in pb.col_idx[pb.row_ptr[r]:pb.row_ptr[r + 1]]:
            base = offs[kof[(r, c)]] + (dof - pb.rb_ptr[r]) * ld[c]
            for j in range(pb.cbp[c], pb.cbp[c + 1]):
                got.append(Y[base + j - pb.cbp[c]])
                ref.append(ref_rows[i, pb.perm[j]])
    assert _relerr(np.array(got), np.array(ref)) <= TOL["Y"]
    ref_pp = O.gram(Psp, Psp)[np.ix_(pb.perm, pb.perm)]
    assert _relerr(d["G_PP"].cpu().numpy(), ref_pp) <= TOL["PP"]


def test_cellmat_in_graph_and_host_entry():
    """The cell-matrix form inside a captured CUDA graph of the step and
    through the host-buffer entry point gives the eager device step's result
    (up to the order of the atomic additions)."""
    import torch
    from paper_1907_01005_gb300 import StepGraph, apply_H_gram, apply_H_gram_host
    cfg, pb = _problem("small_p2")
    d = pb.dev
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    Y0, Gpy0, Gpp0 = d["Y"].cpu().numpy(), d["G_PY"].cpu().numpy(), d["G_PP"].cpu().numpy()
    g = StepGraph(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    d["Y"].zero_()
    d["G_PY"].zero_()
    g.launch()
    g.launch()                               # replays reset the work counter and Y
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    assert _relerr(d["Y"].cpu().numpy(), Y0) <= 1e-6
    assert _relerr(d["G_PY"].cpu().numpy(), Gpy0) <= 1e-6
    assert _relerr(d["G_PP"].cpu().numpy(), Gpp0) <= 1e-14
    del g
    M = pb.n_cols
    Ph = torch.from_numpy(pb.P_host.copy()).pin_memory()
    Yh = torch.zeros(d["Y"].shape, dtype=d["Y"].dtype).pin_memory()
    G1 = torch.zeros((M, M), dtype=torch.float64).pin_memory()
    G2 = torch.zeros((M, M), dtype=torch.float64).pin_memory()
    apply_H_gram_host(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], Ph, Yh, G1, G2)
    assert pb.mesh.check_device() == 0
    assert _relerr(Yh.numpy(), Y0) <= 1e-6
    assert _relerr(G1.numpy(), Gpy0) <= 1e-6
    assert _relerr(G2.numpy(), Gpp0) <= 1e-14
