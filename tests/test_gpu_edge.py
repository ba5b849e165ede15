"""Edge cases on the GPU: a pattern that is not closed (Y keeps only the
masked entries of H P, and P^T Y is not symmetric) and an empty pattern."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL = {2: dict(Y=1e-12, PY=1e-12), 1: dict(Y=1e-5, PY=1e-6)}


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["small_p2", "small_p4", "small_p1"])
def test_open_pattern_mask_semantics(name, dtype):
    import torch
    from paper_1907_01005_gb300 import apply_H, gram_PtY, harness
    cfg = inputs.get_config(name)
    pb = harness.build_problem(cfg, dtype, pattern="support")
    harness.to_device(pb)
    d = pb.dev
    apply_H(pb.mesh, pb.P, pb.Y)
    gram_PtY(pb.P, pb.Y, d["G_PY"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    # oracle with the same (support-only) pattern
    fp32 = dtype == 1
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    perm, ptr = O.column_blocks(blk, inputs.orbital_centres(cfg), cfg.n_col_blocks)
    mv = O.build_orbitals(mesh, cfg, inputs.orbital_centres(cfg), round_fp32=fp32)
    Psp = O.sparse_multivector(mesh, mv).tocsc()
    nb = len(ptr) - 1
    pat = np.zeros((blk.n_patches, nb), bool)
    for c in range(nb):
        for j in range(ptr[c], ptr[c + 1]):
            a = perm[j]
            pat[blk.owner_rank(Psp.indices[Psp.indptr[a]:Psp.indptr[a + 1]]), c] = True
    cb_of_orb = O.entry_mask(blk, pat, perm, ptr)
    H = O.assemble(mesh, O.potential_fn(cfg, fp32))
    Yref = O.apply_masked(H, Psp, blk, pat, cb_of_orb)
    assert abs(len(pb.col_idx) - pat.sum()) == 0
    dofs, cols, vals = harness.unpack_entries(pb, d["Y"].cpu().numpy())
    ref = np.asarray(Yref.tocsr()[pb.keys[dofs], pb.perm[cols]]).ravel()
    assert _relerr(vals, ref) <= TOL[dtype]["Y"]
    G = d["G_PY"].cpu().numpy()
    Gref = O.gram(Psp, sp.csc_matrix(Yref))[np.ix_(pb.perm, pb.perm)]
    assert _relerr(G, Gref) <= TOL[dtype]["PY"]
    assert np.abs(Gref - Gref.T).max() > 1e-6 * np.abs(Gref).max()     # the mask is visible


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
def test_empty_pattern(dtype):
    import torch
    from paper_1907_01005_gb300 import BCSR, Mesh, apply_H_gram
    m = Mesh(4, 4, 4, 0.25, 0.25, 0.25, 2)
    m.upload()
    tdt = torch.float64 if dtype == 2 else torch.float32
    m.set_potential(torch.zeros(int(m.info.n_q), dtype=tdt, device="cuda"), dtype)
    R = m.n_row_blocks
    cbp = np.array([0, 8, 16], np.int32)
    P = BCSR(m, cbp, np.zeros(R + 1, np.int64), np.zeros(1, np.int32), dtype)
    Y = BCSR(m, cbp, np.zeros(R + 1, np.int64), np.zeros(1, np.int32), dtype)
    assert P.info.n_values == 0
    pv, pt = P.alloc()
    yv, _ = Y.alloc(with_tables=False)
    P.bind(pv, pt)
    Y.bind(yv, None)
    G1 = torch.full((16, 16), 7.0, dtype=torch.float64, device="cuda")
    G2 = torch.full((16, 16), 7.0, dtype=torch.float64, device="cuda")
    apply_H_gram(m, P, Y, G1, G2)
    torch.cuda.synchronize()
    assert m.check_device() == 0
    assert float(G1.abs().max()) == 0.0 and float(G2.abs().max()) == 0.0
