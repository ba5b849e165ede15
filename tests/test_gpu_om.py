"""Post-multiplication (Alg. 7), the orbital-minimisation gradient and the
directional derivative (Sec. 2, Eqs. gradient, G_ops1/G_ops2/G_ops4)
through the C ABI against the FP64 oracle.

Tolerances (normwise): FP64 1e-12.  FP32: the post-multiplication of FP32
values by X rounded to FP32 with FP32 sums of up to ~150 terms, 1e-5; the
gradient combines the FP32 apply (1e-5) with it, 1e-4; the trace sums the
exact FP64 products of the FP32 entries of G, so it inherits G's 1e-4."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

NAMES = ["tiny", "small_p2", "small_p4", "small_p1"]


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _like(pb, device="cuda"):
    """A multivector with P's pattern, bound to fresh device values."""
    from paper_1907_01005_gb300 import BCSR
    B = BCSR(pb.mesh, pb.cbp, pb.row_ptr, pb.col_idx, pb.dtype)
    v, t = B.alloc(device, with_tables=True)
    B.bind(v, t)
    return B


def _oracle_state(cfg, fp32):
    mesh = O.BoxMesh.from_config(cfg)
    r = O.run(cfg, fp32_inputs=fp32)
    Mmat = O.assemble(mesh, None, mass=True)
    PhiM = O.apply_masked(Mmat, r.P, r.blk, r.pattern, r.cb_of_orb)
    return r, PhiM


def _to_sparse(pb, values):
    from paper_1907_01005_gb300 import harness
    dofs, cols, vals = harness.unpack_entries(pb, values)
    n = int(pb.mesh.info.lx * pb.mesh.info.ly * pb.mesh.info.lz)
    return sp.csc_matrix((vals.astype(np.float64), (pb.keys[dofs], pb.perm[cols])), shape=(n, pb.n_cols))


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", NAMES)
def test_mmult_parity(name, dtype):
    import torch
    from paper_1907_01005_gb300 import harness, mmult
    cfg = inputs.get_config(name)
    pb = harness.build_problem(cfg, dtype)
    harness.to_device(pb)
    M = pb.n_cols
    rng = np.random.default_rng(11)
    X = rng.normal(size=(M, M))
    C = _like(pb)
    C.values.normal_()
    C0 = C.values.cpu().numpy().copy()
    Xd = torch.from_numpy(X).cuda()
    mmult(pb.P, Xd, C, alpha=0.5, gamma=-1.5, beta=2.0)
    torch.cuda.synchronize()
    got = _to_sparse(pb, C.values.cpu().numpy())
    r = O.run(cfg, fp32_inputs=(dtype == 1), with_apply=False)
    # X in the library's column order is X_lib[j, k] = X_orb[perm j, perm k]
    Xo = np.empty_like(X)
    Xo[np.ix_(pb.perm, pb.perm)] = X
    ref = 0.5 * (O.mmult_masked(r.P, Xo, r.blk, r.pattern, r.cb_of_orb) - 1.5 * r.P) + 2.0 * _to_sparse(pb, C0)
    tol = 1e-12 if dtype == 2 else 1e-5
    assert _relerr(got.toarray(), ref.toarray()) <= tol


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", NAMES)
def test_om_gradient_and_trace(name, dtype):
    import torch
    from paper_1907_01005_gb300 import apply_H, apply_M, gram_PtY, harness, om_gradient, trace_dot
    cfg = inputs.get_config(name)
    pb = harness.build_problem(cfg, dtype)
    harness.to_device(pb)
    d = pb.dev
    M = pb.n_cols
    YM, G, D = _like(pb), _like(pb), _like(pb)
    apply_H(pb.mesh, pb.P, pb.Y)
    apply_M(pb.mesh, pb.P, YM)
    Hb = torch.zeros((M, M), dtype=torch.float64, device="cuda")
    Mb = torch.zeros((M, M), dtype=torch.float64, device="cuda")
    gram_PtY(pb.P, pb.Y, Hb)
    gram_PtY(pb.P, YM, Mb)
    om_gradient(pb.Y, YM, Hb, Mb, G)
    g = torch.zeros(1, dtype=torch.float64, device="cuda")
    D.values.copy_(torch.from_numpy(np.random.default_rng(4).normal(size=D.values.numel())).to(D.values.dtype))
    trace_dot(D, G, g)
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    r, PhiM = _oracle_state(cfg, dtype == 1)
    Gref, _, _ = O.om_gradient(r.P, r.Y, PhiM, r.blk, r.pattern, r.cb_of_orb)
    got = _to_sparse(pb, G.values.cpu().numpy())
    tol = 1e-12 if dtype == 2 else 1e-4
    assert _relerr(got.toarray(), Gref.toarray()) <= tol
    Dsp = _to_sparse(pb, D.values.cpu().numpy())
    gref = O.trace_dot(Dsp, Gref)
    assert abs(float(g.item()) - gref) <= tol * O.trace_dot(abs(Dsp), abs(Gref))


def _rows_sparse(pb, values, rbs):
    """The stored entries of row blocks `rbs` as a sparse (n_nodes, M) matrix
    in oracle coordinates (lattice keys, orbital ids)."""
    offs, ld = pb.P.block_offsets(), pb.P.row_strides()
    dofs, cols, vals = [], [], []
    for r in rbs:
        nr = int(pb.rb_ptr[r + 1] - pb.rb_ptr[r])
        for k in range(pb.row_ptr[r], pb.row_ptr[r + 1]):
            c = pb.col_idx[k]
            w = int(pb.cbp[c + 1] - pb.cbp[c])
            vals.append(values[offs[k]: offs[k] + nr * ld[c]].reshape(nr, ld[c])[:, :w].ravel())
            dofs.append(np.repeat(np.arange(pb.rb_ptr[r], pb.rb_ptr[r + 1]), w))
            cols.append(np.tile(np.arange(pb.cbp[c], pb.cbp[c + 1]), nr))
    dofs, cols, vals = np.concatenate(dofs), np.concatenate(cols), np.concatenate(vals).astype(np.float64)
    n = int(pb.mesh.info.lx * pb.mesh.info.ly * pb.mesh.info.lz)
    return sp.csc_matrix((vals, (pb.keys[dofs], pb.perm[cols])), shape=(n, pb.n_cols))


@pytest.mark.slow
@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
def test_mmult_paper_scale_sampled(dtype):
    """846,369 DoFs x 320 orbitals at p = 2: row blocks hold up to 17 column
    blocks, so the widest span several 128-column chunks and the boundary
    ones several 64-row chunks.  Checked on the widest row blocks, boundary
    row blocks and random ones against the oracle's Alg. 7 on those rows."""
    import torch
    from paper_1907_01005_gb300 import harness, mmult
    cfg = inputs.get_config("p2")
    pb = harness.build_problem(cfg, dtype)
    harness.to_device(pb)
    M = pb.n_cols
    X = np.random.default_rng(5).normal(size=(M, M))
    C = _like(pb)
    C.values.normal_()
    C0 = C.values.cpu().numpy().copy()
    mmult(pb.P, torch.from_numpy(X).cuda(), C, alpha=0.5, gamma=-1.5, beta=2.0)
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    Cv = C.values.cpu().numpy()
    nblk = np.diff(pb.row_ptr)
    rows = np.diff(pb.rb_ptr)
    rng = np.random.default_rng(6)
    rbs = np.unique(np.concatenate([np.argsort(nblk)[-8:], np.nonzero(rows > 64)[0][:6],
                                    rng.choice(np.nonzero(nblk > 0)[0], 12, replace=False)]))
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    centres = inputs.orbital_centres(cfg)
    perm, ptr = O.column_blocks(blk, centres, cfg.n_col_blocks)
    mv = O.build_orbitals(mesh, cfg, centres, round_fp32=(dtype == 1))
    pat = O.block_pattern(blk, mv, perm, ptr)
    cb_of_orb = O.entry_mask(blk, pat, perm, ptr)
    Xo = np.empty_like(X)
    Xo[np.ix_(pb.perm, pb.perm)] = X
    A = _rows_sparse(pb, pb.P_host, rbs)
    ref = 0.5 * (O.mmult_masked(A, Xo, blk, pat, cb_of_orb) - 1.5 * A) + 2.0 * _rows_sparse(pb, C0, rbs)
    got = _rows_sparse(pb, Cv, rbs)
    tol = 1e-12 if dtype == 2 else 1e-5
    err = abs(got - ref).max() / abs(ref).max()            # sparse: the dense matrix would be 2 GB
    assert err <= tol, err
