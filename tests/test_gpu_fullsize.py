"""GPU parity at the paper-scale sizes (846,369 DoFs x 320 orbitals, p=2 and
p=4) and at the larger clustered workloads (1,686,177 DoFs x 640 orbitals),
through the same fe_apply_H_gram call the benchmark times.

The oracle cannot assemble and apply the whole operator quickly at this
size, so Y is checked on sampled rows (each computed one by one from the
cells around the node), among them rows on the patches' upper faces, edges
and corners, which receive halo contributions from the neighbour patches;
P^T P against the oracle's full FP64 product, and
P^T Y on four or more column blocks (among them both ends of the widest
union of a Gram work group), whose columns of Y the oracle computes from the
rows of the pattern only.  Tolerances are the normwise bounds of the
small-size tests, with the maximum taken over the checked entries.
"""
import numpy as np
import pytest

from oracle import fe_oracle as O
from synth import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = {2: dict(Y=1e-12, PY=1e-12, PP=1e-12), 1: dict(Y=1e-5, PY=1e-6, PP=1e-10)}


def _gpu(cfg, dtype):
    import torch
    from paper_1907_01005_gb300 import apply_H_gram, harness
    pb = harness.build_problem(cfg, dtype)
    harness.to_device(pb)
    d = pb.dev
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    return pb, d["Y"].cpu().numpy(), d["G_PY"].cpu().numpy(), d["G_PP"].cpu().numpy()


def _oracle_inputs(cfg, fp32):
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    centres = inputs.orbital_centres(cfg)
    perm, ptr = O.column_blocks(blk, centres, cfg.n_col_blocks)
    mv = O.build_orbitals(mesh, cfg, centres, round_fp32=fp32)
    pat = O.block_pattern(blk, mv, perm, ptr)
    cb_of_orb = O.entry_mask(blk, pat, perm, ptr)
    return mesh, blk, perm, ptr, mv, pat, cb_of_orb


CASES = [("p2", 1), ("p2", 2), ("p4", 1), ("p4", 2), ("large_p2", 1), ("large_p2", 2), ("large_p4", 1),
         ("large_p4", 2)]


def _pty_blocks(pb, rng, n=4):
    """Column blocks whose P^T Y columns are checked: those at both ends of the
    widest union of 8 consecutive row blocks (the Gram's work groups), the
    column block stored in the most row blocks, and random ones up to n."""
    w = np.diff(pb.cbp)
    best, uni = -1, None
    for r0 in range(0, pb.mesh.n_row_blocks, 8):
        u = np.unique(pb.col_idx[pb.row_ptr[r0]:pb.row_ptr[min(r0 + 8, pb.mesh.n_row_blocks)]])
        if len(u) and w[u].sum() > best:
            best, uni = w[u].sum(), u
    counts = np.bincount(pb.col_idx, minlength=len(w))
    pick = [int(uni[0]), int(uni[-1]), int(np.argmax(counts))]
    rest = [c for c in range(len(w)) if c not in pick]
    pick += [int(c) for c in rng.choice(rest, max(0, n - len(set(pick))), replace=False)]
    return sorted(set(pick))


@pytest.mark.parametrize("name,dtype", CASES, ids=[f"{n}-f{32 if d == 1 else 64}" for n, d in CASES])
def test_paper_scale(name, dtype):
    cfg = inputs.get_config(name)
    fp32 = dtype == 1
    pb, Y, G_PY, G_PP = _gpu(cfg, dtype)
    mesh, blk, perm, ptr, mv, pat, cb_of_orb = _oracle_inputs(cfg, fp32)
    Psp = O.sparse_multivector(mesh, mv)
    tol = TOL[dtype]

    # ---- P^T P: full FP64 product of the oracle ----------------------------
    ref_pp = O.gram(Psp, Psp)[np.ix_(pb.perm, pb.perm)]
    err = np.abs(G_PP - ref_pp).max() / np.abs(ref_pp).max()
    assert err <= tol["PP"], err

    # ---- Y on sampled rows ----------------------------------------------------
    rng = np.random.default_rng(7)
    ld = pb.P.row_strides()
    offs = pb.P.block_offsets()
    dense = {}
    rows_of_k = np.repeat(np.arange(pb.mesh.n_row_blocks), np.diff(pb.row_ptr))
    for k in range(len(pb.col_idx)):
        dense[(rows_of_k[k], pb.col_idx[k])] = k
    # rows with large values (near orbital centres) plus random stored rows
    stored_rb = np.nonzero(np.diff(pb.row_ptr) > 0)[0]
    sample_rb = rng.choice(stored_rb, 40, replace=False)
    dofs = np.concatenate([rng.choice(np.arange(pb.rb_ptr[r], pb.rb_ptr[r + 1]), 3, replace=False)
                           for r in sample_rb])
    # rows on the patches' upper faces, edges and corners: they receive the
    # halo contributions of the upper neighbour patches (1, 3 or 7 of them)
    q = 2 * cfg.p
    shared = []
    for r in sample_rb:
        dd = np.arange(pb.rb_ptr[r], pb.rb_ptr[r + 1])
        I, J, K = mesh.ijk(pb.keys[dd])
        on = ((I % q == 0) & (I > 0)).astype(int) + ((J % q == 0) & (J > 0)) + ((K % q == 0) & (K > 0))
        for lo in (1, 2, 3):
            cand = dd[on >= lo]
            if len(cand):
                shared.append(int(rng.choice(cand)))
    big = [int(np.argmax(np.abs(v))) for v in mv.vals[:6]]
    key_to_dof = np.empty(mesh.n_nodes, np.int64)
    key_to_dof[pb.keys] = np.arange(len(pb.keys))
    dofs = np.unique(np.concatenate([dofs, shared, [key_to_dof[mv.keys[a][i]] for a, i in enumerate(big)]]))
    keys = pb.keys[dofs]
    ref_rows = O.apply_rows(mesh, O.potential_fn(cfg, fp32), Psp, keys)   # (HP)[keys, orbital]
    got, ref = [], []
    for i, d in enumerate(dofs):
        r = int(np.searchsorted(pb.rb_ptr, d, side="right") - 1)
        for c in pb.col_idx[pb.row_ptr[r]:pb.row_ptr[r + 1]]:
            k = dense[(r, c)]
            base = offs[k] + (d - pb.rb_ptr[r]) * ld[c]
            for j in range(pb.cbp[c], pb.cbp[c + 1]):
                got.append(Y[base + j - pb.cbp[c]])
                ref.append(ref_rows[i, pb.perm[j]])
    got, ref = np.array(got), np.array(ref)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= tol["Y"], err

    # ---- P^T Y on sampled column blocks --------------------------------------
    for c in _pty_blocks(pb, rng):
        rows = np.nonzero(pat[:, c])[0]
        rkeys = np.nonzero(np.isin(blk.owner_rank(np.arange(mesh.n_nodes)), rows))[0]
        cells = O.mesh_cells_touching(mesh, rkeys)
        H = O.assemble(mesh, O.potential_fn(cfg, fp32), cells=cells)
        orbs = perm[ptr[c]:ptr[c + 1]]
        Pc = Psp[:, orbs]
        Yc = O.apply_masked(H, Pc, blk, pat, cb_of_orb[orbs])
        ref_py = O.gram(Psp, Yc)[pb.perm]                     # rows: all columns, cols: block c
        got_py = G_PY[:, ptr[c]:ptr[c + 1]]
        err = np.abs(got_py - ref_py).max() / np.abs(ref_py).max()
        assert err <= tol["PY"], err
