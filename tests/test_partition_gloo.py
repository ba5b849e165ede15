"""The row partition over ranks (Sec. 3.4, Alg. 3; Alg. 8's reduction) as a
world-size-2 gloo job on CPU, checked against the single-process oracle.

Each rank owns a contiguous range of row blocks, imports the ghost P tiles
of its lower-neighbour patches owned by the other rank, applies H to the
cells of its own patches (the oracle's assembly restricted to those cells
stands in for the per-rank kernel), sends its contributions to the other
rank's rows (compress), and all-reduces its partial P^T Y and P^T P.  The
finished own tiles of Y and both Gram products must equal the oracle's
single-process results."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(name):
    """Oracle reference plus the tile view of P and Y: rows of row block rb
    are its owned node keys in ascending order, columns of column block c
    the orbitals perm[ptr[c]:ptr[c+1]]."""
    import sys
    sys.path.insert(0, ROOT)
    from oracle import fe_oracle as O
    from synth import inputs
    cfg = inputs.get_config(name)
    r = O.run(cfg)
    blk = r.blk
    R = blk.n_patches
    own = blk.owner_rank(np.arange(r.mesh.n_nodes))
    rows_of = [np.nonzero(own == rb)[0] for rb in range(R)]
    widths = np.diff(r.ptr)
    cols_of = [r.perm[r.ptr[c]:r.ptr[c + 1]] for c in range(len(widths))]
    has = r.pattern
    row_ptr = np.concatenate([[0], np.cumsum(has.sum(1))]).astype(np.int64)
    col_idx = np.nonzero(has)[1].astype(np.int64)
    patch_xyz = blk.patch_xyz[blk.rank_to_patch]
    return cfg, r, rows_of, cols_of, widths, row_ptr, col_idx, patch_xyz


def _tile(S, rows, cols):
    return torch.from_numpy(np.asarray(S.tocsr()[rows][:, cols].todense()))


def _rank_main(rank, world, port, name, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import scipy.sparse as sp
    import torch.distributed as dist
    from oracle import fe_oracle as O
    from paper_1907_01005_gb300 import partition as PT
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg, r, rows_of, cols_of, widths, row_ptr, col_idx, patch_xyz = _problem(name)
    part = PT.RowPartition(patch_xyz, row_ptr, col_idx, np.array([len(x) for x in rows_of]), widths, world)
    mine = list(part.own(rank))
    P_own = {(rb, c): _tile(r.P, rows_of[rb], cols_of[c]) for rb in mine for c in sorted(part.pattern(rb))}
    # update ghost values: the imported tiles equal the owner's
    ghosts = PT.update_ghosts(part, rank, P_own)
    assert set(ghosts) == {k for v in part.ghosts(rank).values() for k in v}
    for (q, c), t in ghosts.items():
        assert torch.equal(t, _tile(r.P, rows_of[q], cols_of[c]))
    # the rank's local P: own rows and ghosts, zero elsewhere
    n, M = r.P.shape
    I, J, V = [], [], []
    for (rb, c), t in list(P_own.items()) + list(ghosts.items()):
        rr, cc = np.meshgrid(rows_of[rb], cols_of[c], indexing="ij")
        I.append(rr.ravel()); J.append(cc.ravel()); V.append(t.numpy().ravel())
    P_loc = sp.csr_matrix((np.concatenate(V), (np.concatenate(I), np.concatenate(J))), shape=(n, M))
    # H on the cells of the rank's own patches only
    blk = r.blk
    cells = np.arange(r.mesh.n_cells)
    prank = blk.cell_rank(cells) // 8
    my_cells = cells[(prank >= part.ranges[rank]) & (prank < part.ranges[rank + 1])]
    H_r = O.assemble(r.mesh, O.potential_fn(cfg), cells=my_cells)
    HP = sp.csr_matrix(H_r @ P_loc)
    halo_keys = [k for v in part.halo(rank).values() for k in v]
    Y_part = {k: _tile(HP, rows_of[k[0]], cols_of[k[1]]) for k in list(P_own) + halo_keys}
    Y_own = PT.compress(part, rank, Y_part)
    err_y = 0.0
    for (rb, c), t in Y_own.items():
        ref = _tile(r.Y, rows_of[rb], cols_of[c])
        err_y = max(err_y, float((t - ref).abs().max()))
    # partial Gram products over the own rows, then the sum over ranks
    G_py = torch.zeros(M, M, dtype=torch.float64)
    G_pp = torch.zeros(M, M, dtype=torch.float64)
    for rb in mine:
        cs = sorted(part.pattern(rb))
        for c1 in cs:
            for c2 in cs:
                i1 = torch.from_numpy(cols_of[c1]); i2 = torch.from_numpy(cols_of[c2])
                G_py[i1[:, None], i2[None, :]] += P_own[(rb, c1)].T @ Y_own[(rb, c2)]
                G_pp[i1[:, None], i2[None, :]] += P_own[(rb, c1)].T @ P_own[(rb, c2)]
    G_py = PT.reduce_gram(G_py)
    G_pp = PT.reduce_gram(G_pp)
    sy = float(np.abs(r.G_PY).max())
    sp_ = float(np.abs(r.G_PP).max())
    out[rank] = dict(
        err_y=err_y / max(1e-300, float(abs(r.Y).max())),
        err_py=float((G_py.numpy() - r.G_PY).__abs__().max()) / sy,
        err_pp=float((G_pp.numpy() - r.G_PP).__abs__().max()) / sp_,
        n_own=len(mine), n_ghost=len(ghosts), n_halo=len(halo_keys))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["small_p2", "small_p4"])
def test_row_partition_two_gloo_ranks(name):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, name, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        d = res[rank]
        assert d["n_own"] > 0 and d["n_ghost"] + d["n_halo"] >= 0
        assert d["err_y"] < 1e-12, d
        assert d["err_py"] < 1e-12, d
        assert d["err_pp"] < 1e-12, d
    # rank 1's patches sit above rank 0's: it imports ghosts, rank 0 none
    assert res[1]["n_ghost"] > 0 and res[0]["n_ghost"] == 0


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_partition_index_logic(world):
    """Host logic without communication: ranges cover the row blocks once,
    each rank's ghosts are exactly what its peers send, and every tile that
    the cells of a rank's patches touch is either its own or a ghost."""
    import sys
    sys.path.insert(0, ROOT)
    from paper_1907_01005_gb300 import partition as PT
    _, r, rows_of, cols_of, widths, row_ptr, col_idx, patch_xyz = _problem("small_p2")
    part = PT.RowPartition(patch_xyz, row_ptr, col_idx, np.array([len(x) for x in rows_of]), widths, world)
    R = len(rows_of)
    assert part.ranges[0] == 0 and part.ranges[-1] == R and np.all(np.diff(part.ranges) >= 0)
    assert sorted(sum((list(part.own(k)) for k in range(world)), [])) == list(range(R))
    for rank in range(world):
        for peer, keys in part.ghosts(rank).items():
            assert part.ghost_sends(peer)[rank] == keys
            assert all(part.owner(q) == peer for q, _ in keys)
        touched = set()
        for p in part.own(rank):
            for q in part.lower_neighbours(p) + [p]:
                touched.update((q, c) for c in part.pattern(q))
        have = {(rb, c) for rb in part.own(rank) for c in part.pattern(rb)}
        have |= {k for v in part.ghosts(rank).values() for k in v}
        assert touched <= have
    # lower neighbours: patch coordinates differ by an offset in {0,1}^3 \ {0}
    for rb in range(R):
        for q in part.lower_neighbours(rb):
            d = patch_xyz[rb] - patch_xyz[q]
            assert set(d.tolist()) <= {0, 1} and d.sum() > 0
