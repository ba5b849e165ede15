"""Row partition of the hot path over ranks (Sec. 3.4, Alg. 3; Alg. 8's
reduction of the M x M products).

The row blocks (patches of 2x2x2 cells in Morton order) are split into
contiguous ranges, one per rank, balanced by stored values.  A rank applies
H to the cells of its own patches.  Those cells touch, besides the rank's own
rows, the lower-face rows that belong to the (at most 7) lower neighbour
patches (owner rule: the component-wise lowest patch owns a shared node),
so:
  * ghosts (Alg. 3, "update ghost values"): the rank imports the P tiles
    (row block q, column block c) of the lower neighbours q owned elsewhere,
    for every column block c that q stores (the cells of an own patch read
    q's face rows in every such block, whether or not the patch itself
    stores c);
  * halo ("compress"): the rank's contributions to those rows, the Y tiles
    of the same set (Y keeps q's pattern), are sent to q's owner, which adds
    them to its own partial sums in a fixed order (by source rank, then
    tile);
  * Gram: every rank forms P^T Y and P^T P over its own rows; one sum over
    ranks (all-reduce) gives the M x M results.
Tiles travel packed into one contiguous buffer per peer (copied out of the
multivector first, copied back in after), in the order both sides derive
from the partition alone.

This module holds the index logic and the exchanges (torch.distributed
point-to-point and all-reduce); tiles are tensors of rows x width.  A tile
store is a dict {(row block, column block): tensor}.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch
import torch.distributed as dist

# lower-neighbour offsets e = (dx, dy, dz) in {0,1}^3 \ {0}: the neighbour is
# patch (px - dx, py - dy, pz - dz)
_OFFSETS = [(e & 1, (e >> 1) & 1, (e >> 2) & 1) for e in range(1, 8)]


@dataclass
class RowPartition:
    """Contiguous row-block ranges per rank and the tile sets each rank
    imports (ghosts of P) and exports (halo of Y).

    patch_xyz  (R, 3) patch coordinates of row block r (Morton order)
    row_ptr, col_idx  the block pattern (CSR over row blocks)
    rows       (R,) rows of each row block
    widths     (n_col_blocks,) columns of each column block
    world      number of ranks
    """
    patch_xyz: np.ndarray
    row_ptr: np.ndarray
    col_idx: np.ndarray
    rows: np.ndarray
    widths: np.ndarray
    world: int
    ranges: np.ndarray = field(init=False)
    _pat: list = field(init=False, repr=False)
    _rb_of_xyz: dict = field(init=False, repr=False)

    def __post_init__(self):
        R = len(self.rows)
        if self.world < 1:
            raise ValueError("world size must be at least 1")
        self._pat = [set(self.col_idx[self.row_ptr[r]:self.row_ptr[r + 1]].tolist()) for r in range(R)]
        self._rb_of_xyz = {tuple(int(v) for v in self.patch_xyz[r]): r for r in range(R)}
        # balance stored values: rows x (sum of the stored blocks' widths)
        work = np.array([self.rows[r] * sum(int(self.widths[c]) for c in self._pat[r]) for r in range(R)],
                        dtype=np.float64)
        cum = np.concatenate([[0.0], np.cumsum(work)])
        cuts = [0]
        for k in range(1, self.world):
            cuts.append(int(np.searchsorted(cum, cum[-1] * k / self.world, side="left")))
        cuts.append(R)
        self.ranges = np.maximum.accumulate(np.array(cuts, dtype=np.int64))

    # ---- ownership and neighbours -------------------------------------------
    def owner(self, rb: int) -> int:
        return int(np.searchsorted(self.ranges, rb, side="right") - 1)

    def own(self, rank: int) -> range:
        return range(int(self.ranges[rank]), int(self.ranges[rank + 1]))

    def lower_neighbours(self, rb: int) -> list[int]:
        px, py, pz = (int(v) for v in self.patch_xyz[rb])
        out = []
        for dx, dy, dz in _OFFSETS:
            q = self._rb_of_xyz.get((px - dx, py - dy, pz - dz))
            if q is not None:
                out.append(q)
        return out

    def pattern(self, rb: int) -> set:
        return self._pat[rb]

    # ---- Alg. 3: the tiles a rank needs from, and owes to, other ranks -------
    def boundary_tiles(self, rank: int) -> dict[int, list[tuple[int, int]]]:
        """{peer: sorted (q, c)}: tiles of row blocks q owned by peer != rank
        that the cells of this rank's patches touch, for the column blocks c
        that q stores.  The same set is imported as P (ghosts) and exported as
        Y contributions (halo)."""
        need: dict[int, set] = {}
        for p in self.own(rank):
            for q in self.lower_neighbours(p):
                peer = self.owner(q)
                if peer == rank or not self._pat[q]:
                    continue
                need.setdefault(peer, set()).update((q, c) for c in self._pat[q])
        return {peer: sorted(v) for peer, v in sorted(need.items())}

    def ghosts(self, rank: int) -> dict[int, list[tuple[int, int]]]:
        """P tiles to import, by owning peer (update ghost values)."""
        return self.boundary_tiles(rank)

    def ghost_sends(self, rank: int) -> dict[int, list[tuple[int, int]]]:
        """P tiles of this rank's row blocks that peers import."""
        out = {}
        for peer in range(self.world):
            if peer != rank:
                t = self.boundary_tiles(peer).get(rank)
                if t:
                    out[peer] = t
        return out

    def halo(self, rank: int) -> dict[int, list[tuple[int, int]]]:
        """Y tiles of other ranks' rows this rank contributes to (compress)."""
        return self.boundary_tiles(rank)

    def halo_receives(self, rank: int) -> dict[int, list[tuple[int, int]]]:
        """Y tiles of this rank's rows that peers contribute to."""
        return self.ghost_sends(rank)


# ---- exchanges ------------------------------------------------------------------
def _pack(tiles: dict, keys: list) -> torch.Tensor:
    """The listed tiles copied into one contiguous buffer, in list order."""
    return torch.cat([tiles[k].reshape(-1) for k in keys]) if keys else torch.empty(0)


def _unpack(buf: torch.Tensor, keys: list, shape_of) -> dict:
    out, o = {}, 0
    for k in keys:
        shp = shape_of(k)
        n = int(np.prod(shp))
        out[k] = buf[o:o + n].reshape(shp).clone()
        o += n
    if o != buf.numel():
        raise ValueError("exchange buffer size does not match the partition")
    return out


def _tile_shape(part: RowPartition, key) -> tuple[int, int]:
    q, c = key
    return int(part.rows[q]), int(part.widths[c])


def _exchange(part: RowPartition, rank: int, sends: dict, recvs: dict, tiles: dict, dtype) -> dict:
    """Point-to-point: one packed buffer to every peer in `sends`, one from
    every peer in `recvs`; returns {peer: {key: tile}}."""
    reqs, inbox = [], {}
    device = next(iter(tiles.values())).device if tiles else torch.device("cpu")
    for peer, keys in recvs.items():
        n = sum(int(np.prod(_tile_shape(part, k))) for k in keys)
        inbox[peer] = torch.empty(n, dtype=dtype, device=device)
        reqs.append(dist.irecv(inbox[peer], src=peer))
    outbox = {peer: _pack(tiles, keys).to(dtype).contiguous() for peer, keys in sends.items()}
    for peer, buf in outbox.items():
        reqs.append(dist.isend(buf, dst=peer))
    for r in reqs:
        r.wait()
    return {peer: _unpack(inbox[peer], recvs[peer], lambda k: _tile_shape(part, k)) for peer in sorted(inbox)}


def update_ghosts(part: RowPartition, rank: int, P_own: dict, dtype=torch.float64) -> dict:
    """Alg. 3 / Sec. 3.1 "update ghost values": returns the ghost P tiles
    {(q, c): tile} this rank imports (P_own holds its own row blocks)."""
    got = _exchange(part, rank, part.ghost_sends(rank), part.ghosts(rank), P_own, dtype)
    out = {}
    for peer in sorted(got):
        out.update(got[peer])
    return out


def compress(part: RowPartition, rank: int, Y_partial: dict, dtype=torch.float64) -> dict:
    """Sec. 3.1 "compress": sends this rank's contributions to other ranks'
    rows and adds the contributions to its own rows, by source rank in
    ascending order (a fixed order, so the result does not depend on
    arrival).  Y_partial holds this rank's partial sums for its own tiles
    and for the halo tiles; returns the finished own tiles."""
    got = _exchange(part, rank, part.halo(rank), part.halo_receives(rank), Y_partial, dtype)
    own = {k: v.clone() for k, v in Y_partial.items() if part.owner(k[0]) == rank}
    for peer in sorted(got):
        for k, v in got[peer].items():
            own[k] = own[k] + v
    return own


def reduce_gram(G_partial: torch.Tensor) -> torch.Tensor:
    """Alg. 8's reduction: the M x M partial products of all ranks summed."""
    G = G_partial.clone()
    dist.all_reduce(G, op=dist.ReduceOp.SUM)
    return G
