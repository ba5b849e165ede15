"""FP64 CPU oracle for the matrix-free BCSR Hamiltonian hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this module.  It shares no code with the
CUDA library: it computes its own 1D points, shape functions, mesh numbering,
row blocks, column blocks, patterns, assembled operator and Gram products.

What it computes (Davydov & Kronbichler, arXiv:1907.01005):

* Eq. (fe_matrices), Sec. 3.1: for Lagrange Q_p elements on hexahedra,
      M_ij = sum_K int_K N_i N_j,
      H_ij = sum_K int_K [ 1/2 grad N_i . grad N_j + N_i V N_j ],
  with H = -1/2 Laplacian + V (Sec. 2).  Element integrals are evaluated by
  brute force: every 3D shape function and its gradient is evaluated directly
  (a product of 1D Lagrange polynomials, no sum factorisation) at every point
  of a tensor Gauss rule with p+1 points per direction.
* Eq. (fe_matrices_cell_based), Sec. 3.2: H = sum_K P_K^T H_K P_K, assembled
  into a global CSR matrix (scipy.sparse).  Homogeneous Dirichlet conditions
  (the space is a subspace of H^1_0, Sec. 3.1) are applied by dropping every
  row and column that belongs to a boundary node.
* Alg. 1 (row renumbering and blocking), read for a structured box: the coarse
  cells are 2x2x2 patches ordered along a Morton curve; a row block holds the
  nodes of one patch not claimed by an earlier patch, so a node belongs to the
  component-wise lowest patch that contains it.
* Alg. 2 (column renumbering and blocking): every orbital is located in the
  cell that contains its centre, orbitals are sorted by the position of that
  cell in the ordered cell list (ties by orbital id), and the sorted list is
  split into contiguous groups of near-equal size.
* Sec. 3.5 (the destination pattern grows): the block pattern of a column
  block holds every row block that owns a node of a cell that contains a node
  of the column block's support.  With this closed pattern mask(P) * (H P)
  equals H P.
* Y = mask(P) * (H P): the matrix-free SpMM of Alg. 6 restricted to P's
  block pattern, computed here as an assembled SpMM.
* Alg. 8 (Tmmult), by its definition C = A^T B: G_PY = P^T Y and G_PP = P^T P
  over the stored blocks, in FP64.
* Alg. 7 (mmult) with a destination pattern, and the orbital-minimisation
  quantities of Sec. 2: the energy (Eq. energy), its gradient (Eq. gradient,
  built from Eqs. inner1/inner2 and G_ops1/G_ops2) and the directional
  derivative tr(D^T G) (Eq. G_ops4).

Every function is pinned by tests/test_oracle_pins.py against closed forms,
brute force on tiny inputs, or numbers printed in the paper.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# 1D points and Lagrange polynomials
# ---------------------------------------------------------------------------


def gauss_points(n: int):
    """Gauss-Legendre points and weights on [0, 1] (n points, exact for
    polynomial degree 2n-1)."""
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def gll_points(p: int) -> np.ndarray:
    """Support points of Q_p on [0, 1]: the Gauss-Lobatto-Legendre points,
    i.e. 0, 1 and the roots of P_p'(t) mapped from [-1, 1].  (Reading: the
    paper does not name the support points; this is the FE_Q convention of
    the library it builds on.)"""
    if p == 1:
        return np.array([0.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(p).deriv().roots()
    inner = np.sort(np.real(inner))
    return np.concatenate([[0.0], 0.5 * (inner + 1.0), [1.0]])


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[k, j] = l_j(x_k), with l_j the Lagrange polynomial through `nodes`
    that is 1 at nodes[j] and 0 at the others (product formula)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    L = np.ones((len(x), m))
    for j in range(m):
        for k in range(m):
            if k != j:
                L[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return L


def lagrange_derivs(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[k, j] = l_j'(x_k): derivative of the product formula by the product
    rule, sum over the dropped factor."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    D = np.zeros((len(x), m))
    for j in range(m):
        for drop in range(m):
            if drop == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[drop]))
            for k in range(m):
                if k != j and k != drop:
                    term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            D[:, j] += term
    return D


# ---------------------------------------------------------------------------
# Reference cell tables (brute force, no sum factorisation)
# ---------------------------------------------------------------------------


@dataclass
class RefCell:
    p: int
    nodes1d: np.ndarray      # GLL points on [0,1]
    qpts1d: np.ndarray       # Gauss points on [0,1]
    qw1d: np.ndarray
    B: np.ndarray            # (nq, nn) shape values N_a(xi_q)
    G: np.ndarray            # (3, nq, nn) reference gradients dN_a/dxi_d (xi_q)
    W: np.ndarray            # (nq,) tensor weights
    qxi: np.ndarray          # (nq, 3) reference coordinates of the q-points


def ref_cell(p: int) -> RefCell:
    """Tables of every 3D shape function N_a(xi) = l_ax(xi_x) l_ay(xi_y) l_az(xi_z)
    and its reference gradient at every tensor Gauss point.  Node index
    a = ax + (p+1)(ay + (p+1) az); q-point index q = qx + n(qy + n qz)."""
    n = p + 1
    nodes = gll_points(p)
    qp, qw = gauss_points(n)
    l = lagrange_values(nodes, qp)      # (n, p+1)
    dl = lagrange_derivs(nodes, qp)
    nn, nq = (p + 1) ** 3, n ** 3
    B = np.zeros((nq, nn))
    G = np.zeros((3, nq, nn))
    W = np.zeros(nq)
    qxi = np.zeros((nq, 3))
    for qz in range(n):
        for qy in range(n):
            for qx in range(n):
                q = qx + n * (qy + n * qz)
                W[q] = qw[qx] * qw[qy] * qw[qz]
                qxi[q] = (qp[qx], qp[qy], qp[qz])
                for az in range(p + 1):
                    for ay in range(p + 1):
                        for ax in range(p + 1):
                            a = ax + (p + 1) * (ay + (p + 1) * az)
                            B[q, a] = l[qx, ax] * l[qy, ay] * l[qz, az]
                            G[0, q, a] = dl[qx, ax] * l[qy, ay] * l[qz, az]
                            G[1, q, a] = l[qx, ax] * dl[qy, ay] * l[qz, az]
                            G[2, q, a] = l[qx, ax] * l[qy, ay] * dl[qz, az]
    return RefCell(p, nodes, qp, qw, B, G, W, qxi)


# ---------------------------------------------------------------------------
# Mesh: a box of nx*ny*nz axis-aligned cells of size hx*hy*hz with Q_p nodes
# ---------------------------------------------------------------------------


class BoxMesh:
    """Nodes live on the lattice (p nx + 1) x (p ny + 1) x (p nz + 1); the
    oracle numbers them by their lattice key  I + Lx (J + Ly K)."""

    def __init__(self, nx, ny, nz, hx, hy, hz, p, dirichlet=1):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.h = np.array([hx, hy, hz], dtype=np.float64)
        self.p = int(p)
        self.dirichlet = int(dirichlet)
        self.L = np.array([p * nx + 1, p * ny + 1, p * nz + 1], dtype=np.int64)
        self.n_nodes = int(np.prod(self.L))
        self.n_cells = self.nx * self.ny * self.nz
        self.ref = ref_cell(self.p)

    @classmethod
    def from_config(cls, cfg):
        return cls(cfg.nx, cfg.ny, cfg.nz, cfg.hx, cfg.hy, cfg.hz, cfg.p, cfg.dirichlet)

    # lattice helpers -------------------------------------------------------
    def key(self, I, J, K):
        return I + self.L[0] * (J + self.L[1] * K)

    def ijk(self, key):
        key = np.asarray(key, dtype=np.int64)
        I = key % self.L[0]
        J = (key // self.L[0]) % self.L[1]
        K = key // (self.L[0] * self.L[1])
        return I, J, K

    def node_coords(self, key=None) -> np.ndarray:
        """Physical coordinates x = h (cell + xi_local) of lattice nodes."""
        if key is None:
            key = np.arange(self.n_nodes, dtype=np.int64)
        ijk = self.ijk(key)
        out = np.empty((len(ijk[0]), 3))
        ncell = (self.nx, self.ny, self.nz)
        for d in range(3):
            c = np.minimum(ijk[d] // self.p, ncell[d] - 1)
            loc = ijk[d] - self.p * c
            out[:, d] = self.h[d] * (c + self.ref.nodes1d[loc])
        return out

    def boundary(self, key=None) -> np.ndarray:
        if key is None:
            key = np.arange(self.n_nodes, dtype=np.int64)
        if not self.dirichlet:
            return np.zeros(len(np.atleast_1d(key)), dtype=bool)
        I, J, K = self.ijk(key)
        return ((I == 0) | (I == self.L[0] - 1) | (J == 0) | (J == self.L[1] - 1)
                | (K == 0) | (K == self.L[2] - 1))

    def cell_index(self, cx, cy, cz):
        return cx + self.nx * (cy + self.ny * cz)

    def cell_nodes(self, cells=None) -> np.ndarray:
        """(ncells, (p+1)^3) lattice keys of the nodes of each cell, in the
        reference order a = ax + (p+1)(ay + (p+1) az)."""
        if cells is None:
            cells = np.arange(self.n_cells, dtype=np.int64)
        cells = np.asarray(cells, dtype=np.int64)
        cx = cells % self.nx
        cy = (cells // self.nx) % self.ny
        cz = cells // (self.nx * self.ny)
        p = self.p
        a = np.arange(p + 1)
        AX, AY, AZ = np.meshgrid(a, a, a, indexing="ij")
        # reference order: ax fastest -> flatten with order (az, ay, ax)
        AX = AX.transpose(2, 1, 0).ravel()
        AY = AY.transpose(2, 1, 0).ravel()
        AZ = AZ.transpose(2, 1, 0).ravel()
        I = p * cx[:, None] + AX[None, :]
        J = p * cy[:, None] + AY[None, :]
        K = p * cz[:, None] + AZ[None, :]
        return self.key(I, J, K)

    def cell_qpoints(self, cells=None) -> np.ndarray:
        """(ncells, nq, 3) physical Gauss points of each cell."""
        if cells is None:
            cells = np.arange(self.n_cells, dtype=np.int64)
        cells = np.asarray(cells, dtype=np.int64)
        cx = cells % self.nx
        cy = (cells // self.nx) % self.ny
        cz = cells // (self.nx * self.ny)
        c = np.stack([cx, cy, cz], axis=1).astype(np.float64)
        return (c[:, None, :] + self.ref.qxi[None, :, :]) * self.h[None, None, :]


# ---------------------------------------------------------------------------
# Element matrices and assembly (Eq. fe_matrices / fe_matrices_cell_based)
# ---------------------------------------------------------------------------


def element_matrices(mesh: BoxMesh, Vq: np.ndarray | None, mass: bool = False):
    """Element matrices for a batch of cells.

    Vq: (ncells, nq) potential values at the cells' Gauss points.
    Returns (ncells, nn, nn) with
        H_K[a,b] = sum_q W_q |J| [ 1/2 sum_d h_d^-2 G_d[q,a] G_d[q,b] + V_q B[q,a] B[q,b] ]
    or, with mass=True,  M_K[a,b] = sum_q W_q |J| B[q,a] B[q,b]  (Vq ignored).
    |J| = hx hy hz and dxi_d/dx_d = 1/h_d for the axis-aligned affine cell.
    """
    r = mesh.ref
    detJ = float(np.prod(mesh.h))
    wq = r.W * detJ
    if mass:
        Mk = (r.B * wq[:, None]).T @ r.B
        return Mk[None]
    lap = np.zeros((r.B.shape[1], r.B.shape[1]))
    for d in range(3):
        lap += (r.G[d] * (wq / mesh.h[d] ** 2)[:, None]).T @ r.G[d]
    lap *= 0.5
    if Vq is None:
        return lap[None]
    Vq = np.atleast_2d(Vq)
    # V part: B^T diag(wq V_K) B for every cell, as one matrix product
    X = (Vq * wq[None, :])[:, :, None] * r.B[None, :, :]          # (C, q, a)
    pot = np.einsum("cqa,qb->cab", X, r.B, optimize=True)
    return lap[None] + pot


def assemble(mesh: BoxMesh, Vfunc=None, mass: bool = False, chunk: int = 8192, cells=None):
    """Global CSR matrix over all lattice nodes (oracle numbering = lattice key),
    with Dirichlet rows and columns removed (set to zero) when mesh.dirichlet.
    With `cells`, only those cells are summed (rows whose cells are all in
    the subset are then complete)."""
    rows, cols, vals = [], [], []
    nn = (mesh.p + 1) ** 3
    all_cells = np.arange(mesh.n_cells, dtype=np.int64) if cells is None else np.asarray(cells, np.int64)
    for s in range(0, len(all_cells), chunk):
        cells = all_cells[s:s + chunk]
        keys = mesh.cell_nodes(cells)                      # (C, nn)
        if mass:
            Ek = np.broadcast_to(element_matrices(mesh, None, mass=True), (len(cells), nn, nn))
        else:
            if Vfunc is None:
                Vq = np.zeros((len(cells), mesh.ref.W.size))
            else:
                qp = mesh.cell_qpoints(cells)
                Vq = Vfunc(qp.reshape(-1, 3)).reshape(len(cells), -1)
            Ek = element_matrices(mesh, Vq)
            Ek = np.broadcast_to(Ek, (len(cells), nn, nn))
        rows.append(np.repeat(keys, nn, axis=1).ravel())
        cols.append(np.tile(keys, (1, nn)).ravel())
        vals.append(np.ascontiguousarray(Ek).ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes)).tocsr()
    A.sum_duplicates()
    if mesh.dirichlet:
        D = sp.diags((~mesh.boundary()).astype(np.float64))
        A = (D @ A @ D).tocsr()
        A.eliminate_zeros()
    return A


# ---------------------------------------------------------------------------
# Row blocks (Alg. 1 reading) and Morton order
# ---------------------------------------------------------------------------


def _spread3(v: np.ndarray, bits: int = 21) -> np.ndarray:
    """Bit b of v moved to bit 3b."""
    v = np.asarray(v, dtype=np.uint64)
    out = np.zeros_like(v)
    for b in range(bits):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton_code(px, py, pz) -> np.ndarray:
    """Morton (Z-order) code with x in bit 0, y in bit 1, z in bit 2 of each
    bit triple."""
    return _spread3(px) | (_spread3(py) << np.uint64(1)) | (_spread3(pz) << np.uint64(2))


class Blocking:
    """Patches (2x2x2 cells) in Morton order; row block r = patch of rank r."""

    def __init__(self, mesh: BoxMesh):
        if mesh.nx % 2 or mesh.ny % 2 or mesh.nz % 2:
            raise ValueError("cells per direction must be even")
        self.mesh = mesh
        self.np_ = np.array([mesh.nx // 2, mesh.ny // 2, mesh.nz // 2], dtype=np.int64)
        self.n_patches = int(np.prod(self.np_))
        pid = np.arange(self.n_patches, dtype=np.int64)
        px = pid % self.np_[0]
        py = (pid // self.np_[0]) % self.np_[1]
        pz = pid // (self.np_[0] * self.np_[1])
        code = morton_code(px, py, pz)
        order = np.lexsort((pid, code))       # rank -> natural patch id
        self.rank_to_patch = order
        self.patch_to_rank = np.empty_like(order)
        self.patch_to_rank[order] = np.arange(self.n_patches)
        self.patch_xyz = np.stack([px, py, pz], 1)   # by natural id

    def patch_id(self, px, py, pz):
        return px + self.np_[0] * (py + self.np_[1] * pz)

    def owner_rank(self, key) -> np.ndarray:
        """Row block of each node: the patch of lowest Morton rank containing
        it, which for a monotone order is the component-wise lowest patch."""
        I, J, K = self.mesh.ijk(key)
        q = 2 * self.mesh.p
        px = np.maximum(0, (I - 1) // q)
        py = np.maximum(0, (J - 1) // q)
        pz = np.maximum(0, (K - 1) // q)
        return self.patch_to_rank[self.patch_id(px, py, pz)]

    def rows_per_block(self) -> np.ndarray:
        own = self.owner_rank(np.arange(self.mesh.n_nodes))
        return np.bincount(own, minlength=self.n_patches)

    def cell_rank(self, cells) -> np.ndarray:
        """Position of each cell in the ordered active-cell list of Alg. 1:
        patches in Morton order, the 8 children of a patch lexicographically."""
        m = self.mesh
        cells = np.asarray(cells, dtype=np.int64)
        cx = cells % m.nx
        cy = (cells // m.nx) % m.ny
        cz = cells // (m.nx * m.ny)
        r = self.patch_to_rank[self.patch_id(cx // 2, cy // 2, cz // 2)]
        return 8 * r + (cx % 2) + 2 * (cy % 2) + 4 * (cz % 2)


# ---------------------------------------------------------------------------
# Column blocks (Alg. 2 reading)
# ---------------------------------------------------------------------------


def column_blocks(blk: Blocking, centres: np.ndarray, n_blocks: int):
    """Returns (perm, col_block_ptr): new column j holds orbital perm[j]; block
    c spans columns [ptr[c], ptr[c+1]).  The first M mod G blocks hold one
    extra column."""
    m = blk.mesh
    centres = np.asarray(centres, dtype=np.float64)
    M = len(centres)
    ncell = np.array([m.nx, m.ny, m.nz])
    cidx = np.clip(np.floor(centres / m.h[None, :]).astype(np.int64), 0, ncell[None, :] - 1)
    cells = m.cell_index(cidx[:, 0], cidx[:, 1], cidx[:, 2])
    rank = blk.cell_rank(cells)
    perm = np.lexsort((np.arange(M), rank))
    base, rem = divmod(M, n_blocks)
    sizes = np.array([base + (1 if g < rem else 0) for g in range(n_blocks)])
    ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return perm.astype(np.int64), ptr


# ---------------------------------------------------------------------------
# Supports, values and the closed block pattern
# ---------------------------------------------------------------------------


@dataclass
class Multivector:
    """Sparse multivector by lattice key: for each orbital alpha, the sorted
    node keys of its support and the values there (oracle side)."""
    keys: list          # list of int64 arrays
    vals: list          # list of float64 arrays


def build_orbitals(mesh: BoxMesh, cfg, centres=None, round_fp32: bool = False,
                   orbitals=None) -> Multivector:
    """Support = interior nodes with |x - c| <= R; values from the shared
    generator at the oracle's own node coordinates.  With `orbitals` (a set of
    ids) the other orbitals are left empty."""
    from synth import inputs
    if centres is None:
        centres = inputs.orbital_centres(cfg)
    keys, vals = [], []
    for a in range(len(centres)):
        if orbitals is not None and a not in orbitals:
            keys.append(np.zeros(0, np.int64))
            vals.append(np.zeros(0))
            continue
        lo, hi = centres[a] - cfg.radius, centres[a] + cfg.radius
        ks = _ball_candidates(mesh, lo, hi)
        xyz = mesh.node_coords(ks)
        sup = inputs.orbital_support(cfg, xyz, a, centres) & ~mesh.boundary(ks)
        ks = ks[sup]
        v = inputs.orbital_values(cfg, xyz[sup], ks, a, centres)
        if round_fp32:
            v = v.astype(np.float32).astype(np.float64)
        keys.append(ks)
        vals.append(v)
    return Multivector(keys, vals)


def _axis_coords(mesh: BoxMesh, d: int) -> np.ndarray:
    n = (mesh.nx, mesh.ny, mesh.nz)[d]
    I = np.arange(mesh.L[d])
    c = np.minimum(I // mesh.p, n - 1)
    return mesh.h[d] * (c + mesh.ref.nodes1d[I - mesh.p * c])


def _ball_candidates(mesh: BoxMesh, lo, hi) -> np.ndarray:
    idx = []
    for d in range(3):
        x = _axis_coords(mesh, d)
        idx.append(np.nonzero((x >= lo[d] - 1e-12) & (x <= hi[d] + 1e-12))[0])
    I, J, K = np.meshgrid(idx[0], idx[1], idx[2], indexing="ij")
    return np.sort(mesh.key(I.ravel(), J.ravel(), K.ravel()).astype(np.int64))


def block_pattern(blk: Blocking, mv: Multivector, perm: np.ndarray, ptr: np.ndarray) -> np.ndarray:
    """Boolean (n_row_blocks, n_col_blocks) closed pattern: (r, c) is set iff
    row block r owns a node of a cell that contains a support node of some
    orbital of column block c."""
    m = blk.mesh
    nb = len(ptr) - 1
    pat = np.zeros((blk.n_patches, nb), dtype=bool)
    for c in range(nb):
        ks = np.unique(np.concatenate([mv.keys[perm[j]] for j in range(ptr[c], ptr[c + 1])]
                                      + [np.zeros(0, np.int64)]))
        if len(ks) == 0:
            continue
        cells = mesh_cells_touching(m, ks)
        nodes = np.unique(m.cell_nodes(cells).ravel())
        pat[np.unique(blk.owner_rank(nodes)), c] = True
    return pat


def mesh_cells_touching(m: BoxMesh, keys: np.ndarray) -> np.ndarray:
    """All cells whose closure contains at least one of the given nodes."""
    I, J, K = m.ijk(keys)
    p = m.p
    out = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                cx = I // p - dx
                cy = J // p - dy
                cz = K // p - dz
                ok = (cx >= 0) & (cx < m.nx) & (cy >= 0) & (cy < m.ny) & (cz >= 0) & (cz < m.nz)
                ok &= (p * cx <= I) & (I <= p * (cx + 1))
                ok &= (p * cy <= J) & (J <= p * (cy + 1))
                ok &= (p * cz <= K) & (K <= p * (cz + 1))
                out.append(m.cell_index(cx[ok], cy[ok], cz[ok]))
    return np.unique(np.concatenate(out))


def entry_mask(blk: Blocking, pat: np.ndarray, perm: np.ndarray, ptr: np.ndarray):
    """mask[key, alpha] as a function: True iff (row block of key, column
    block of alpha) is in the pattern.  Returns (owner_rank per key,
    column block per orbital id)."""
    M = len(perm)
    cb_of_col = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    cb_of_orb = np.empty(M, dtype=np.int64)
    cb_of_orb[perm] = cb_of_col
    return cb_of_orb


def dense_multivector(mesh: BoxMesh, mv: Multivector, cols=None) -> np.ndarray:
    """Dense (n_nodes, len(cols)) FP64 array (small meshes / few columns)."""
    if cols is None:
        cols = range(len(mv.keys))
    cols = list(cols)
    P = np.zeros((mesh.n_nodes, len(cols)))
    for j, a in enumerate(cols):
        P[mv.keys[a], j] = mv.vals[a]
    return P


def sparse_multivector(mesh: BoxMesh, mv: Multivector) -> sp.csc_matrix:
    M = len(mv.keys)
    rows = np.concatenate(mv.keys) if M else np.zeros(0, np.int64)
    cols = np.concatenate([np.full(len(k), a) for a, k in enumerate(mv.keys)]) if M else rows
    vals = np.concatenate(mv.vals) if M else np.zeros(0)
    return sp.csc_matrix((vals, (rows, cols)), shape=(mesh.n_nodes, M))


# ---------------------------------------------------------------------------
# Y = mask(P) * (H P) and the Gram products (Alg. 6 result, Alg. 8)
# ---------------------------------------------------------------------------


def apply_masked(H: sp.csr_matrix, Psp: sp.csc_matrix, blk: Blocking, pat: np.ndarray,
                 cb_of_orb: np.ndarray) -> sp.csc_matrix:
    """Y = mask(P) * (H P) as a sparse (n_nodes, M) matrix."""
    HP = (H @ Psp).tocoo()
    own = blk.owner_rank(HP.row)
    keep = pat[own, cb_of_orb[HP.col]]
    return sp.csc_matrix((HP.data[keep], (HP.row[keep], HP.col[keep])), shape=HP.shape)


def gram(A: sp.spmatrix, B: sp.spmatrix) -> np.ndarray:
    """C = A^T B in FP64 (dense M x M)."""
    return np.asarray((A.T @ B).todense())


def mmult_masked(A: sp.spmatrix, X: np.ndarray, blk: Blocking, pat: np.ndarray,
                 cb_of_orb: np.ndarray) -> sp.csc_matrix:
    """Alg. 7 with a destination pattern: C = mask(pattern) * (A X), A a sparse
    (n_nodes, M) multivector, X a dense (M, M) matrix; the products that fall
    outside the destination's block pattern are discarded (the truncation of
    Alg. 7).  Returned as a sparse (n_nodes, M) matrix, FP64."""
    AX = sp.coo_matrix(np.asarray(A @ X))
    own = blk.owner_rank(AX.row)
    keep = pat[own, cb_of_orb[AX.col]]
    return sp.csc_matrix((AX.data[keep], (AX.row[keep], AX.col[keep])), shape=AX.shape)


def om_energy(Psp: sp.spmatrix, H: sp.spmatrix, M: sp.spmatrix) -> float:
    """Sec. 2, Eq. energy: E(Phi) = tr((2 I - Phi^T M Phi) Phi^T H Phi)."""
    Hb = gram(Psp, H @ Psp)
    Mb = gram(Psp, M @ Psp)
    return float(np.trace((2.0 * np.eye(Hb.shape[0]) - Mb) @ Hb))


def om_gradient(Psp: sp.spmatrix, PhiH: sp.spmatrix, PhiM: sp.spmatrix, blk: Blocking, pat: np.ndarray,
                cb_of_orb: np.ndarray):
    """Sec. 2, Eq. gradient with the operations of Eqs. inner1/inner2 and
    G_ops1/G_ops2: Hbar = Phi^T Phi_H, Mbar = Phi^T Phi_M,
    G = -2 Phi_M Hbar + 2 Phi_H (2 I - Mbar), truncated to the pattern.
    Returns (G, Hbar, Mbar)."""
    Hb = gram(Psp, PhiH)
    Mb = gram(Psp, PhiM)
    I = np.eye(Hb.shape[0])
    G = mmult_masked(PhiM, -2.0 * Hb, blk, pat, cb_of_orb) + mmult_masked(PhiH, 2.0 * (2.0 * I - Mb), blk, pat,
                                                                           cb_of_orb)
    return sp.csc_matrix(G), Hb, Mb


def trace_dot(D: sp.spmatrix, G: sp.spmatrix) -> float:
    """Eq. G_ops4: tr(D^T G) = sum_alpha D_alpha . G_alpha."""
    return float(D.multiply(G).sum())


def apply_rows(mesh: BoxMesh, Vfunc, Psp: sp.csc_matrix, keys: np.ndarray) -> np.ndarray:
    """(H P)[keys, :] computed one row at a time from the cells around each
    node (for sampling at sizes where the full assembly is too slow).  Rows
    of boundary nodes are zero (Dirichlet)."""
    keys = np.asarray(keys, dtype=np.int64)
    Pcsr = Psp.tocsr()
    out = np.zeros((len(keys), Psp.shape[1]))
    bnd = mesh.boundary(keys)
    nn = (mesh.p + 1) ** 3
    for i, k in enumerate(keys):
        if bnd[i]:
            continue
        cells = mesh_cells_touching(mesh, np.array([k]))
        cn = mesh.cell_nodes(cells)                          # (C, nn)
        Vq = Vfunc(mesh.cell_qpoints(cells).reshape(-1, 3)).reshape(len(cells), -1) \
            if Vfunc is not None else np.zeros((len(cells), mesh.ref.W.size))
        Ek = np.broadcast_to(element_matrices(mesh, Vq), (len(cells), nn, nn))
        for c in range(len(cells)):
            a = int(np.nonzero(cn[c] == k)[0][0])
            row = Ek[c, a, :].copy()
            row[mesh.boundary(cn[c])] = 0.0
            out[i] += Pcsr[cn[c]].T @ row
    return out


# ---------------------------------------------------------------------------
# One-call driver used by the tests
# ---------------------------------------------------------------------------


@dataclass
class OracleResult:
    mesh: BoxMesh
    blk: Blocking
    perm: np.ndarray
    ptr: np.ndarray
    pattern: np.ndarray
    cb_of_orb: np.ndarray
    P: sp.csc_matrix
    Y: sp.csc_matrix | None
    G_PY: np.ndarray | None
    G_PP: np.ndarray


def run(cfg, fp32_inputs: bool = False, with_apply: bool = True, H=None) -> OracleResult:
    """Whole hot path on the config: blocks, pattern, Y, P^T Y, P^T P.
    With fp32_inputs the P values and V are rounded to FP32 first (so the
    mixed-precision path is judged on its own arithmetic, not input rounding)."""
    from synth import inputs
    mesh = BoxMesh.from_config(cfg)
    blk = Blocking(mesh)
    centres = inputs.orbital_centres(cfg)
    perm, ptr = column_blocks(blk, centres, cfg.n_col_blocks)
    mv = build_orbitals(mesh, cfg, centres, round_fp32=fp32_inputs)
    pat = block_pattern(blk, mv, perm, ptr)
    cb_of_orb = entry_mask(blk, pat, perm, ptr)
    Psp = sparse_multivector(mesh, mv)
    G_PP = gram(Psp, Psp)
    Y = G_PY = None
    if with_apply:
        if H is None:
            H = assemble(mesh, potential_fn(cfg, fp32_inputs))
        Y = apply_masked(H, Psp, blk, pat, cb_of_orb)
        G_PY = gram(Psp, Y)
    return OracleResult(mesh, blk, perm, ptr, pat, cb_of_orb, Psp, Y, G_PY, G_PP)


def potential_fn(cfg, fp32: bool = False):
    from synth import inputs

    def V(xyz):
        v = inputs.potential(cfg, xyz)
        return v.astype(np.float32).astype(np.float64) if fp32 else v
    return V
