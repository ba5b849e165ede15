"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than itself: closed
forms of 1D/3D finite-element matrices, exact integrals of polynomials,
eigen-relations of tensor-product sine modes, brute-force loops on tiny
inputs, dense linear algebra, or mesh statistics printed in the paper
(Tables 1 and 3).  A dropped term, a wrong sign, a wrong scale factor, a
transposed operand or a wrong axis fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fe_oracle as O
from synth import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# 1D points
# ---------------------------------------------------------------------------
def test_gauss_points_closed_forms():
    x, w = O.gauss_points(3)
    r = 0.5 * math.sqrt(3.0 / 5.0)
    np.testing.assert_allclose(x, [0.5 - r, 0.5, 0.5 + r], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], rtol=0, atol=1e-15)
    # five-point rule, textbook values on [-1, 1]
    a = math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3
    b = math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3
    wa = (322 + 13 * math.sqrt(70)) / 900
    wb = (322 - 13 * math.sqrt(70)) / 900
    x, w = O.gauss_points(5)
    np.testing.assert_allclose(x, 0.5 * (np.array([-b, -a, 0, a, b]) + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * np.array([wb, wa, 128 / 225, wa, wb]), atol=1e-15)


def test_gll_points_closed_forms():
    np.testing.assert_allclose(O.gll_points(1), [0, 1])
    np.testing.assert_allclose(O.gll_points(2), [0, 0.5, 1], atol=1e-15)
    s5 = 0.5 / math.sqrt(5)
    np.testing.assert_allclose(O.gll_points(3), [0, 0.5 - s5, 0.5 + s5, 1], atol=1e-15)
    s = 0.5 * math.sqrt(3 / 7)
    np.testing.assert_allclose(O.gll_points(4), [0, 0.5 - s, 0.5, 0.5 + s, 1], atol=1e-15)


def test_lagrange_tables():
    nodes = O.gll_points(2)
    L = O.lagrange_values(nodes, nodes)
    np.testing.assert_allclose(L, np.eye(3), atol=1e-15)
    x = np.array([0.1, 0.37, 0.9])
    # closed forms on {0, 1/2, 1}
    l0 = 2 * (x - 0.5) * (x - 1)
    l1 = -4 * x * (x - 1)
    l2 = 2 * x * (x - 0.5)
    np.testing.assert_allclose(O.lagrange_values(nodes, x), np.stack([l0, l1, l2], 1), atol=1e-15)
    d = np.stack([4 * x - 3, -8 * x + 4, 4 * x - 1], 1)
    np.testing.assert_allclose(O.lagrange_derivs(nodes, x), d, atol=1e-14)


# ---------------------------------------------------------------------------
# Element matrices against textbook closed forms
# ---------------------------------------------------------------------------
def _q1(h):
    return (np.array([[1, -1], [-1, 1]]) / h, np.array([[2, 1], [1, 2]]) * h / 6)


def _q2(h):
    K = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / (3 * h)
    M = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) * h / 30
    return K, M


def _tensor3(Kx, Mx, Ky, My, Kz, Mz):
    """Stiffness and mass of a brick from 1D factors; node index
    a = ax + n (ay + n az) so the x factor is the innermost Kronecker factor."""
    K = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    M = np.kron(Mz, np.kron(My, Mx))
    return K, M


@pytest.mark.parametrize("p,f", [(1, _q1), (2, _q2)])
def test_element_matrices_textbook(p, f):
    hx, hy, hz = 0.5, 0.75, 1.25
    mesh = O.BoxMesh(2, 2, 2, hx, hy, hz, p, dirichlet=0)
    K, M = _tensor3(*f(hx), *f(hy), *f(hz))
    H0 = O.element_matrices(mesh, np.zeros((1, (p + 1) ** 3)))[0]
    np.testing.assert_allclose(H0, 0.5 * K, rtol=0, atol=1e-13 * np.abs(K).max())
    Mk = O.element_matrices(mesh, None, mass=True)[0]
    np.testing.assert_allclose(Mk, M, rtol=0, atol=1e-15 * np.abs(M).max() * 10)
    # constant potential c adds c * M (Eq. fe_matrices, V term)
    c = -1.7
    Hc = O.element_matrices(mesh, np.full((1, (p + 1) ** 3), c))[0]
    np.testing.assert_allclose(Hc, 0.5 * K + c * M, rtol=0, atol=1e-13 * np.abs(K).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_element_row_sums_and_volume(p):
    mesh = O.BoxMesh(2, 2, 2, 0.3, 0.7, 1.1, p, dirichlet=0)
    H0 = O.element_matrices(mesh, np.zeros((1, (p + 1) ** 3)))[0]
    assert np.abs(H0.sum(1)).max() < 1e-13 * np.abs(H0).max()   # constants in the kernel
    Mk = O.element_matrices(mesh, None, mass=True)[0]
    assert abs(Mk.sum() - 0.3 * 0.7 * 1.1) < 1e-15
    np.testing.assert_allclose(H0, H0.T, atol=1e-14)


# ---------------------------------------------------------------------------
# Assembled operator against exact integrals of polynomials
# ---------------------------------------------------------------------------
def _I(k, L):
    """int_0^L x^k dx."""
    return L ** (k + 1) / (k + 1)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_assembled_bilinear_form_on_polynomials(p):
    """u^T H w = 1/2 int grad u . grad w + int u V w for u, w monomials of
    degree <= p per variable and V linear: exact under Gauss with p+1 points."""
    hx, hy, hz = 0.5, 0.75, 1.25
    nx, ny, nz = 2, 2, 2
    Lx, Ly, Lz = nx * hx, ny * hy, nz * hz
    v = (1.0, 2.0, -1.0, 0.5)

    def Vf(xyz):
        return v[0] + v[1] * xyz[:, 0] + v[2] * xyz[:, 1] + v[3] * xyz[:, 2]

    mesh = O.BoxMesh(nx, ny, nz, hx, hy, hz, p, dirichlet=0)
    H = O.assemble(mesh, Vf)
    xyz = mesh.node_coords()
    ex = [(a, b, c) for c in range(p + 1) for b in range(p + 1) for a in range(p + 1)]
    U = np.stack([xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** c for a, b, c in ex], 1)
    got = U.T @ (H @ U)
    want = np.zeros_like(got)
    for i, (a, b, c) in enumerate(ex):
        for j, (d, e, f) in enumerate(ex):
            g = 0.0
            if a and d:
                g += a * d * _I(a + d - 2, Lx) * _I(b + e, Ly) * _I(c + f, Lz)
            if b and e:
                g += b * e * _I(a + d, Lx) * _I(b + e - 2, Ly) * _I(c + f, Lz)
            if c and f:
                g += c * f * _I(a + d, Lx) * _I(b + e, Ly) * _I(c + f - 2, Lz)
            s = v[0] * _I(a + d, Lx) * _I(b + e, Ly) * _I(c + f, Lz)
            s += v[1] * _I(a + d + 1, Lx) * _I(b + e, Ly) * _I(c + f, Lz)
            s += v[2] * _I(a + d, Lx) * _I(b + e + 1, Ly) * _I(c + f, Lz)
            s += v[3] * _I(a + d, Lx) * _I(b + e, Ly) * _I(c + f + 1, Lz)
            want[i, j] = 0.5 * g + s
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_assembled_identities_q2():
    """Interior rows away from the boundary: (K 1)_i = 0, (K x)_i = 0,
    (K x^2)_i = -2 (M 1)_i with K = 2 H(V=0), and (M 1)_i is the product of 1D
    node integrals (h/3 at a shared vertex, 2h/3 at a midpoint for Q2)."""
    h = 0.25
    mesh = O.BoxMesh(4, 4, 4, h, h, h, 2, dirichlet=1)
    K = 2.0 * O.assemble(mesh, None)
    M = O.assemble(mesh, None, mass=True)
    xyz = mesh.node_coords()
    I, J, Kk = mesh.ijk(np.arange(mesh.n_nodes))
    # rows whose cells contain no boundary node (lattice 0..8, cells of 2)
    inner = (I >= 3) & (I <= 5) & (J >= 3) & (J <= 5) & (Kk >= 3) & (Kk <= 5)
    one = np.ones(mesh.n_nodes) * ~mesh.boundary()
    x = xyz[:, 0] * ~mesh.boundary()
    x2 = xyz[:, 0] ** 2 * ~mesh.boundary()
    assert np.abs((K @ one)[inner]).max() < 1e-13
    assert np.abs((K @ x)[inner]).max() < 1e-13
    np.testing.assert_allclose((K @ x2)[inner], -2 * (M @ one)[inner], atol=1e-14)
    w1 = np.where(I % 2 == 0, h / 3, 2 * h / 3) * np.where(J % 2 == 0, h / 3, 2 * h / 3) \
        * np.where(Kk % 2 == 0, h / 3, 2 * h / 3)
    np.testing.assert_allclose((M @ one)[inner], w1[inner], rtol=1e-14)


# ---------------------------------------------------------------------------
# Sine modes: tensor products of 1D generalized eigenvectors
# ---------------------------------------------------------------------------
def _elem1d_numpy(p, h):
    """1D Q_p element stiffness and mass by exact polynomial integration with
    numpy.polynomial, on the GLL points (independent of the oracle's
    Lagrange and quadrature code)."""
    from numpy.polynomial import polynomial as Pl
    if p == 1:
        nodes = np.array([0.0, 1.0])
    else:
        r = np.sort(np.real(np.polynomial.legendre.Legendre.basis(p).deriv().roots()))
        nodes = np.concatenate([[0.0], 0.5 * (r + 1), [1.0]])
    basis = []
    for j in range(p + 1):
        others = np.delete(nodes, j)
        c = Pl.polyfromroots(others)
        c = c / Pl.polyval(nodes[j], c)
        basis.append(c)
    K = np.zeros((p + 1, p + 1))
    M = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            pm = Pl.polyint(Pl.polymul(basis[i], basis[j]))
            pk = Pl.polyint(Pl.polymul(Pl.polyder(basis[i]), Pl.polyder(basis[j])))
            M[i, j] = (Pl.polyval(1.0, pm) - Pl.polyval(0.0, pm)) * h
            K[i, j] = (Pl.polyval(1.0, pk) - Pl.polyval(0.0, pk)) / h
    return K, M


def _assemble1d(p, n, h, elem):
    N = p * n + 1
    K = np.zeros((N, N))
    M = np.zeros((N, N))
    Ke, Me = elem(p, h) if elem is _elem1d_numpy else elem(h)
    for c in range(n):
        s = slice(p * c, p * c + p + 1)
        K[s, s] += Ke
        M[s, s] += Me
    return K[1:-1, 1:-1], M[1:-1, 1:-1]   # Dirichlet


def test_q1_1d_closed_form_eigenvalues():
    n, h = 8, 1.0 / 8
    K, M = _assemble1d(1, n, h, _q1)
    mu, V = sla.eigh(K, M)
    k = np.arange(1, n)
    want = 6 / h ** 2 * (1 - np.cos(k * np.pi * h)) / (2 + np.cos(k * np.pi * h))
    np.testing.assert_allclose(mu, want, rtol=1e-13)
    xs = np.arange(1, n) * h
    for j, kk in enumerate(k):
        s = np.sin(kk * np.pi * xs)
        v = V[:, j] / V[np.argmax(np.abs(V[:, j])), j] * s[np.argmax(np.abs(V[:, j]))]
        np.testing.assert_allclose(v, s, atol=1e-12)


@pytest.mark.parametrize("p,n", [(1, 4), (2, 4), (3, 2), (4, 2)])
def test_sine_mode_eigen_relation_3d(p, n):
    """u = v_a (x) v_b (x) v_c satisfies H u = 1/2 (mu_a+mu_b+mu_c) M u (V = 0,
    homogeneous Dirichlet, unit cube)."""
    h = 1.0 / n
    elem = {1: _q1, 2: _q2}.get(p, _elem1d_numpy)
    K1, M1 = _assemble1d(p, n, h, elem)
    mu, V = sla.eigh(K1, M1)
    mesh = O.BoxMesh(n, n, n, h, h, h, p, dirichlet=1)
    H = O.assemble(mesh, None)
    Mg = O.assemble(mesh, None, mass=True)
    L = p * n + 1
    rng = np.random.default_rng(0)
    for _ in range(4):
        a, b, c = rng.integers(0, len(mu), size=3)
        u3 = np.zeros((L, L, L))   # index [K, J, I]
        u3[1:-1, 1:-1, 1:-1] = np.einsum("k,j,i->kji", V[:, c], V[:, b], V[:, a])
        u = u3.ravel()
        lhs = H @ u
        rhs = 0.5 * (mu[a] + mu[b] + mu[c]) * (Mg @ u)
        # 1e-11: the test-side 1D matrices come from monomial-basis integration
        assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(rhs).max()


def test_sine_mode_eigenvalue_convergence_q2():
    """The lowest 1D eigenvalue converges to pi^2 at rate h^(2p) = h^4."""
    errs = []
    for n in (4, 8, 16):
        K1, M1 = _assemble1d(2, n, 1.0 / n, _q2)
        errs.append(sla.eigh(K1, M1, eigvals_only=True)[0] - np.pi ** 2)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.array(errs) > 0) and np.all(rates > 3.7)


# ---------------------------------------------------------------------------
# Blocking, Morton order and column blocks
# ---------------------------------------------------------------------------
def test_paper_mesh_statistics():
    gold = json.load(open(os.path.join(GOLDEN, "paper_mesh_statistics.json")))
    cases = {"p2_c160": (64, 40, 40, 2), "p4_c160": (32, 20, 20, 4),
             "p2_c320": (128, 40, 40, 2), "p4_c320": (64, 20, 20, 4)}
    for k, (nx, ny, nz, p) in cases.items():
        g = gold[k]
        mesh = O.BoxMesh(nx, ny, nz, 1, 1, 1, p)
        blk = O.Blocking(mesh)
        assert mesh.n_cells == g["cells"]
        assert mesh.n_nodes == g["dofs"]
        assert (p + 1) ** 3 == g["dofs_per_cell"]
        assert blk.n_patches == g["row_blocks"]
        rows = blk.rows_per_block()
        assert rows.sum() == g["dofs"]
        # the paper prints the mean to a few decimals: agree to half an ulp of that
        decimals = len(repr(g["row_block_mean"]).split(".")[1])
        assert abs(rows.mean() - g["row_block_mean"]) <= 0.5 * 10.0 ** -decimals


def test_morton_monotone_and_owner_is_lowest():
    mesh = O.BoxMesh(8, 6, 4, 1, 1, 1, 2)
    blk = O.Blocking(mesh)
    rk = blk.patch_to_rank.reshape(blk.np_[2], blk.np_[1], blk.np_[0])
    assert np.all(np.diff(rk, axis=2) > 0) and np.all(np.diff(rk, axis=1) > 0) and np.all(np.diff(rk, axis=0) > 0)
    # brute force: owner = lowest-rank patch whose closure contains the node
    q = 2 * mesh.p
    keys = np.arange(mesh.n_nodes)
    I, J, K = mesh.ijk(keys)
    own = blk.owner_rank(keys)
    for n in range(0, mesh.n_nodes, 7):
        best = None
        for pz in range(blk.np_[2]):
            for py in range(blk.np_[1]):
                for px in range(blk.np_[0]):
                    if q * px <= I[n] <= q * (px + 1) and q * py <= J[n] <= q * (py + 1) and q * pz <= K[n] <= q * (pz + 1):
                        r = blk.patch_to_rank[blk.patch_id(px, py, pz)]
                        best = r if best is None else min(best, r)
        assert own[n] == best


def test_column_blocks_alg2():
    cfg = inputs.get_config("p2")
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    c = inputs.orbital_centres(cfg)
    perm, ptr = O.column_blocks(blk, c, cfg.n_col_blocks)
    sizes = np.diff(ptr)
    assert len(sizes) == 38 and sizes.sum() == 320
    assert (sizes == 9).sum() == 16 and (sizes == 8).sum() == 22
    assert sorted(perm.tolist()) == list(range(320))
    assert abs(sizes.mean() - 8.42105) < 1e-5        # Table 1 column block mean
    # sorted by the rank of the containing cell
    cell = np.clip(np.floor(c / mesh.h), 0, [mesh.nx - 1, mesh.ny - 1, mesh.nz - 1]).astype(int)
    rank = blk.cell_rank(mesh.cell_index(cell[:, 0], cell[:, 1], cell[:, 2]))
    assert np.all(np.diff(rank[perm]) >= 0)
    t = inputs.get_config("tiny")
    tm = O.BoxMesh.from_config(t)
    _, tptr = O.column_blocks(O.Blocking(tm), inputs.orbital_centres(t), 2)
    assert tptr.tolist() == [0, 8, 16]


# ---------------------------------------------------------------------------
# Pattern: brute force, closure, fill
# ---------------------------------------------------------------------------
def _pattern_brute(mesh, blk, mv, perm, ptr):
    """Pure-Python loops straight from the definition."""
    p = mesh.p
    pat = np.zeros((blk.n_patches, len(ptr) - 1), dtype=bool)
    support = [set() for _ in range(len(ptr) - 1)]
    for cb in range(len(ptr) - 1):
        for j in range(ptr[cb], ptr[cb + 1]):
            support[cb].update(int(k) for k in mv.keys[perm[j]])
    for cz in range(mesh.nz):
        for cy in range(mesh.ny):
            for cx in range(mesh.nx):
                nodes = [int(mesh.key(p * cx + a, p * cy + b, p * cz + c))
                         for c in range(p + 1) for b in range(p + 1) for a in range(p + 1)]
                for cb in range(len(ptr) - 1):
                    if any(n in support[cb] for n in nodes):
                        for n in nodes:
                            pat[int(blk.owner_rank(np.array([n]))[0]), cb] = True
    return pat


@pytest.mark.parametrize("name", ["tiny", "small_p2", "small_p1", "small_p4"])
def test_pattern_brute_force(name):
    cfg = inputs.get_config(name)
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    perm, ptr = O.column_blocks(blk, inputs.orbital_centres(cfg), cfg.n_col_blocks)
    mv = O.build_orbitals(mesh, cfg)
    pat = O.block_pattern(blk, mv, perm, ptr)
    np.testing.assert_array_equal(pat, _pattern_brute(mesh, blk, mv, perm, ptr))
    # support is inside the ball and off the Dirichlet boundary
    for a in range(cfg.n_orb):
        xyz = mesh.node_coords(mv.keys[a])
        c = inputs.orbital_centres(cfg)[a]
        assert np.all(((xyz - c) ** 2).sum(1) <= cfg.radius ** 2)
        assert not mesh.boundary(mv.keys[a]).any()


@pytest.mark.parametrize("name", ["small_p2", "small_p3"])
def test_closed_pattern_masked_equals_full(name):
    cfg = inputs.get_config(name)
    r = O.run(cfg)
    H = O.assemble(r.mesh, O.potential_fn(cfg))
    HP = (H @ r.P).toarray()
    Y = r.Y.toarray()
    assert np.abs(HP - Y).max() == 0.0
    assert r.pattern.mean() < 0.9      # the mask is not trivially full here


def test_mask_semantics_on_open_pattern():
    """With an undilated pattern (row blocks of the support only), Y keeps
    exactly the masked entries of H P and P^T Y is no longer symmetric."""
    cfg = inputs.get_config("small_p2")
    r = O.run(cfg)
    H = O.assemble(r.mesh, O.potential_fn(cfg))
    nb = len(r.ptr) - 1
    pat = np.zeros_like(r.pattern)
    Pc = r.P.tocsc()
    for c in range(nb):
        for j in range(r.ptr[c], r.ptr[c + 1]):
            a = r.perm[j]
            support = Pc.indices[Pc.indptr[a]:Pc.indptr[a + 1]]
            pat[r.blk.owner_rank(support), c] = True
    Y = O.apply_masked(H, r.P, r.blk, pat, r.cb_of_orb).toarray()
    HP = (H @ r.P).toarray()
    keys = np.arange(r.mesh.n_nodes)
    m = pat[r.blk.owner_rank(keys)][:, r.cb_of_orb]
    np.testing.assert_array_equal(Y, np.where(m, HP, 0.0))
    assert np.abs(HP - Y).max() > 0
    G = O.gram(r.P, sp.csc_matrix(Y))
    assert np.abs(G - G.T).max() > 1e-6 * np.abs(G).max()


@pytest.mark.slow
@pytest.mark.parametrize("name,target", [("p2", 0.20), ("p4", 0.15)])
def test_paper_scale_fill(name, target):
    cfg = inputs.get_config(name)
    mesh = O.BoxMesh.from_config(cfg)
    blk = O.Blocking(mesh)
    perm, ptr = O.column_blocks(blk, inputs.orbital_centres(cfg), cfg.n_col_blocks)
    pat = O.block_pattern(blk, O.build_orbitals(mesh, cfg), perm, ptr)
    assert abs(pat.mean() - target) <= 0.01


# ---------------------------------------------------------------------------
# Gram products and the full tiny pipeline
# ---------------------------------------------------------------------------
def test_tiny_pipeline_dense_cross_check():
    cfg = inputs.get_config("tiny")
    r = O.run(cfg)
    mesh = r.mesh
    assert mesh.n_nodes == 729 and (~mesh.boundary()).sum() == 343
    assert r.blk.n_patches == 8 and r.ptr.tolist() == [0, 8, 16]
    Hd = O.assemble(mesh, O.potential_fn(cfg)).toarray()
    Pd = r.P.toarray()
    Yd = r.Y.toarray()
    np.testing.assert_allclose(Yd, Hd @ Pd, rtol=0, atol=1e-14 * np.abs(Yd).max())
    np.testing.assert_allclose(r.G_PP, Pd.T @ Pd, rtol=0, atol=1e-14 * np.abs(r.G_PP).max())
    np.testing.assert_allclose(r.G_PY, Pd.T @ Hd @ Pd, rtol=0, atol=1e-13 * np.abs(r.G_PY).max())
    assert np.abs(r.G_PP - r.G_PP.T).max() == 0.0
    assert np.abs(r.G_PY - r.G_PY.T).max() <= 1e-14 * np.abs(r.G_PY).max()
    np.linalg.cholesky(r.G_PP)      # SPD
    # Dirichlet rows are zero
    assert np.abs(Yd[mesh.boundary()]).max() == 0.0


def test_rayleigh_quotient_of_sine_column():
    """u^T H u / u^T M u = 1/2 (mu_a + mu_b + mu_c) for a sine mode column."""
    n, h, p = 4, 0.25, 2
    K1, M1 = _assemble1d(p, n, h, _q2)
    mu, V = sla.eigh(K1, M1)
    mesh = O.BoxMesh(n, n, n, h, h, h, p, dirichlet=1)
    H = O.assemble(mesh, None)
    Mg = O.assemble(mesh, None, mass=True)
    L = p * n + 1
    u3 = np.zeros((L, L, L))
    u3[1:-1, 1:-1, 1:-1] = np.einsum("k,j,i->kji", V[:, 2], V[:, 0], V[:, 1])
    Pu = sp.csc_matrix(u3.ravel()[:, None])
    ratio = O.gram(Pu, H @ Pu)[0, 0] / O.gram(Pu, Mg @ Pu)[0, 0]
    assert abs(ratio - 0.5 * (mu[0] + mu[1] + mu[2])) < 1e-12 * ratio


def test_apply_rows_matches_assembly():
    cfg = inputs.get_config("small_p2")
    r = O.run(cfg)
    rng = np.random.default_rng(3)
    keys = rng.choice(r.mesh.n_nodes, 40, replace=False)
    rows = O.apply_rows(r.mesh, O.potential_fn(cfg), r.P, keys)
    H = O.assemble(r.mesh, O.potential_fn(cfg))
    full = (H @ r.P).toarray()[keys]
    np.testing.assert_allclose(rows, full, rtol=0, atol=1e-13 * max(1.0, np.abs(full).max()))


# ---------------------------------------------------------------------------
# Post-multiplication (Alg. 7) and the orbital-minimisation gradient (Sec. 2)
# ---------------------------------------------------------------------------
def _tiny_state(name="tiny"):
    cfg = inputs.get_config(name)
    r = O.run(cfg, with_apply=False)
    H = O.assemble(r.mesh, O.potential_fn(cfg))
    M = O.assemble(r.mesh, None, mass=True)
    return cfg, r, H, M


def test_mmult_identity_and_brute_force():
    """C = mask(A X): X = I gives A back (A lies in the pattern); a random X
    matches an entry-by-entry sum over the stored entries of A."""
    cfg, r, H, M = _tiny_state()
    P = r.P.tocsc()
    Mn = P.shape[1]
    C = O.mmult_masked(P, np.eye(Mn), r.blk, r.pattern, r.cb_of_orb)
    assert abs(C - P).max() == 0.0
    rng = np.random.default_rng(3)
    X = rng.normal(size=(Mn, Mn))
    C = O.mmult_masked(P, X, r.blk, r.pattern, r.cb_of_orb).toarray()
    Pd = P.toarray()
    own = r.blk.owner_rank(np.arange(P.shape[0]))
    for i in rng.choice(P.shape[0], 40, replace=False):
        for b in range(Mn):
            ref = sum(Pd[i, a] * X[a, b] for a in range(Mn) if Pd[i, a] != 0.0)
            ref = ref if r.pattern[own[i], r.cb_of_orb[b]] else 0.0
            assert abs(C[i, b] - ref) <= 1e-12 * (1 + abs(ref))


def test_om_gradient_is_the_derivative_of_the_energy():
    """tr(D^T G) equals the central finite difference of E(Phi + eps D) for a
    random direction D inside the pattern (Sec. 2: the directional
    derivative); the truncation of G to the pattern does not change it."""
    cfg, r, H, M = _tiny_state()
    P = r.P.tocsc()
    G, Hb, Mb = O.om_gradient(P, (H @ P).tocsc(), (M @ P).tocsc(), r.blk, r.pattern, r.cb_of_orb)
    rng = np.random.default_rng(5)
    Dd = sp.csc_matrix((rng.normal(size=P.nnz), P.indices, P.indptr), shape=P.shape)   # same support as P
    eps = 1e-5
    fd = (O.om_energy(P + eps * Dd, H, M) - O.om_energy(P - eps * Dd, H, M)) / (2 * eps)
    g = O.trace_dot(Dd, G)
    assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (fd, g)
    # the energy uses the same projections
    assert O.om_energy(P, H, M) == pytest.approx(float(np.trace((2 * np.eye(Hb.shape[0]) - Mb) @ Hb)), rel=1e-14)
