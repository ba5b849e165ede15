"""Host-side checks of the serving workload mix (no GPU)."""


def test_serving_pool_holds_every_mesh_size():
    """The serving pool takes the mesh sizes in turn, so a pool of at least
    three workloads holds each of the serving meshes (p = 4 halves the cell
    count per direction, rounded up to even)."""
    from synth import inputs
    pool = inputs.serving_mix(6)
    p2 = {(c.nx, c.ny, c.nz) for c in pool if c.p == 2}
    sizes = set()
    for c in pool:
        sizes.add((c.nx, c.ny, c.nz) if c.p == 2 else (2 * c.nx, 2 * c.ny, 2 * c.nz))
    for m in inputs.SERVING_MESHES:
        assert any(abs(s[0] - m[0]) <= 2 and abs(s[1] - m[1]) <= 2 and abs(s[2] - m[2]) <= 2 for s in sizes), (m, sizes)
    assert p2


def test_serving_mix_is_seeded():
    from synth import inputs
    a = [(c.nx, c.ny, c.nz, c.p, c.n_orb) for c in inputs.serving_mix(8)]
    b = [(c.nx, c.ny, c.nz, c.p, c.n_orb) for c in inputs.serving_mix(8)]
    assert a == b
    assert all(32 <= m <= 640 for *_, m in a)
