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


def test_admission_order_shortest_first_with_age_bound():
    """Queued requests go shortest predicted first; one that has waited more
    than age_factor times its prediction goes ahead of all unaged ones."""
    from types import SimpleNamespace as R
    from paper_1907_01005_gb300.serving import admission_order
    service = {0: 10e-3, 1: 0.1e-3, 2: 1e-3}           # large, small, medium payloads
    q = [R(pid=0, arrival=0.0), R(pid=2, arrival=0.001), R(pid=1, arrival=0.002)]
    order = admission_order(q, service, now=0.003, age_factor=4.0, min_age_s=2e-3)
    assert [r.pid for r, _ in order] == [1, 2, 0] and not any(a for _, a in order)
    # much later the large request is aged (waited > 4 x 10 ms) and leads
    order = admission_order(q, service, now=0.045, age_factor=4.0, min_age_s=2e-3)
    assert order[0][0].pid == 0 and order[0][1]


def test_last_slot_is_kept_for_small_or_aged_requests():
    from paper_1907_01005_gb300.serving import may_take_slot
    assert may_take_slot(2, 4, False, 10e-3, 1e-3)        # more than one slot free: anyone
    assert not may_take_slot(1, 4, False, 10e-3, 1e-3)    # last slot: not for a large request
    assert may_take_slot(1, 4, False, 0.5e-3, 1e-3)       # ... but for a small one
    assert may_take_slot(1, 4, True, 10e-3, 1e-3)         # ... or an aged one
    assert may_take_slot(1, 1, False, 10e-3, 1e-3)        # a single-slot server keeps nothing back
