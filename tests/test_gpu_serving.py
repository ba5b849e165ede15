"""Serving: continuous batching over the C ABI.  Every request's result is
the same whether it runs alone or in a mix of concurrent requests (Y bit for
bit; the Gram products within the FP32-mixed tolerances, their FP64 atomics
adding in another order), admission respects the memory budget (idle
payloads are evicted and restored), and every payload's result is checked
against the oracle."""
import numpy as np
import pytest

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL = dict(Y=1e-5, PY=1e-6, PP=1e-10)
NAMES = ["small_p2", "small_p4", "wide_p2", "narrow_p2", "small_p1", "tiny"]


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _problems():
    from paper_1907_01005_gb300 import harness
    return [harness.build_problem(inputs.get_config(n), 1) for n in NAMES]


def test_same_result_alone_and_in_the_mix():
    from paper_1907_01005_gb300.serving import Server
    srv = Server(slots=4)
    pids = [srv.register(pb) for pb in _problems()]
    alone = {}
    for pid in pids:                       # one at a time
        r = srv.submit(pid, want_y=True)
        srv.drain()
        alone[pid] = r.result
    # the mix: every payload twice, all submitted at once (a busy payload's
    # second request waits while others overtake it)
    reqs = [srv.submit(pid, want_y=True) for pid in pids + pids[::-1]]
    srv.drain()
    assert all(r.done > 0 for r in reqs)
    overlap = sum(1 for a in reqs for b in reqs if a is not b and a.admitted < b.done and b.admitted < a.done)
    assert overlap > 0, "no two requests were on the GPU at the same time"
    for r in reqs:
        ref = alone[r.pid]
        assert np.array_equal(r.result["Y"], ref["Y"])
        assert _relerr(r.result["G_PY"], ref["G_PY"]) <= TOL["PY"]
        assert _relerr(r.result["G_PP"], ref["G_PP"]) <= TOL["PP"]
    # every payload's result against the oracle
    from paper_1907_01005_gb300 import harness
    for pid in pids:
        pb = srv.payloads[pid].problem
        o = O.run(pb.cfg, fp32_inputs=True)
        assert _relerr(alone[pid]["G_PY"], o.G_PY[np.ix_(pb.perm, pb.perm)]) <= TOL["PY"], pb.cfg.name
        assert _relerr(alone[pid]["G_PP"], o.G_PP[np.ix_(pb.perm, pb.perm)]) <= TOL["PP"], pb.cfg.name
        dofs, cols, vals = harness.unpack_entries(pb, alone[pid]["Y"])
        ref_y = np.asarray(o.Y.tocsr()[pb.keys[dofs], pb.perm[cols]]).ravel()
        assert _relerr(vals, ref_y) <= TOL["Y"], pb.cfg.name


def test_admission_by_memory_budget():
    from paper_1907_01005_gb300.serving import Server
    probs = _problems()
    srv = Server(slots=3)
    pids = [srv.register(pb) for pb in probs]
    needs = [srv.payloads[p].footprint() + srv._mesh_bytes_needed(srv.payloads[p]) + 65536 for p in pids]
    srv.budget = max(max(needs), sum(needs) // 2)       # about half the payloads fit at once
    trace = [(0.0005 * i, pids[i % len(pids)]) for i in range(3 * len(pids))]
    reqs = srv.run_trace(trace)
    assert srv.peak_used <= srv.budget
    assert srv.evictions > 0
    # results of repeated requests of one payload agree (evicted and restored in between)
    by_pid = {}
    for r in reqs:
        if r.pid in by_pid:
            assert _relerr(r.result["G_PP"], by_pid[r.pid]["G_PP"]) <= TOL["PP"]
        else:
            by_pid[r.pid] = r.result
