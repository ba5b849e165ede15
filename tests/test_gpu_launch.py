"""Launch shapes of the same step: persistent vs grid launch of the apply,
a cap on the SMs of the persistent launches, the CUDA graph of the whole
step, and the autotuner's choice all give the oracle's result within the
parity tolerances.  Y is written without atomics in a fixed order, so it is
the same bit for bit under every launch shape; the Gram products differ only
in the order of their FP64 atomic additions."""
import json

import numpy as np
import pytest

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL = {2: dict(Y=1e-12, PY=1e-12, PP=1e-12), 1: dict(Y=1e-5, PY=1e-6, PP=1e-10)}


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _setup(name, dtype):
    from paper_1907_01005_gb300 import harness
    pb = harness.build_problem(inputs.get_config(name), dtype)
    harness.to_device(pb)
    return pb


def _outputs(pb):
    d = pb.dev
    return d["Y"].cpu().numpy(), d["G_PY"].cpu().numpy(), d["G_PP"].cpu().numpy()


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["small_p2", "small_p1", "small_p4"])
def test_persistent_and_graph_match_oracle(name, dtype):
    import torch
    from paper_1907_01005_gb300 import StepGraph, apply_H_gram
    pb = _setup(name, dtype)
    d = pb.dev
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    Y0, PY0, PP0 = _outputs(pb)
    r = O.run(pb.cfg, fp32_inputs=(dtype == 1))
    tol = TOL[dtype]
    ref_py = r.G_PY[np.ix_(pb.perm, pb.perm)]
    ref_pp = r.G_PP[np.ix_(pb.perm, pb.perm)]
    for knobs, sm_cap in [((1, 2, 0), 0), ((1, 8, 0), 0), ((0, 4, 1), 0), ((0, 4, 2), 0), ((1, 4, 0), 7)]:
        pb.P.set_launch(*knobs)
        pb.P.set_sm_limit(sm_cap)
        d["Y"].fill_(np.nan)
        apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
        torch.cuda.synchronize()
        assert pb.mesh.check_device() == 0
        Y, PY, PP = _outputs(pb)
        assert np.array_equal(Y, Y0), (knobs, sm_cap)
        assert _relerr(PY, ref_py) <= tol["PY"], knobs
        assert _relerr(PP, ref_pp) <= tol["PP"], knobs
    pb.P.set_sm_limit(0)
    # graph of the step, launched twice on fresh garbage
    pb.P.set_launch(1, 4, 0)
    g = StepGraph(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    for _ in range(2):
        d["Y"].fill_(np.nan)
        d["G_PY"].fill_(np.nan)
        d["G_PP"].fill_(np.nan)
        g.launch()
        torch.cuda.synchronize()
        Y, PY, PP = _outputs(pb)
        assert np.array_equal(Y, Y0)
        assert _relerr(PY, ref_py) <= tol["PY"]
        assert _relerr(PP, ref_pp) <= tol["PP"]
    del g


def test_autotune_and_cache(tmp_path):
    import torch
    from paper_1907_01005_gb300 import apply_H_gram, autotune
    pb = _setup("small_p2", 1)
    d = pb.dev
    cache = tmp_path / "tune.jsonl"
    ms = autotune(pb.mesh, pb.P, pb.Y, str(cache))
    assert ms > 0
    knobs = pb.P.get_launch()
    lines = [json.loads(s) for s in cache.read_text().splitlines()]
    assert len(lines) == 1 and (lines[0]["persistent"], lines[0]["ctas_per_sm"]) == knobs[:2]
    # a second problem of the same shape hits the cache
    pb2 = _setup("small_p2", 1)
    assert autotune(pb2.mesh, pb2.P, pb2.Y, str(cache)) == -1.0
    assert pb2.P.get_launch() == knobs
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    r = O.run(pb.cfg, fp32_inputs=True)
    assert _relerr(d["G_PY"].cpu().numpy(), r.G_PY[np.ix_(pb.perm, pb.perm)]) <= TOL[1]["PY"]


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
def test_host_buffer_entry_matches_device_step(dtype, pinned):
    """fe_apply_H_gram_host (copies in and out around the step, Y and G_PP
    leaving on their own streams) returns what the device step computes, and
    the oracle's result; two calls in a row with new P values follow them."""
    import torch
    from paper_1907_01005_gb300 import apply_H_gram, apply_H_gram_host
    cfg = inputs.get_config("small_p2")
    pb = _setup("small_p2", dtype)
    d = pb.dev
    M = pb.n_cols
    tdt = d["P"].dtype

    def host(t):
        return t.pin_memory() if pinned else t
    Ph = host(torch.from_numpy(pb.P_host.copy()))
    Yh = host(torch.zeros(d["Y"].shape, dtype=tdt))
    G1 = host(torch.zeros((M, M), dtype=torch.float64))
    G2 = host(torch.zeros((M, M), dtype=torch.float64))
    apply_H_gram_host(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], Ph, Yh, G1, G2)
    assert pb.mesh.check_device() == 0
    r = O.run(cfg, fp32_inputs=(dtype == 1))
    from paper_1907_01005_gb300 import harness
    dofs, cols, vals = harness.unpack_entries(pb, Yh.numpy())
    ref = np.asarray(r.Y.tocsr()[pb.keys[dofs], pb.perm[cols]]).ravel()
    assert _relerr(vals, ref) <= TOL[dtype]["Y"]
    assert _relerr(G1.numpy(), r.G_PY[np.ix_(pb.perm, pb.perm)]) <= TOL[dtype]["PY"]
    assert _relerr(G2.numpy(), r.G_PP[np.ix_(pb.perm, pb.perm)]) <= TOL[dtype]["PP"]
    # a second call with P scaled by 2: every output follows (Y by 2, the Grams
    # by 4), up to the order of the atomic additions into the Gram matrices
    Y1, Gpy1, Gpp1 = Yh.numpy().copy(), G1.numpy().copy(), G2.numpy().copy()
    Ph.mul_(2)
    apply_H_gram_host(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"], Ph, Yh, G1, G2)
    assert _relerr(Yh.numpy(), 2 * Y1) <= 1e-6
    assert _relerr(G1.numpy(), 4 * Gpy1) <= (1e-12 if dtype == 2 else TOL[1]["PY"])
    assert _relerr(G2.numpy(), 4 * Gpp1) <= 1e-12
    # the device step on the same (scaled) P agrees
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    assert _relerr(d["Y"].cpu().numpy(), Yh.numpy()) <= 1e-6
    assert _relerr(d["G_PP"].cpu().numpy(), G2.numpy()) <= 1e-14
