"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (normwise: max|got - ref| / max|ref| per output):
  FP64 path:  Y, P^T Y, P^T P  1e-12
  FP32 path:  Y 1e-5, P^T Y 1e-6, P^T P 1e-10
The FP32 path is judged on FP32-rounded inputs (the oracle gets the same
rounded P and V widened to FP64), so input rounding is not charged to it.
"""
import numpy as np
import pytest

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL = {2: dict(Y=1e-12, PY=1e-12, PP=1e-12), 1: dict(Y=1e-5, PY=1e-6, PP=1e-10)}
SMALL = ["tiny", "tiny_p4", "small_p1", "small_p2", "small_p3", "small_p4", "wide_p2",
         "narrow_p2", "narrow_p4", "free_p2", "free_p4", "multi_p2", "multi_p4", "multi_w16_p2"]


def _run_gpu(cfg, dtype):
    import torch
    from paper_1907_01005_gb300 import apply_H_gram, harness
    pb = harness.build_problem(cfg, dtype)
    harness.to_device(pb)
    d = pb.dev
    apply_H_gram(pb.mesh, pb.P, pb.Y, d["G_PY"], d["G_PP"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    return pb, d["Y"].cpu().numpy(), d["G_PY"].cpu().numpy(), d["G_PP"].cpu().numpy()


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


def _check_y_full(pb, Y_gpu, r, tol):
    from paper_1907_01005_gb300 import harness
    dofs, cols, vals = harness.unpack_entries(pb, Y_gpu)
    keys = pb.keys[dofs]
    orb = pb.perm[cols]
    ref = np.asarray(r.Y.tocsr()[keys, orb]).ravel()
    assert _relerr(vals, ref) <= tol, _relerr(vals, ref)
    # every nonzero of the oracle's Y is a stored entry of the GPU's Y
    stored = set(zip(keys.tolist(), orb.tolist()))
    Yc = r.Y.tocoo()
    nz = Yc.data != 0
    assert all((k, a) in stored for k, a in zip(Yc.row[nz].tolist(), Yc.col[nz].tolist()))
    # Dirichlet rows are exactly zero
    bnd = r.mesh.boundary(keys)
    assert np.all(vals[bnd] == 0)


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", SMALL)
def test_parity_small(name, dtype):
    cfg = inputs.get_config(name)
    pb, Y, G_PY, G_PP = _run_gpu(cfg, dtype)
    r = O.run(cfg, fp32_inputs=(dtype == 1))
    tol = TOL[dtype]
    _check_y_full(pb, Y, r, tol["Y"])
    ref_py = r.G_PY[np.ix_(pb.perm, pb.perm)]
    ref_pp = r.G_PP[np.ix_(pb.perm, pb.perm)]
    assert _relerr(G_PY, ref_py) <= tol["PY"], _relerr(G_PY, ref_py)
    assert _relerr(G_PP, ref_pp) <= tol["PP"], _relerr(G_PP, ref_pp)
    # P^T P is symmetric up to the order of the FP64 atomic additions
    assert _relerr(G_PP, G_PP.T) <= 1e-14


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["small_p2", "small_p4", "multi_p2", "free_p2"])
def test_ordered_write_is_deterministic_and_overwrites_y(name, dtype):
    """The write into Y (no zero-fill, no atomics, fixed order of additions):
    repeated calls, the grid and the persistent launch, and a Y that starts
    out as NaN all give the same Y bit for bit, row padding zero included."""
    import torch
    from paper_1907_01005_gb300 import apply_H, apply_M
    cfg = inputs.get_config(name)
    pb, Y1, _, _ = _run_gpu(cfg, dtype)
    y = pb.dev["Y"]
    results = []
    for persistent, ctas in ((0, 4), (1, 2), (1, 8)):
        pb.P.set_launch(persistent, ctas, 0)
        y.fill_(float("nan"))
        apply_H(pb.mesh, pb.P, pb.Y)
        torch.cuda.synchronize()
        assert pb.mesh.check_device() == 0
        results.append(y.cpu().numpy())
    for r in results:
        assert np.array_equal(r, Y1)
    # the mass operator writes the same way
    y.fill_(float("nan"))
    apply_M(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    M1 = y.cpu().numpy()
    apply_M(pb.mesh, pb.P, pb.Y)
    torch.cuda.synchronize()
    assert not np.isnan(M1).any() and np.array_equal(M1, y.cpu().numpy())
