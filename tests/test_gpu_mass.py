"""Mass operator (Phi_M = M P, overlap matrix P^T M P; Sec. 2 / Eq. inner1)
through the C ABI against the FP64 oracle's assembled mass matrix, on the
same configs and tolerances as the Hamiltonian."""
import numpy as np
import pytest

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL = {2: dict(Y=1e-12, PY=1e-12), 1: dict(Y=1e-5, PY=1e-6)}
NAMES = ["tiny", "tiny_p4", "small_p1", "small_p2", "small_p3", "small_p4", "narrow_p4", "free_p2", "free_p4"]


def _relerr(got, ref):
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", NAMES)
def test_mass_parity(name, dtype):
    import torch
    from paper_1907_01005_gb300 import apply_M, gram_PtY, harness
    cfg = inputs.get_config(name)
    pb = harness.build_problem(cfg, dtype)
    harness.to_device(pb)
    d = pb.dev
    apply_M(pb.mesh, pb.P, pb.Y)
    gram_PtY(pb.P, pb.Y, d["G_PY"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    Y = d["Y"].cpu().numpy()
    G = d["G_PY"].cpu().numpy()
    mesh = O.BoxMesh.from_config(cfg)
    r = O.run(cfg, fp32_inputs=(dtype == 1), H=O.assemble(mesh, None, mass=True))
    dofs, cols, vals = harness.unpack_entries(pb, Y)
    ref = np.asarray(r.Y.tocsr()[pb.keys[dofs], pb.perm[cols]]).ravel()
    assert _relerr(vals, ref) <= TOL[dtype]["Y"], _relerr(vals, ref)
    ref_g = r.G_PY[np.ix_(pb.perm, pb.perm)]
    assert _relerr(G, ref_g) <= TOL[dtype]["PY"], _relerr(G, ref_g)
    # the overlap matrix is symmetric positive definite on the closed pattern
    Gs = 0.5 * (G + G.T)
    assert _relerr(G, G.T) <= 10 * TOL[dtype]["PY"]
    np.linalg.cholesky(Gs)
