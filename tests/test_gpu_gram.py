"""The Gram products (Alg. 8) through the C ABI for inputs other than the
step's own Y = H P.

fe_gram_PtY must form every block of P^T Y whatever Y holds, also when P's
pattern is declared closed (where the step itself may use the symmetric
form).  Y here is an arbitrary multivector on P's pattern: seeded N(0, 1)
values, so P^T Y is not symmetric.  The reference is the oracle's FP64
product C = A^T B of the same stored entries (inputs rounded to FP32 for the
FP32 path, as in the other parity tests)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fe_oracle as O
from synth import inputs

pytestmark = pytest.mark.gpu

TOL_PY = {2: 1e-12, 1: 1e-6}


def _problem(name, dtype):
    from paper_1907_01005_gb300 import harness
    pb = harness.build_problem(inputs.get_config(name), dtype)
    harness.to_device(pb)
    return pb


def _random_on_pattern(pb, seed):
    """Seeded N(0,1) values on every stored entry of P's pattern (row padding zero)."""
    from paper_1907_01005_gb300 import harness
    rng = np.random.default_rng(seed)
    ref = harness.unpack_entries(pb, np.arange(int(pb.P.info.n_values), dtype=np.float64))
    slots = ref[2].astype(np.int64)                   # value slot of each stored entry
    vals = np.zeros(int(pb.P.info.n_values), pb.P_host.dtype)
    vals[slots] = rng.standard_normal(len(slots))
    return vals


def _as_sparse(pb, values):
    """Stored entries of a BCSR value array as an (n_nodes x M) FP64 matrix in
    the oracle's (lattice key, orbital id) index space."""
    from paper_1907_01005_gb300 import harness
    dofs, cols, vals = harness.unpack_entries(pb, values)
    n = (pb.mesh.info.lx * pb.mesh.info.ly * pb.mesh.info.lz)
    return sp.csc_matrix((vals.astype(np.float64), (pb.keys[dofs], pb.perm[cols])), shape=(n, pb.n_cols))


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["small_p2", "small_p4", "multi_p2"])
def test_pty_of_an_unrelated_y_on_a_closed_pattern(name, dtype):
    import torch
    from paper_1907_01005_gb300 import gram_PtY
    pb = _problem(name, dtype)
    assert pb.P.get_closed()
    yv = _random_on_pattern(pb, 1907)
    pb.dev["Y"].copy_(torch.from_numpy(yv))
    gram_PtY(pb.P, pb.Y, pb.dev["G_PY"])
    torch.cuda.synchronize()
    assert pb.mesh.check_device() == 0
    got = pb.dev["G_PY"].cpu().numpy()
    A = _as_sparse(pb, pb.P_host)
    B = _as_sparse(pb, yv)
    ref = O.gram(A, B)[np.ix_(pb.perm, pb.perm)]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= TOL_PY[dtype], err
    # the product really is not symmetric, so a mirrored half would fail above
    assert np.abs(ref - ref.T).max() > 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("dtype", [2, 1], ids=["f64", "f32"])
def test_symmetric_form_matches_full_form_for_y_equal_hp(dtype):
    import torch
    from paper_1907_01005_gb300 import apply_H, gram_PtY, gram_PtY_sym
    pb = _problem("multi_p2", dtype)
    d = pb.dev
    apply_H(pb.mesh, pb.P, pb.Y)
    gram_PtY(pb.P, pb.Y, d["G_PY"])
    G_sym = torch.zeros_like(d["G_PY"])
    gram_PtY_sym(pb.P, pb.Y, G_sym)
    torch.cuda.synchronize()
    full, sym = d["G_PY"].cpu().numpy(), G_sym.cpu().numpy()
    assert np.abs(full - sym).max() <= TOL_PY[dtype] * np.abs(full).max()
    assert np.abs(sym - sym.T).max() <= 1e-14 * np.abs(sym).max()


def test_symmetric_form_needs_a_closed_pattern():
    import ctypes as C
    from paper_1907_01005_gb300 import _capi, harness
    pb = harness.build_problem(inputs.get_config("small_p2"), 1, pattern="support")
    harness.to_device(pb)
    assert not pb.P.get_closed()
    rc = _capi.fe_gram_PtY_sym(pb.P.h, pb.Y.h, C.c_void_p(pb.dev["G_PY"].data_ptr()), C.c_void_p(0))
    assert rc == _capi.FE_ESTATE
    assert "closed" in _capi.last_error()
