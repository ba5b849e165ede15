"""The allocation-free ALU probe (fe_probe_fma_static) against the probe
that allocates its sink (fe_probe_fma), through the C ABI.

Some callers cannot allocate device memory when they want the measurement,
for instance a server that has already promised its whole memory budget to
admitted requests; fe_probe_fma_static serves them from a fixed static
array.  Both calls run the same FMA-chain kernels.  Each CTA stores thread
0's chain sum in its slot, and each call reads slots back and compares them
with the sum the host computes (the static variant through the array's
symbol), returning FE_EDEVICE on a mismatch; so a call that succeeds has
written and read the sink it was meant to use.  On the same device both must
also report the same throughput within the run-to-run spread of a timed
kernel.  The calls alternate twice, so the shared static sink serves two
calls in a row.  Kept in a file of its own, collected last."""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 0.15   # run-to-run spread of a few-ms timed kernel, with margin


def _probe(name, dtype, iters):
    from paper_1907_01005_gb300 import _capi
    f = C.c_double()
    _capi.check(getattr(_capi, name)(dtype, iters, C.byref(f), C.c_void_p(0)))
    return f.value


@pytest.mark.parametrize("dtype,iters", [(1, 4000), (2, 200), (3, 4000)], ids=["f32", "f64", "f32x2"])
def test_static_sink_probe_matches_allocating_probe(dtype, iters):
    import torch
    torch.cuda.init()
    rates = []
    for _ in range(2):
        ref = _probe("fe_probe_fma", dtype, iters)
        got = _probe("fe_probe_fma_static", dtype, iters)
        assert ref > 0 and got > 0
        assert abs(got - ref) <= REL_TOL * ref, (got, ref)
        rates.append(got)
    assert abs(rates[1] - rates[0]) <= REL_TOL * rates[0], rates


def test_static_sink_probe_rejects_bad_arguments():
    from paper_1907_01005_gb300 import _capi
    f = C.c_double()
    assert _capi.fe_probe_fma_static(7, 10, C.byref(f), C.c_void_p(0)) == _capi.FE_EINVAL
    assert "fe_probe_fma_static" in _capi.last_error()
    assert _capi.fe_probe_fma_static(1, 0, C.byref(f), C.c_void_p(0)) == _capi.FE_EINVAL
