"""lbm_field_sums_noalloc: the non-allocating variant of the field sums.

It serves callers that cannot call cudaMalloc (a framework that owns all
device memory through its own pool, a loop that cannot absorb the
synchronisation of cudaMalloc/cudaFree, a monitor that must still report
after memory ran out).  Its result must match lbm_diagnostics, the entry
point that uses handle-owned scratch, within the FP64 tolerance the other
tests use, on two calls in a row.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1812_02459_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_sums_match_diagnostics_twice(precision):
    import torch
    torch.cuda.set_device(0)
    prm, fields = inputs.rising_bubble(nx=96, ny=160, R=14.0, yc=50.0)
    sim = lbm.Sim(prm, *fields, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    shp = (sim.ny, sim.nx)
    bufs = [torch.empty(shp, dtype=dt, device="cuda") for _ in range(4)]
    out = torch.full((lbm.LBM_NDIAG,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (5, 7):                       # two calls in a row, different fields
        sim.step(steps)
        ref = sim.diagnostics()
        sim.fields_device(*bufs)
        lbm.field_sums_noalloc(*bufs, out)
        got = out.cpu().numpy()
        n = shp[0] * shp[1]
        # FP64 sums of n terms agree to 1e-12 of n + |sum|; an FP32 handle's
        # diagnostics add row segments of at most 8 terms in FP32 first,
        # which is off by at most 7 roundings (2^-24) of each |term| <= 1
        rel = 1e-12 if precision == "fp64" else 7 * 2.0 ** -24
        for k in (0, 3, 4, 5, 6, 7):
            assert abs(got[k] - ref[k]) <= rel * (n + abs(ref[k])), (k, got[k], ref[k])
        for k in (1, 2, 8, 9, 10):             # counts and extrema are exact
            assert got[k] == ref[k], (k, got[k], ref[k])
    sim.close()


def test_noalloc_rejects_oversize_and_bad_args():
    import torch
    torch.cuda.set_device(0)
    t = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(lbm.LBM_NDIAG, dtype=torch.float64, device="cuda")
    L = lbm.load()
    import ctypes as C
    ptr = C.c_void_p(t.data_ptr())
    st = L.lbm_field_sums_noalloc(ptr, ptr, ptr, ptr, 8193, 8192, 0, C.c_void_p(out.data_ptr()), None)
    assert st == 1 and b"LBM_NOALLOC_MAX_NODES" in L.lbm_noalloc_last_error()
    st = L.lbm_field_sums_noalloc(ptr, ptr, ptr, ptr, 4, 4, 2, C.c_void_p(out.data_ptr()), None)
    assert st == 1
