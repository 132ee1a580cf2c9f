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


@pytest.mark.parametrize("precision,nx,ny", [("fp64", 96, 160), ("fp32", 96, 160),
                                             ("fp64", 1000, 700), ("fp32", 1000, 700)])
def test_noalloc_sums_match_diagnostics_twice(precision, nx, ny):
    """96 x 160 fits one block's chunk of 16384 nodes; 1000 x 700 spreads over
    43 blocks whose last chunk is ragged (700000 = 42 x 16384 + 11872)."""
    import torch
    torch.cuda.set_device(0)
    prm, fields = inputs.rising_bubble(nx=nx, ny=ny, R=min(nx, ny) / 7.0, yc=ny / 3.0)
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
        # FP64 sums of n terms agree to 1e-12 of n + |sum|, for FP32 handles
        # too: their diagnostics form each term exactly as a float pair and
        # sum the row segments with TwoSum before the FP64 sums
        rel = 1e-12
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


def test_noalloc_at_the_maximum_size():
    """nx*ny = LBM_NOALLOC_MAX_NODES (8192^2, all 4096 partials in use), float
    fields with planted non-finite values, against FP64 sums of the same
    values taken by torch: counts and extrema exact, sums to 1e-12 of
    n + |sum| (both are FP64 sums of the same FP64-converted terms)."""
    import torch
    torch.cuda.set_device(0)
    nx = ny = 8192
    assert nx * ny == lbm.LBM_NOALLOC_MAX_NODES
    gen = torch.Generator(device="cuda").manual_seed(7)
    y = torch.arange(ny, device="cuda", dtype=torch.float64).view(ny, 1).expand(ny, nx)
    x = torch.arange(nx, device="cuda", dtype=torch.float64).view(1, nx).expand(ny, nx)
    r = torch.sqrt((x - 3000.0) ** 2 + (y - 5000.0) ** 2)
    phi = torch.tanh((r - 1500.0) / 2.0).to(torch.float32)          # a bubble: phi < 0 inside
    phi += 1e-3 * torch.rand((ny, nx), generator=gen, device="cuda", dtype=torch.float32)
    p = torch.randn((ny, nx), generator=gen, device="cuda", dtype=torch.float32)
    ux = torch.randn((ny, nx), generator=gen, device="cuda", dtype=torch.float32)
    uy = 1e-3 * torch.randn((ny, nx), generator=gen, device="cuda", dtype=torch.float32)
    p[17, 4001] = float("nan")
    ux[8000, 3] = float("inf")
    out = torch.full((lbm.LBM_NDIAG,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):                       # two calls in a row, the second on changed fields
        if call == 1:
            phi[ny - 1, nx - 1] = 0.75
            uy.mul_(2.0)
        lbm.field_sums_noalloc(phi, p, ux, uy, out)
        got = out.cpu().numpy()
        ph, v = phi.double(), uy.double()
        w = (1.0 - ph) * 0.5
        neg = ph < 0
        ref = [ph.sum(), (ph > 0).sum(), neg.sum(), y[neg].sum(), v[neg].sum(), w.sum(), (w * y).sum(),
               (w * v).sum(), ph.max(), ph.min(),
               sum((~torch.isfinite(t)).sum() for t in (phi, p, ux, uy))]
        ref = [float(t) for t in ref]
        n = nx * ny
        for k in (0, 3, 4, 5, 6, 7):
            assert abs(got[k] - ref[k]) <= 1e-12 * (n + abs(ref[k])), (call, k, got[k], ref[k])
        for k in (1, 2, 8, 9, 10):
            assert got[k] == ref[k], (call, k, got[k], ref[k])
        assert got[10] == 2
