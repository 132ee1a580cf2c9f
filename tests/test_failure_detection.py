"""Failure detection on host-injected faults (checks of the step's state; the
paper has no counterpart).

Faults are planted from the host as field values -- a NaN or an Inf in p or
u, phi outside [-1, 1] -- through lbm_set_fields; nothing here faults, traps
or hangs the GPU.  lbm_check (synchronising) and the periodic check that
lbm_step runs after lbm_set_check (never waiting on the stream) must report
LBM_ERR_NONFINITE / LBM_ERR_RANGE, and the diagnostics must count the
non-finite values.
"""
import numpy as np
import pytest

from paper_1812_02459_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

LBM_OK, LBM_ERR_NONFINITE, LBM_ERR_RANGE = 0, 4, 5


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mix_bf16"])
def test_check_reports_planted_nonfinite_and_range(precision):
    prm, (phi, p, ux, uy) = inputs.static_drop(n=32, R=8.0)
    g = lbm.Sim(prm, phi, p, ux, uy, precision=precision)
    assert g.check(0.05) == LBM_OK
    assert g.diagnostics()[10] == 0

    p_bad = p.copy()
    p_bad[5, 7] = np.nan
    g.set_fields(phi, p_bad, ux, uy)
    assert g.diagnostics()[10] == 1
    assert g.check(0.05) == LBM_ERR_NONFINITE

    ux_bad, uy_bad = ux.copy(), uy.copy()
    ux_bad[3, 3] = np.inf
    uy_bad[9, 30] = -np.inf
    g.set_fields(phi, p, ux_bad, uy_bad)
    assert g.diagnostics()[10] == 2
    assert g.check(0.05) == LBM_ERR_NONFINITE

    for val, node in ((1.2, (16, 16)), (-1.3, (0, 0))):
        phi_bad = phi.copy()
        phi_bad[node] = val
        g.set_fields(phi_bad, p, ux, uy)
        d = g.diagnostics()
        assert (d[8] if val > 0 else d[9]) == pytest.approx(val, rel=1e-6)
        assert d[10] == 0
        assert g.check(0.05) == LBM_ERR_RANGE
        assert g.check(0.5) == LBM_OK

    # a NaN planted in phi spreads through the stencils of a step
    phi_bad = phi.copy()
    phi_bad[16, 16] = np.nan
    g.set_fields(phi_bad, p, ux, uy)
    g.step(2)
    assert g.diagnostics()[10] >= 4
    assert g.check(0.05) == LBM_ERR_NONFINITE

    # re-initialising from clean fields clears it
    g.set_fields(phi, p, ux, uy)
    g.step(2)
    assert g.check(0.05) == LBM_OK
    g.close()


def test_periodic_check_inside_step():
    import torch
    torch.cuda.set_device(0)
    prm, (phi, p, ux, uy) = inputs.static_drop(n=32, R=8.0)
    g = lbm.Sim(prm, phi, p, ux, uy, precision="fp32")
    g.set_check(2, 0.05)
    g.step(5)                       # clean: checks after steps 2 and 4
    torch.cuda.synchronize()
    g.step(1)                       # reads the finished check: still fine
    torch.cuda.synchronize()

    p_bad = p.copy()
    p_bad[4, 4] = np.nan
    g.set_fields(phi, p_bad, ux, uy)
    g.step(2)                       # enqueues a check of the planted NaN
    torch.cuda.synchronize()
    with pytest.raises(lbm.LbmError) as e:
        g.step(1)
    assert e.value.status == LBM_ERR_NONFINITE
    with pytest.raises(lbm.LbmError):   # stays until the fields are reset
        g.step(1)

    phi_bad = phi.copy()
    phi_bad[10, 10] = 1.5
    g.set_fields(phi_bad, p, ux, uy)
    g.set_check(1, 0.05)
    g.step(1)
    torch.cuda.synchronize()
    with pytest.raises(lbm.LbmError) as e:
        g.step(1)
    assert e.value.status == LBM_ERR_RANGE

    g.set_fields(phi, p, ux, uy)
    g.step(3)
    torch.cuda.synchronize()
    g.step(1)
    assert g.check(0.05) == LBM_OK
    g.close()
