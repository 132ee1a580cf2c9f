"""The Cahn-Hilliard part alone under a prescribed velocity (lbm_step_ch),
the mode of the paper's interface-capturing tests (Sec. IV.A single vortex,
Sec. IV.B drop translation), against the oracle's orc_step_ch."""
import math

import numpy as np
import pytest

import oracle
from paper_1812_02459_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def vortex(nx, ny, U0):
    """The single-vortex field of Sec. IV.A Eq. (velocity), in units of the box."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    X, Y = (x + 0.5) / nx, (y + 0.5) / ny
    ux = U0 * np.sin(math.pi * X) ** 2 * np.sin(2 * math.pi * Y)
    uy = -U0 * np.sin(math.pi * Y) ** 2 * np.sin(2 * math.pi * X)
    return ux, uy


def rel_err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx,ny,py", [(48, 48, 1), (48, 48, 0)])
def test_ch_only_matches_oracle(precision, nx, ny, py):
    """200 steps in a fixed vortex field, then 20 steps with the field scaled
    by cos(pi t / T) per step (the GPU takes the factors in one call, the
    oracle one step at a time).  The box is square, so the field is
    divergence-free: a compressive field drives phi past -1 in the bulk,
    where the profile flux lambda J_phi turns anti-diffusive and amplifies
    any rounding difference between two correct implementations."""
    prm = inputs.base_params(sigma=1e-2, M=0.1, periodic_y=py)
    phi0 = inputs.drop(nx, ny, 8.0, nx / 2 + 0.3, 0.62 * ny, prm["W"])
    z = np.zeros_like(phi0)
    ux, uy = vortex(nx, ny, 0.02)
    o = oracle.Sim(prm, phi0, z, z, z)
    g = lbm.Sim(prm, phi0, z, z, z, precision=precision)
    o.step_ch(ux, uy, 200)
    g.step_ch(ux, uy, 200)
    assert rel_err(g.fields()[0], o.fields()[0]) <= TOL[precision]
    T = 40.0
    tf = np.cos(math.pi * (200 + np.arange(20)) / T)
    for c in tf:
        o.step_ch(c * ux, c * uy, 1)
    g.step_ch(ux, uy, 20, tfac=tf)
    og, gg = o.fields(), g.fields()
    assert rel_err(gg[0], og[0]) <= TOL[precision]
    tol_u = 1e-14 if precision == "fp64" else 1e-6      # the last step's velocity, stored in T
    assert np.abs(gg[2] - og[2]).max() <= tol_u * np.abs(og[2]).max()
    # the NS part is untouched: p stays at its initial zero
    assert np.abs(gg[1]).max() == 0.0
    # Sec. IV.A: sum phi is conserved by both parts of the split
    d = g.diagnostics()
    assert abs(d[0] - phi0.sum()) <= (1e-12 if precision == "fp64" else 1e-5) * np.abs(phi0).sum()
