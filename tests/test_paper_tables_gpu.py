"""The paper's printed results that the GPU path reproduces on its own
synthetic setups: the drop-translation trend of Sec. IV.B (Tables 1-2,
Cahn-Hilliard part alone) and the droplet-volume errors of Sec. IV.C
(Table 3, the full coupled method)."""
import math

import numpy as np
import pytest

from paper_1812_02459_gb300 import inputs, lbm

pytestmark = pytest.mark.gpu


def _translation_errors(lam, flux, steps=4000, U=0.01, sigma=0.01, precision="fp64"):
    """Drop translation of Sec. IV.B: L = 100, a 3L x L periodic box, R = 26,
    W = 4, u = (U, 0), 'tau = 0.5 + sqrt(3)/6' read as tau_f (M = eta cs^2
    (tau_f - 1/2), eta = 2).  Returns the relative extreme errors of
    Eq. (maxminPHI) read as |max phi - 1|/2 and |min phi + 1|/2, and the shift
    of the drop's centroid against U t."""
    nx, ny, R = 300, 100, 26.0
    M = 2.0 / 3.0 * (math.sqrt(3.0) / 6.0)
    prm = inputs.base_params(sigma=sigma, M=M, lam=lam, flux_correction=flux)
    phi0 = inputs.drop(nx, ny, R, 50.0, 50.0, prm["W"])
    z = np.zeros_like(phi0)
    g = lbm.Sim(prm, phi0, z, z, z, precision=precision)
    g.step_ch(np.full_like(phi0, U), z, steps)
    phi = g.fields()[0]
    g.close()
    w0, w1 = (1 + phi0) / 2, (1 + phi) / 2
    x = np.arange(nx, dtype=float)
    shift = (w1.sum(0) * x).sum() / w1.sum() - (w0.sum(0) * x).sum() / w0.sum()
    return abs(phi.max() - 1) / 2, abs(phi.min() + 1) / 2, shift / (U * steps) - 1


def test_drop_translation_lambda_trend():
    """Tables 1-2 (U = 0.01, sigma = 0.01): without the profile correction
    (lambda = 0) phi leaves [-1, 1]; lambda = 0.005 brings the extremes back
    within a small fraction of that, and the drop keeps moving with the flow.
    The paper's own values (0.063 / 0.045 at lambda = 0, 2e-5 at 0.005)
    come from an implementation with unstated details, so the trend is
    checked, not the numbers."""
    e = {lam: _translation_errors(lam, 1) for lam in (0.0, 0.001, 0.005, 0.01)}
    orig = _translation_errors(0.0, 0)
    print("translation errors", {k: tuple(round(v, 6) for v in t) for k, t in e.items()}, "original CH", orig)
    assert e[0.0][0] > 1e-3 and e[0.0][1] > 1e-3
    assert e[0.005][0] < 0.2 * e[0.0][0] and e[0.005][1] < 0.2 * e[0.0][1]
    assert e[0.001][0] < e[0.0][0] and e[0.01][0] <= e[0.001][0]
    for lam in (0.005, 0.01):
        assert abs(e[lam][2]) < 0.02


def _table3_volume_error(R, original, steps=200000):
    """Sec. IV.C: a static drop of radius R centred in a 200 x 200 periodic
    box, rho 10 / 1, sigma = 1e-3, tau_f = 0.6 (M = eta cs^2 (tau_f - 1/2),
    eta = 2), W = 4; the present method with lambda = 0.005 and the flux
    correction, "original CH" without both (reading c1).  Returns
    Err = (V(0) - V(t)) / V(0) x 100 with V the count of nodes where
    phi > 0, and V(0)."""
    n = 200
    prm = inputs.base_params(sigma=1e-3, M=2.0 / 3.0 * 0.1, rho_H=10.0, rho_L=1.0,
                             lam=0.0 if original else 0.005, flux_correction=0 if original else 1)
    phi0 = inputs.drop(n, n, R, n / 2, n / 2, prm["W"])
    z = np.zeros_like(phi0)
    g = lbm.Sim(prm, phi0, z, z, z, precision="fp32")
    v0 = g.diagnostics()[1]
    g.step(steps)
    v = g.diagnostics()[1]
    g.close()
    return 100.0 * (v0 - v) / v0, v0


@pytest.mark.slow
@pytest.mark.parametrize("R,printed", [(10, 3.9344), (20, 0.6426)])
def test_table3_volume_errors(R, printed):
    """Table 3 after 2 x 10^5 steps: the original CH method loses 3.9344 %
    (R = 10) and 0.6426 % (R = 20) of the drop's volume, the present method
    none.  The volume is a count of nodes, so the printed percentages are
    node counts (12 of 305 nodes at R = 10, 8 of 1245 at R = 20): the
    reproduction must land on the same count, within one node."""
    err_orig, v0 = _table3_volume_error(R, True)
    err_present, _ = _table3_volume_error(R, False)
    print("table 3", R, err_orig, err_present, v0)
    node = 100.0 / v0
    assert abs(err_orig - printed) <= node + 1e-9
    assert abs(err_present) <= node + 1e-9


def _vortex(original, n_periods=2, L=400, lam=0.005):
    """Sec. IV.A: a circular drop (R = 0.15 L at (0.5 L, 0.75 L)) in the single
    vortex u = U0 sin^2(pi x) sin(2 pi y) cos(pi t/T),
    v = -U0 sin^2(pi y) sin(2 pi x) cos(pi t/T), T = n L/U0, run to 2T when
    the flow has brought it back.  sigma = 1e-3, W = 4, U0 = 0.02, tau_f read
    as 0.5 + sqrt(3)/6 (reading c4).  Returns the range of phi at 2T and
    the rms distance of phi(2T) from phi(0)."""
    U0 = 0.02
    T = n_periods * L / U0
    prm = inputs.base_params(sigma=1e-3, M=2.0 / 3.0 * (math.sqrt(3.0) / 6.0),
                             lam=0.0 if original else lam, flux_correction=0 if original else 1)
    phi0 = inputs.drop(L, L, 0.15 * L, 0.5 * L, 0.75 * L, prm["W"])
    z = np.zeros_like(phi0)
    y, x = np.mgrid[0:L, 0:L].astype(float)
    X, Y = (x + 0.5) / L, (y + 0.5) / L
    ux = U0 * np.sin(math.pi * X) ** 2 * np.sin(2 * math.pi * Y)
    uy = -U0 * np.sin(math.pi * Y) ** 2 * np.sin(2 * math.pi * X)
    g = lbm.Sim(prm, phi0, z, z, z, precision="fp32")
    nsteps = int(2 * T)
    for s0 in range(0, nsteps, 8000):
        k = min(8000, nsteps - s0)
        g.step_ch(ux, uy, k, tfac=np.cos(math.pi * (s0 + np.arange(k)) / T))
    phi = g.fields()[0]
    g.close()
    return phi.min(), phi.max(), float(np.sqrt(((phi - phi0) ** 2).mean()))


@pytest.mark.slow
def test_single_vortex_returns_drop():
    """Sec. IV.A: with the profile and flux corrections phi stays in [-1, 1]
    and the drop comes back to its initial shape far closer than under the
    original CH method, which over- and undershoots by about 0.1.  Here the
    present method runs at lambda = 0.005: at the paper's lambda = 0.05 this
    implementation goes unstable on the stretched filament, as the paper
    reports for its own translation test at small sigma (Tables 1-2)."""
    lo, hi, d_present = _vortex(False)
    lo_o, hi_o, d_orig = _vortex(True)
    print("vortex", (lo, hi, d_present), (lo_o, hi_o, d_orig))
    assert lo > -1.0 - 1e-3 and hi < 1.0 + 1e-3
    assert min(lo_o, -hi_o) < -1.05
    assert d_present < 0.25 * d_orig
