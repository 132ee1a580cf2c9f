"""The capillary wave against Prosperetti's analytic solution
(tests/capillary_analytic.py): a small-amplitude cosine interface between two
fluids of equal kinematic viscosity, released from rest, no gravity (the
paper's capillary-wave case, Sec. IV).  The analytic routine is pinned to its
own limits first; then the C oracle and the GPU path are compared with it.

The simulation runs in a channel of depth 2 lambda (walls in y, k h = 2 pi
per side, so the finite depth is negligible) with the interface width W = 4.
The diffuse interface makes the period a few percent long, and the error
shrinks as lambda / W grows: measured with FP64, equal densities, 7.0 % at
lambda = 64, 5.0 % at 128, 4.0 % at 256."""
import numpy as np
import pytest

import oracle
from paper_1812_02459_gb300 import inputs

from capillary_analytic import amplitude

NU = 1.0 / 30


def test_analytic_limits():
    k = 2 * np.pi / 64
    for rho1, sigma in ((1.0, 0.08), (10.0, 0.4), (1000.0, 0.02)):
        assert amplitude(np.array([0.0]), sigma, k, rho1, 1.0, NU)[0] == pytest.approx(1.0, abs=1e-12)
        w0 = np.sqrt(sigma * k ** 3 / (rho1 + 1.0))
        t = np.array([0.3, 0.8, 1.7]) * 2 * np.pi / w0
        # vanishing viscosity: the undamped oscillation cos(omega0 t)
        assert np.allclose(amplitude(t, sigma, k, rho1, 1.0, 1e-12), np.cos(w0 * t), atol=1e-5)
    # free-surface limit (upper fluid 1e5 times lighter), weak damping: after
    # many periods the envelope decays at Lamb's rate, exp(-2 nu k^2 t)
    k = 2 * np.pi / 256
    rho1, nu = 1e5, 1e-4
    sigma = 0.5 * rho1
    w0 = np.sqrt(sigma * k ** 3 / (rho1 + 1.0))
    for periods in (10, 40):
        t = np.linspace(periods, periods + 2, 800) * 2 * np.pi / w0
        env = np.abs(amplitude(t, sigma, k, rho1, 1.0, nu)).max()
        assert env == pytest.approx(np.exp(-2 * nu * k * k * t[0]), rel=1e-4)


def interface_mode(phi, k):
    """Amplitude of the cos(k x) mode of the interface height (the phi = 0
    crossing of each column, heavy fluid below, linearly interpolated)."""
    ny, nx = phi.shape
    h = np.empty(nx)
    for x in range(nx):
        c = phi[:, x]
        j = np.where((c[:-1] > 0) & (c[1:] <= 0))[0][0]
        h[x] = j + c[j] / (c[j] - c[j + 1])
    return 2.0 / nx * np.sum(h * np.cos(k * np.arange(nx)))


def wave(lam, rho1):
    prm = inputs.base_params(M=0.05, sigma=0.08, rho_H=rho1, rho_L=1.0, nu_H=NU, nu_L=NU,
                             periodic_x=1, periodic_y=0)
    phi = inputs.flat_interface(lam, 2 * lam, lam, prm["W"], amp=0.01 * lam, wavelength=lam)
    z = np.zeros((2 * lam, lam))
    return prm, (phi, z, z, z)


def first_crossing(ts, a):
    i = np.where(np.sign(a[:-1]) != np.sign(a[1:]))[0][0]
    return ts[i] + (ts[i + 1] - ts[i]) * a[i] / (a[i] - a[i + 1])


def track(sim, lam, steps, every):
    k = 2 * np.pi / lam
    a0 = interface_mode(sim.fields()[0], k)
    ts, am = [0.0], [1.0]
    for i in range(steps // every):
        sim.step(every)
        ts.append(every * (i + 1.0))
        am.append(interface_mode(sim.fields()[0], k) / a0)
    return np.array(ts), np.array(am)


def test_oracle_against_analytic():
    """The C oracle at lambda = 64, equal densities, to the first trough."""
    lam = 64
    prm, fields = wave(lam, 1.0)
    sim = oracle.Sim(prm, *fields)
    ts, am = track(sim, lam, 700, 10)
    an = amplitude(ts, 0.08, 2 * np.pi / lam, 1.0, 1.0, NU)
    c_sim, c_an = first_crossing(ts, am), first_crossing(ts, an)
    assert 0.0 < c_sim / c_an - 1.0 < 0.09      # the period is a few percent long (7.0 % measured)
    assert abs(am.min() - an.min()) < 0.06      # depth of the first trough, of a0 (0.034 measured)


@pytest.mark.gpu
def test_gpu_converges_to_analytic():
    """FP64 on the GPU at lambda = 64 and 128: the period error shrinks as
    lambda / W grows, for equal densities and a density ratio of 10."""
    from paper_1812_02459_gb300 import lbm
    for rho1, bounds in ((1.0, (0.08, 0.06)), (10.0, (0.08, 0.065))):
        errs = []
        for lam, bound in zip((64, 128), bounds):
            prm, fields = wave(lam, rho1)
            sim = lbm.Sim(prm, *fields, precision="fp64")
            steps = (1200 if lam == 64 else 3200) * (2 if rho1 > 1 else 1)
            ts, am = track(sim, lam, steps, 10 if lam == 64 else 20)
            sim.close()
            an = amplitude(ts, 0.08, 2 * np.pi / lam, rho1, 1.0, NU)
            err = first_crossing(ts, am) / first_crossing(ts, an) - 1.0
            assert 0.0 < err < bound, (rho1, lam, err)
            errs.append(err)
        assert errs[1] < errs[0]
