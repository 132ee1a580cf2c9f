"""The oracle's Cahn-Hilliard step under a prescribed velocity (orc_step_ch;
the paper's interface-capturing tests of Sec. IV.A, where the flow is given):
the CH collision, streaming and the TVD-RK3 correction without the NS
lattice.  Pinned to what the mathematics fixes: the sum of phi is conserved
to round-off (every step is a conservative update on a periodic grid), and a
drop carried by a uniform flow is the drop at rest, shifted -- up to an
advection error that vanishes with the speed."""
import numpy as np
import pytest

import oracle
from paper_1812_02459_gb300 import inputs

N = 64


def drop_case():
    prm = inputs.base_params(M=0.1, sigma=1e-3, rho_H=10.0, rho_L=1.0)
    return prm, inputs.drop(N, N, 10.0, N / 2, N / 2, prm["W"])


def carried(prm, phi0, U, steps):
    z = np.zeros((N, N))
    u = np.full((N, N), U)
    s = oracle.Sim(prm, phi0, z, u, z)
    s.step_ch(u, z, steps)
    return s.fields()[0]


def test_sum_of_phi_conserved():
    prm, phi0 = drop_case()
    for U, V in ((0.0, 0.0), (0.05, -0.03)):
        z = np.zeros((N, N))
        s = oracle.Sim(prm, phi0, z, np.full((N, N), U), np.full((N, N), V))
        s0 = s.fields()[0].sum()
        s.step_ch(np.full((N, N), U), np.full((N, N), V), 200)
        assert abs(s.fields()[0].sum() - s0) <= 1e-12 * phi0.size


def test_uniform_flow_shifts_the_drop():
    """A 16-node shift at three speeds: the difference from the drop relaxed
    at rest for the same number of steps, shifted, falls with the speed."""
    prm, phi0 = drop_case()
    errs = []
    for U in (0.1, 0.05, 0.02):
        steps = int(round(16 / U))
        rest = carried(prm, phi0, 0.0, steps)
        errs.append(np.abs(carried(prm, phi0, U, steps) - np.roll(rest, 16, axis=1)).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.015          # 0.0088 measured
    # the drop at rest only relaxes its discrete profile
    assert np.abs(carried(prm, phi0, 0.0, 200) - phi0).max() < 0.01
