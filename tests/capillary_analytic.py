"""Small-amplitude capillary wave between two fluids of equal kinematic
viscosity: the initial-value solution of Prosperetti (Phys. Fluids 24, 1217,
1981) for an interface released from rest with amplitude a0, no gravity,
unbounded fluids.  Used as an analytic reference for the capillary-wave
workload (the paper's Sec. IV capillary-wave case, E5).

With beta = rho1 rho2 / (rho1 + rho2)^2, omega0^2 = sigma k^3 / (rho1 + rho2)
and n = nu k^2, the amplitude is

  a(t)/a0 = 4 (1 - 4 beta) n^2 / (8 (1 - 4 beta) n^2 + omega0^2) erfc(sqrt(n t))
          + sum_i  z_i / Z_i  omega0^2 / (z_i^2 - n)  exp((z_i^2 - n) t) erfc(z_i sqrt(t)),

z_i the four roots of
  z^4 - 4 beta n^(1/2) z^3 + 2 (1 - 6 beta) n z^2 + 4 (1 - 3 beta) n^(3/2) z
      + (1 - 4 beta) n^2 + omega0^2 = 0,
Z_i = prod_{j != i} (z_j - z_i).  exp(z^2 t) erfc(z sqrt t) is evaluated as the
Faddeeva function w(i z sqrt t), which stays finite for every root.
"""
import numpy as np
from scipy.special import erfc, wofz


def amplitude(t, sigma, k, rho1, rho2, nu):
    """a(t)/a0 at the times t (array), real part (the imaginary parts of the
    conjugate roots' terms cancel)."""
    t = np.asarray(t, dtype=float)
    beta = rho1 * rho2 / (rho1 + rho2) ** 2
    w02 = sigma * k ** 3 / (rho1 + rho2)
    n = nu * k * k
    sn = np.sqrt(n)
    z = np.roots([1.0, -4.0 * beta * sn, 2.0 * (1.0 - 6.0 * beta) * n, 4.0 * (1.0 - 3.0 * beta) * n * sn,
                  (1.0 - 4.0 * beta) * n * n + w02]).astype(complex)
    a = 4.0 * (1.0 - 4.0 * beta) * n * n / (8.0 * (1.0 - 4.0 * beta) * n * n + w02) * erfc(np.sqrt(n * t))
    a = a.astype(complex)
    for i in range(4):
        Zi = np.prod([z[j] - z[i] for j in range(4) if j != i])
        ci = z[i] / Zi * w02 / (z[i] ** 2 - n)
        a = a + ci * np.exp(-n * t) * wofz(1j * z[i] * np.sqrt(t))
    return a.real
