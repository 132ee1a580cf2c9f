"""Seeded synthetic inputs: initial fields and parameter sets of the workloads.

This module holds no arithmetic of the lattice Boltzmann method itself.  It
only writes down initial order-parameter, pressure and velocity fields (the
tanh interface profile of Sec. II.A Eq. (equilibrium_profile) placed as a
drop, a bubble or a perturbed flat interface) and plain dictionaries of model
parameters.  Both the CUDA path and the FP64 oracle consume what it returns.

Fields are float64 numpy arrays shaped [ny, nx]; x = column index i,
y = row index j, node coordinates are the integer indices.
"""
import math

import numpy as np

# MRT rates: s_f[3], s_f[5] are replaced by 1/tau_f and s_g[7], s_g[8] by
# 1/tau_g(x) inside the solver; the rest are the paper-silent defaults.
S_F_DEFAULT = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0)
S_G_DEFAULT = (1.0, 1.0, 1.0, 1.0, 1.7, 1.0, 1.7, 1.0, 1.0)


def base_params(**kw):
    """Parameter dictionary with the defaults used throughout the workloads."""
    p = dict(M=0.1, eta=2.0, W=4.0, sigma=1e-3, lam=0.005, flux_correction=1,
             rho_H=10.0, rho_L=1.0, nu_H=0.1, nu_L=0.1,
             s_f=list(S_F_DEFAULT), s_g=list(S_G_DEFAULT),
             gx=0.0, gy=0.0, g_rho_ref=0.0, filter_order=11, filter_a=0.5,
             picard_iters=2, picard_zeta=0.0, grad_eps=1e-4,
             periodic_x=1, periodic_y=1)
    p.update(kw)
    p["lambda"] = p.pop("lam")
    return p


def zeros(nx, ny):
    return np.zeros((ny, nx))


def drop(nx, ny, R, xc, yc, W, inside=+1.0):
    """phi = inside * tanh(2 (R - r)/W): a circular drop (inside=+1, heavy) or bubble (-1)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return inside * np.tanh(2.0 * (R - r) / W)


def flat_interface(nx, ny, y0, W, amp=0.0, wavelength=None):
    """Heavy fluid (phi=+1) below y = y0 + amp cos(2 pi x / wavelength)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    wl = wavelength if wavelength is not None else nx
    h = y0 + amp * np.cos(2.0 * math.pi * x / wl)
    return np.tanh(2.0 * (h - y) / W)


def random_fields(nx, ny, seed, phi_amp=0.9, u_amp=1e-3, p_amp=1e-4):
    """Smooth random fields for parity checks: a few random Fourier modes."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)

    def smooth(amp):
        out = np.zeros((ny, nx))
        for _ in range(4):
            kx = rng.integers(1, 3); ky = rng.integers(1, 3)
            ph = rng.uniform(0, 2 * math.pi)
            out += rng.normal() * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny) + ph)
        return amp * out / 4.0

    phi = np.tanh(3.0 * smooth(1.0)) * phi_amp
    return phi, smooth(p_amp), smooth(u_amp), smooth(u_amp)


# ---- the named workloads -------------------------------------------------

def static_drop(n=64, R=16.0):
    """Static drop (Laplace law): periodic n x n, drop R centred, rho ratio 10."""
    prm = base_params(M=0.1, sigma=1e-3, rho_H=10.0, rho_L=1.0, nu_H=0.1, nu_L=0.1)
    phi = drop(n, n, R, n / 2, n / 2, prm["W"], inside=+1.0)
    return prm, (phi, zeros(n, n), zeros(n, n), zeros(n, n))


def bubble_params(R, rho_ratio=1000.0, mu_ratio=100.0, Eo=10.0, Mo=1e-3, nu_H=1.0 / 300, M=0.05):
    """Rising-bubble parameters from the Eotvos and Morton numbers.

    Eo = rho_H g (2R)^2 / sigma, Mo = g mu_H^4 (rho_H - rho_L) / (rho_H^2 sigma^3),
    with rho_L = 1, rho_H = rho_ratio, mu_H = rho_H nu_H, mu_L = mu_H / mu_ratio.
    Gravity is measured against the liquid's hydrostatic pressure
    (g_rho_ref = rho_H): the buoyancy (rho - rho_H) g acts on the bubble only.
    """
    rho_H, rho_L = rho_ratio, 1.0
    mu_H = rho_H * nu_H
    mu_L = mu_H / mu_ratio
    sigma = math.sqrt(Eo * mu_H ** 4 * (rho_H - rho_L) / (4.0 * R * R * rho_H ** 3 * Mo))
    g = Eo * sigma / (rho_H * 4.0 * R * R)
    return base_params(M=M, sigma=sigma, rho_H=rho_H, rho_L=rho_L, nu_H=nu_H,
                       nu_L=mu_L / rho_L, gx=0.0, gy=-g, g_rho_ref=rho_H,
                       periodic_x=1, periodic_y=0)


def rising_bubble(nx=256, ny=512, R=32.0, yc=128.0, nu_H=1.0 / 600):
    """Rising bubble: periodic x, walls in y, light bubble (phi=-1) in heavy liquid,
    density ratio 1000, viscosity ratio 100, Eo = 10, Mo = 1e-3.  At R = 32 the
    liquid viscosity 1/600 keeps the buoyancy and surface tension in the range
    where the scheme runs stably at this density ratio (sigma = 0.0043)."""
    prm = bubble_params(R, nu_H=nu_H)
    phi = drop(nx, ny, R, nx / 2, yc, prm["W"], inside=-1.0)
    return prm, (phi, zeros(nx, ny), zeros(nx, ny), zeros(nx, ny))


def rising_bubble_large(nx=1024, ny=2048, R=128.0, yc=512.0):
    """The same bubble at four times the resolution (same Eo, Mo; nu_H = 1/300,
    which gives the same sigma = 0.0043 as the 256 x 512 case)."""
    return rising_bubble(nx, ny, R, yc, nu_H=1.0 / 300)


def capillary_wave(n=512, rho_ratio=1000.0):
    """Capillary wave: heavy below a cos-perturbed flat interface, amplitude 0.01 n."""
    prm = base_params(M=0.05, sigma=0.02, rho_H=rho_ratio, rho_L=1.0,
                      nu_H=1.0 / 30, nu_L=1.0 / 30, periodic_x=1, periodic_y=0)
    phi = flat_interface(n, n, n / 2, prm["W"], amp=0.01 * n)
    return prm, (phi, zeros(n, n), zeros(n, n), zeros(n, n))


def translating_drop(n=256, R=32.0, U0=0.01):
    """Drop carried by a uniform flow: periodic n x n, rho ratio 100."""
    prm = base_params(M=0.1, sigma=0.01, rho_H=100.0, rho_L=1.0, nu_H=0.1, nu_L=0.1)
    phi = drop(n, n, R, n / 2, n / 2, prm["W"], inside=+1.0)
    return prm, (phi, zeros(n, n), np.full((n, n), U0), zeros(n, n))
