"""FP64 oracle of the fractional-step MRT lattice Boltzmann method -- TEST INFRASTRUCTURE.

A ctypes front end over ``liblbm_oracle.so`` (plain single-threaded C, built
by ``oracle/build.py``).  Only the test-suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package; the product path
never does.  It shares no code with the CUDA library.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)


class OrcParams(C.Structure):
    """Mirror of ``orc_params`` in lbm_oracle.h."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("periodic_x", C.c_int), ("periodic_y", C.c_int),
        ("M", C.c_double), ("eta", C.c_double), ("W", C.c_double),
        ("sigma", C.c_double), ("lambda_", C.c_double),
        ("flux_correction", C.c_int),
        ("rho_H", C.c_double), ("rho_L", C.c_double),
        ("nu_H", C.c_double), ("nu_L", C.c_double),
        ("s_f", C.c_double * 9), ("s_g", C.c_double * 9),
        ("gx", C.c_double), ("gy", C.c_double), ("g_rho_ref", C.c_double),
        ("filter_order", C.c_int), ("filter_a", C.c_double),
        ("picard_iters", C.c_int), ("picard_zeta", C.c_double),
        ("grad_eps", C.c_double),
        ("flags", C.c_uint),
    ]


_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_int
        L.orc_create.argtypes = [C.POINTER(OrcParams), _dp, _dp, _dp, _dp, C.POINTER(C.c_void_p)]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_step_ch.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.orc_step_ch.restype = C.c_int
        L.orc_fields.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_dynamic_pressure.argtypes = [C.c_void_p, _dp]
        L.orc_set_state.argtypes = [C.c_void_p] + [_dp] * 10
        L.orc_diagnostics.argtypes = [C.c_void_p, _dp]
        L.orc_last_picard_sweeps.restype = C.c_int
        L.orc_last_picard_sweeps.argtypes = [C.c_void_p]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_fd_rhs.argtypes = [C.POINTER(OrcParams), _dp, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(nx, ny, prm):
    """Fill an OrcParams from grid sizes and a plain dict of model parameters."""
    p = OrcParams()
    p.nx, p.ny = int(nx), int(ny)
    p.periodic_x = int(prm.get("periodic_x", 1))
    p.periodic_y = int(prm.get("periodic_y", 1))
    p.M = prm["M"]; p.eta = prm["eta"]; p.W = prm["W"]; p.sigma = prm["sigma"]
    p.lambda_ = prm["lambda"]
    p.flux_correction = int(prm.get("flux_correction", 1))
    p.rho_H = prm["rho_H"]; p.rho_L = prm["rho_L"]
    p.nu_H = prm["nu_H"]; p.nu_L = prm["nu_L"]
    for k in range(9):
        p.s_f[k] = prm["s_f"][k]
        p.s_g[k] = prm["s_g"][k]
    p.gx = prm.get("gx", 0.0); p.gy = prm.get("gy", 0.0)
    p.g_rho_ref = prm.get("g_rho_ref", 0.0)
    p.filter_order = int(prm.get("filter_order", 11))
    p.filter_a = prm.get("filter_a", 0.5)
    p.picard_iters = int(prm.get("picard_iters", 2))
    p.picard_zeta = prm.get("picard_zeta", 0.0)
    p.grad_eps = prm.get("grad_eps", 1e-4)
    p.flags = int(prm.get("flags", 0))
    return p


# ---- building blocks ------------------------------------------------------

def lattice():
    c = (C.c_int * 18)(); w = (C.c_double * 9)()
    lib().orc_lattice(c, w)
    return np.array(c[:], dtype=np.int64).reshape(9, 2), np.array(w[:])


def mrt_matrix():
    m = (C.c_double * 81)(); lib().orc_mrt_matrix(m)
    return np.array(m[:]).reshape(9, 9)


def mrt_inverse():
    m = (C.c_double * 81)(); lib().orc_mrt_inverse(m)
    return np.array(m[:]).reshape(9, 9)


def filter_coeffs(order):
    d = (C.c_double * 6)(); lib().orc_filter_coeffs(C.c_int(order), d)
    return np.array(d[:])


def _node9(fn, *args):
    out = (C.c_double * 9)()
    fn(*[C.c_double(a) for a in args], out)
    return np.array(out[:])


def feq(phi, mu, ux, uy, eta):
    return _node9(lib().orc_feq, phi, mu, ux, uy, eta)


def geq(p, ux, uy):
    return _node9(lib().orc_geq, p, ux, uy)


def src_ch(phi, ax, ay):
    return _node9(lib().orc_src_ch, phi, ax, ay)


def src_ns(rho, Fx, Fy, ux, uy, dpx, dpy):
    return _node9(lib().orc_src_ns, rho, Fx, Fy, ux, uy, dpx, dpy)


def _arr9(a):
    return (C.c_double * 9)(*[float(v) for v in a])


def collide_f(f, fe, F, s):
    out = (C.c_double * 9)()
    lib().orc_collide_f(_arr9(f), _arr9(fe), _arr9(F), _arr9(s), out)
    return np.array(out[:])


def strain_moments(g, geq, s, rho, Fx, Fy, ux, uy):
    """(S_xx, S_xy, S_yy) of Sec. III.B Eq. (Fmu) at one node."""
    out = (C.c_double * 3)()
    lib().orc_strain_moments(_arr9(g), _arr9(geq), _arr9(s), C.c_double(rho), C.c_double(Fx), C.c_double(Fy),
                             C.c_double(ux), C.c_double(uy), out)
    return np.array(out[:])


def collide_g(g, ge_f, ge_h, G, s):
    out = (C.c_double * 9)()
    lib().orc_collide_g(_arr9(g), _arr9(ge_f), _arr9(ge_h), _arr9(G), _arr9(s), out)
    return np.array(out[:])


def _field_op2(fname, a, px, py, parity):
    a = _f64(a); ny, nx = a.shape
    gx = np.empty_like(a); gy = np.empty_like(a)
    getattr(lib(), fname)(C.c_int(nx), C.c_int(ny), C.c_int(px), C.c_int(py),
                          C.c_int(parity), _ptr(a), _ptr(gx), _ptr(gy))
    return gx, gy


def _field_op1(fname, a, px, py, parity):
    a = _f64(a); ny, nx = a.shape
    out = np.empty_like(a)
    getattr(lib(), fname)(C.c_int(nx), C.c_int(ny), C.c_int(px), C.c_int(py),
                          C.c_int(parity), _ptr(a), _ptr(out))
    return out


def grad_iso(a, px=1, py=1, parity=1):
    return _field_op2("orc_grad_iso", a, px, py, parity)


def lap_iso(a, px=1, py=1, parity=1):
    return _field_op1("orc_lap_iso", a, px, py, parity)


def grad_fd4(a, px=1, py=1, parity=1):
    return _field_op2("orc_grad_fd4", a, px, py, parity)


def lap_fd4(a, px=1, py=1, parity=1):
    return _field_op1("orc_lap_fd4", a, px, py, parity)


def filter_field(a, order=11, alpha=0.5, px=1, py=1, parity=1):
    a = _f64(a); ny, nx = a.shape
    out = np.empty_like(a)
    lib().orc_filter(C.c_int(nx), C.c_int(ny), C.c_int(px), C.c_int(py), C.c_int(parity),
                     C.c_int(order), C.c_double(alpha), _ptr(a), _ptr(out))
    return out


def stream(fstar, px=1, py=1):
    fstar = _f64(fstar); q, ny, nx = fstar.shape
    out = np.empty_like(fstar)
    lib().orc_stream(C.c_int(nx), C.c_int(ny), C.c_int(px), C.c_int(py), _ptr(fstar), _ptr(out))
    return out


def fd_rhs(psi, prm):
    psi = _f64(psi); ny, nx = psi.shape
    p = make_params(nx, ny, prm)
    out = np.empty_like(psi)
    lib().orc_fd_rhs(C.byref(p), _ptr(psi), _ptr(out))
    return out


_RHS = C.CFUNCTYPE(None, _dp, _dp, C.c_int, C.c_void_p)


def rk3(phibar, L):
    """Advance phibar by the TVD-RK3 combination with a Python right-hand side L(psi)."""
    phibar = _f64(phibar).ravel()
    n = phibar.size

    def cb(psi_p, out_p, nn, ctx):
        psi = np.ctypeslib.as_array(psi_p, shape=(nn,))
        out = np.ctypeslib.as_array(out_p, shape=(nn,))
        out[:] = L(psi.copy())

    fn = _RHS(cb)
    out = np.empty_like(phibar)
    lib().orc_rk3(C.c_int(n), _ptr(phibar), _ptr(out), fn, None)
    return out


# ---- whole-method simulation ------------------------------------------------

class Sim:
    """An FP64 oracle simulation; fields are numpy arrays shaped [ny, nx]."""

    def __init__(self, prm, phi0, p0, ux0, uy0):
        phi0, p0, ux0, uy0 = (_f64(a) for a in (phi0, p0, ux0, uy0))
        self.ny, self.nx = phi0.shape
        self.params = make_params(self.nx, self.ny, prm)
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(self.params), _ptr(phi0), _ptr(p0), _ptr(ux0), _ptr(uy0),
                              C.byref(h))
        if rc != 0:
            raise ValueError(f"orc_create failed with {rc}")
        self._h = h

    def step(self, n=1):
        rc = lib().orc_step(self._h, C.c_int(n))
        if rc != 0:
            raise FloatingPointError(f"oracle step returned {rc} (non-finite field)")

    def step_ch(self, ux, uy, n=1):
        """n steps of the Cahn-Hilliard part alone under the prescribed velocity (ux, uy)."""
        ux, uy = _f64(ux), _f64(uy)
        rc = lib().orc_step_ch(self._h, C.c_int(n), _ptr(ux), _ptr(uy))
        if rc != 0:
            raise FloatingPointError(f"oracle CH step returned {rc} (non-finite phi)")

    def fields(self):
        shp = (self.ny, self.nx)
        phi, p, ux, uy = (np.empty(shp) for _ in range(4))
        lib().orc_fields(self._h, _ptr(phi), _ptr(p), _ptr(ux), _ptr(uy))
        return phi, p, ux, uy

    def dynamic_pressure(self):
        """p' = rho(phi) p, Sec. II.B (p = p'/rho), as a [ny, nx] array."""
        out = np.empty((self.ny, self.nx))
        lib().orc_dynamic_pressure(self._h, _ptr(out))
        return out

    def state(self):
        shp = (self.ny, self.nx)
        f = np.empty((9,) + shp); g = np.empty((9,) + shp)
        uhx, uhy, upx, upy = (np.empty(shp) for _ in range(4))
        lib().orc_state(self._h, _ptr(f), _ptr(g), _ptr(uhx), _ptr(uhy), _ptr(upx), _ptr(upy))
        return dict(f=f, g=g, uhx=uhx, uhy=uhy, upx=upx, upy=upy)

    def set_state(self, f, g, phi, p, ux, uy, uhx, uhy, upx, upy):
        arrs = [_f64(a) for a in (f, g, phi, p, ux, uy, uhx, uhy, upx, upy)]
        lib().orc_set_state(self._h, *[_ptr(a) for a in arrs])

    def diagnostics(self):
        out = (C.c_double * 10)()
        lib().orc_diagnostics(self._h, out)
        return np.array(out[:])

    def last_picard_sweeps(self):
        return lib().orc_last_picard_sweeps(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
