"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the lattice update runs in the CUDA kernels of ``liblbm.so``;
this module only converts arguments and raises on error codes.  There is no
CPU fallback: if the library cannot be loaded, importing a solver fails.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)

LBM_NDIAG = 11
LBM_MIN_EXTENT = 12
PRECISIONS = {"fp64": 0, "fp32": 1, "mix_bf16": 2, "mix_fp16": 3}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_CUDA", 3: "LBM_ERR_OOM",
          4: "LBM_ERR_NONFINITE", 5: "LBM_ERR_RANGE", 6: "LBM_ERR_STATE"}


class LbmGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("periodic_x", C.c_int),
                ("periodic_y", C.c_int), ("precision", C.c_int)]


class LbmParams(C.Structure):
    _fields_ = [
        ("M", C.c_double), ("eta", C.c_double), ("W", C.c_double), ("sigma", C.c_double),
        ("lambda_", C.c_double), ("flux_correction", C.c_int),
        ("rho_H", C.c_double), ("rho_L", C.c_double), ("nu_H", C.c_double), ("nu_L", C.c_double),
        ("s_f", C.c_double * 9), ("s_g", C.c_double * 9),
        ("gx", C.c_double), ("gy", C.c_double), ("g_rho_ref", C.c_double),
        ("filter_order", C.c_int), ("filter_a", C.c_double),
        ("picard_iters", C.c_int), ("picard_zeta", C.c_double),
        ("grad_eps", C.c_double), ("flags", C.c_uint),
    ]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


EXPORTS = ("lbm_create", "lbm_step", "lbm_step_ch", "lbm_fields", "lbm_dynamic_pressure", "lbm_fields_device",
           "lbm_set_fields",
           "lbm_diagnostics", "lbm_diagnostics_async", "lbm_check", "lbm_set_check", "lbm_get_state", "lbm_set_state",
           "lbm_profile", "lbm_profile_read", "lbm_kernel_name", "lbm_kernel_variant",
           "lbm_field_sums_noalloc", "lbm_noalloc_last_error",
           "lbm_adjoint_begin", "lbm_adjoint_end", "lbm_adjoint_engine",
           "lbm_device_bytes", "lbm_destroy", "lbm_last_error", "lbm_debug_violations")
LBM_NKERNELS = 4

_lib = None


def load(path=None):
    """Load liblbm.so (building it first when missing); raise if that fails."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        p = _build.build()
    L = C.CDLL(p)
    vp = C.c_void_p
    L.lbm_create.restype = C.c_int
    L.lbm_create.argtypes = [C.POINTER(LbmGrid), C.POINTER(LbmParams), _dp, _dp, _dp, _dp, vp,
                             C.POINTER(vp)]
    L.lbm_step.restype = C.c_int
    L.lbm_step.argtypes = [vp, C.c_int]
    L.lbm_step_ch.restype = C.c_int
    L.lbm_step_ch.argtypes = [vp, C.c_int, _dp, _dp, _dp]
    L.lbm_fields.restype = C.c_int
    L.lbm_fields.argtypes = [vp, _dp, _dp, _dp, _dp]
    L.lbm_dynamic_pressure.restype = C.c_int
    L.lbm_dynamic_pressure.argtypes = [vp, _dp]
    L.lbm_fields_device.restype = C.c_int
    L.lbm_fields_device.argtypes = [vp, vp, vp, vp, vp, C.c_int]
    L.lbm_set_fields.restype = C.c_int
    L.lbm_set_fields.argtypes = [vp, _dp, _dp, _dp, _dp]
    L.lbm_diagnostics.restype = C.c_int
    L.lbm_diagnostics.argtypes = [vp, _dp]
    L.lbm_diagnostics_async.restype = C.c_int
    L.lbm_diagnostics_async.argtypes = [vp, _dp]
    L.lbm_check.restype = C.c_int
    L.lbm_check.argtypes = [vp, C.c_double]
    L.lbm_set_check.restype = C.c_int
    L.lbm_set_check.argtypes = [vp, C.c_int, C.c_double]
    L.lbm_get_state.restype = C.c_int
    L.lbm_get_state.argtypes = [vp] + [_dp] * 10
    L.lbm_set_state.restype = C.c_int
    L.lbm_set_state.argtypes = [vp] + [_dp] * 10
    L.lbm_profile.restype = C.c_int
    L.lbm_profile.argtypes = [vp, C.c_int]
    L.lbm_profile_read.restype = C.c_int
    L.lbm_profile_read.argtypes = [vp, _dp, C.POINTER(C.c_longlong)]
    L.lbm_kernel_name.restype = C.c_char_p
    L.lbm_kernel_name.argtypes = [C.c_int]
    L.lbm_kernel_variant.restype = C.c_char_p
    L.lbm_kernel_variant.argtypes = [C.c_void_p, C.c_int]
    L.lbm_field_sums_noalloc.restype = C.c_int
    L.lbm_field_sums_noalloc.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, vp, vp]
    L.lbm_noalloc_last_error.restype = C.c_char_p
    L.lbm_noalloc_last_error.argtypes = []
    L.lbm_adjoint_begin.restype = C.c_int
    L.lbm_adjoint_begin.argtypes = [vp, C.c_int, C.c_int]
    L.lbm_adjoint_end.restype = C.c_int
    L.lbm_adjoint_end.argtypes = [vp, _dp, _dp, _dp, _dp]
    L.lbm_adjoint_engine.restype = C.c_int
    L.lbm_adjoint_engine.argtypes = [vp]
    L.lbm_device_bytes.restype = C.c_size_t
    L.lbm_device_bytes.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_destroy.argtypes = [vp]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_last_error.argtypes = [vp]
    L.lbm_debug_violations.restype = C.c_ulonglong
    L.lbm_debug_violations.argtypes = []
    if path is None:
        _lib = L
    return L


def make_params(prm):
    """lbm_params from a plain dict (keys as in inputs.base_params)."""
    p = LbmParams()
    p.M = prm["M"]; p.eta = prm["eta"]; p.W = prm["W"]; p.sigma = prm["sigma"]
    p.lambda_ = prm["lambda"]; p.flux_correction = int(prm.get("flux_correction", 1))
    p.rho_H = prm["rho_H"]; p.rho_L = prm["rho_L"]; p.nu_H = prm["nu_H"]; p.nu_L = prm["nu_L"]
    for k in range(9):
        p.s_f[k] = prm["s_f"][k]
        p.s_g[k] = prm["s_g"][k]
    p.gx = prm.get("gx", 0.0); p.gy = prm.get("gy", 0.0); p.g_rho_ref = prm.get("g_rho_ref", 0.0)
    p.filter_order = int(prm.get("filter_order", 11)); p.filter_a = prm.get("filter_a", 0.5)
    p.picard_iters = int(prm.get("picard_iters", 2)); p.picard_zeta = prm.get("picard_zeta", 0.0)
    p.grad_eps = prm.get("grad_eps", 1e-4); p.flags = int(prm.get("flags", 0))
    return p


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def current_stream():
    """The current torch CUDA stream handle, or 0 (legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


LBM_NOALLOC_MAX_NODES = 67108864


def field_sums_noalloc(phi, p, ux, uy, out, stream=None):
    """lbm_field_sums_noalloc on caller-owned device tensors (float32 or float64,
    shaped [ny, nx]); out is a device float64 tensor of LBM_NDIAG elements."""
    L = load()
    ny, nx = phi.shape
    dt = {"torch.float64": 0, "torch.float32": 1}[str(phi.dtype)]
    ptr = lambda t: C.c_void_p(t.data_ptr())
    st = L.lbm_field_sums_noalloc(ptr(phi), ptr(p), ptr(ux), ptr(uy), nx, ny, dt, ptr(out),
                                  C.c_void_p(current_stream() if stream is None else stream))
    if st != 0:
        raise LbmError(st, L.lbm_noalloc_last_error().decode())


class Sim:
    """A simulation on the GPU; host fields are float64 numpy arrays shaped [ny, nx]."""

    def __init__(self, prm, phi0, p0, ux0, uy0, precision="fp32", stream=None, lib=None):
        self._lib = lib if lib is not None else load()
        phi0, p0, ux0, uy0 = (_f64(a) for a in (phi0, p0, ux0, uy0))
        self.ny, self.nx = phi0.shape
        self.precision = precision
        g = LbmGrid(self.nx, self.ny, int(prm.get("periodic_x", 1)), int(prm.get("periodic_y", 1)),
                    PRECISIONS[precision])
        self.params = make_params(prm)
        h = C.c_void_p()
        st = self._lib.lbm_create(C.byref(g), C.byref(self.params), _ptr(phi0), _ptr(p0), _ptr(ux0),
                                  _ptr(uy0), C.c_void_p(current_stream() if stream is None else stream),
                                  C.byref(h))
        if st != 0:
            raise LbmError(st, self._lib.lbm_last_error(None).decode())
        self._h = h

    def _ck(self, st):
        if st != 0:
            raise LbmError(st, self._lib.lbm_last_error(self._h).decode())

    def step(self, n=1):
        self._ck(self._lib.lbm_step(self._h, int(n)))

    def step_ch(self, ux, uy, n=1, tfac=None):
        """n steps of the Cahn-Hilliard part alone under the prescribed velocity
        tfac[k] * (ux, uy) at step k (tfac None: 1)."""
        ux, uy = _f64(ux), _f64(uy)
        tf = None if tfac is None else _f64(np.asarray(tfac, dtype=np.float64).ravel())
        if tf is not None and tf.size < n:
            raise ValueError("tfac needs one factor per step")
        self._ck(self._lib.lbm_step_ch(self._h, int(n), _ptr(ux), _ptr(uy), None if tf is None else _ptr(tf)))

    def fields(self, out=None):
        """(phi, p, ux, uy) as host float64 [ny, nx] arrays; out: four caller-owned
        contiguous float64 arrays to fill (page-locked ones copy fastest)."""
        shp = (self.ny, self.nx)
        if out is None:
            out = [np.empty(shp) for _ in range(4)]
        elif len(out) != 4 or any(a.dtype != np.float64 or a.shape != shp or not a.flags.c_contiguous for a in out):
            raise ValueError("out must be four contiguous float64 arrays of shape (ny, nx)")
        self._ck(self._lib.lbm_fields(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def dynamic_pressure(self, out=None):
        """p' = rho(phi) p as a host float64 [ny, nx] array (out: a caller-owned
        contiguous float64 array to fill)."""
        shp = (self.ny, self.nx)
        if out is None:
            out = np.empty(shp)
        elif out.dtype != np.float64 or out.shape != shp or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of shape (ny, nx)")
        self._ck(self._lib.lbm_dynamic_pressure(self._h, _ptr(out)))
        return out

    def fields_device(self, phi, p, ux, uy):
        """Copy into caller-owned device tensors (dtype of the handle's arithmetic)."""
        import torch
        dt = 0 if phi.dtype == torch.float64 else 1
        ptrs = [None if t is None else C.c_void_p(t.data_ptr()) for t in (phi, p, ux, uy)]
        self._ck(self._lib.lbm_fields_device(self._h, *ptrs, dt))

    def set_fields(self, phi0, p0, ux0, uy0):
        arrs = [_f64(a) for a in (phi0, p0, ux0, uy0)]
        self._ck(self._lib.lbm_set_fields(self._h, *[_ptr(a) for a in arrs]))

    def diagnostics(self, out=None):
        o = np.empty(LBM_NDIAG) if out is None else out
        self._ck(self._lib.lbm_diagnostics(self._h, _ptr(o)))
        return o

    def diagnostics_async(self, out):
        """Enqueue the sums into out (a page-locked float64 array of LBM_NDIAG,
        e.g. a pinned torch tensor's .numpy()); valid once the stream has passed."""
        if out.dtype != np.float64 or out.size < LBM_NDIAG or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of LBM_NDIAG values")
        self._ck(self._lib.lbm_diagnostics_async(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def check(self, delta=0.05):
        return self._lib.lbm_check(self._h, C.c_double(delta))

    def set_check(self, every, delta=0.05):
        """Let step() check the sums every `every` steps without waiting (0: off)."""
        self._ck(self._lib.lbm_set_check(self._h, int(every), C.c_double(delta)))

    def state(self):
        shp = (self.ny, self.nx)
        f = np.empty((9,) + shp); g = np.empty((9,) + shp)
        rest = [np.empty(shp) for _ in range(8)]
        self._ck(self._lib.lbm_get_state(self._h, _ptr(f), _ptr(g), *[_ptr(a) for a in rest]))
        keys = ("phi", "p", "ux", "uy", "uhx", "uhy", "upx", "upy")
        d = dict(zip(keys, rest))
        d["f"], d["g"] = f, g
        return d

    def set_state(self, f, g, phi, p, ux, uy, uhx, uhy, upx, upy):
        arrs = [_f64(a) for a in (f, g, phi, p, ux, uy, uhx, uhy, upx, upy)]
        self._ck(self._lib.lbm_set_state(self._h, *[_ptr(a) for a in arrs]))

    def profile(self, on=True):
        """Start (clearing totals) or stop per-kernel device timing."""
        self._ck(self._lib.lbm_profile(self._h, 1 if on else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since profiling started."""
        ms = np.zeros(LBM_NKERNELS)
        n = (C.c_longlong * LBM_NKERNELS)()
        self._ck(self._lib.lbm_profile_read(self._h, _ptr(ms), n))
        return {self._lib.lbm_kernel_name(k).decode(): (float(ms[k]), int(n[k]))
                for k in range(LBM_NKERNELS)}

    def kernel_variants(self):
        """{kernel kind name: name of the kernel this handle launches for it}."""
        return {self._lib.lbm_kernel_name(k).decode(): self._lib.lbm_kernel_variant(self._h, k).decode()
                for k in range(LBM_NKERNELS)}

    def adjoint_begin(self, nsteps, checkpoint_every):
        """Advance nsteps keeping checkpoints for the reverse sweep."""
        self._ck(self._lib.lbm_adjoint_begin(self._h, int(nsteps), int(checkpoint_every)))

    def adjoint_end(self, dL_dphi):
        """Reverse sweep: (dL/dphi0 [ny, nx], dL/dsigma, dL/dM) for the seed dL/dphi_final."""
        seed = _f64(dL_dphi)
        g = np.empty((self.ny, self.nx))
        ds = C.c_double(); dm = C.c_double()
        self._ck(self._lib.lbm_adjoint_end(self._h, _ptr(seed), _ptr(g), C.byref(ds), C.byref(dm)))
        return g, ds.value, dm.value

    def adjoint_engine(self):
        """1: the last reverse sweep ran compiled level kernels; 0: the tape interpreter; -1: none yet."""
        return int(self._lib.lbm_adjoint_engine(self._h))

    def device_bytes(self):
        return int(self._lib.lbm_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
