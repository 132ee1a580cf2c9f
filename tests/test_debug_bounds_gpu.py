"""The FP32 kernels' shared-memory indexing, checked on the GPU.

liblbm_debug.so is the library built with LBM_DEBUG: every paired
shared-memory access of the FP32 kernels (the TMA windows and strips of the
collision, RK3 stages, Picard sweeps and filter, and the column-pair strip
kernels) is checked against the launch's dynamic shared memory, skipped if
outside and recorded.  Grids chosen to take every FP32 kernel variant and
every boundary case of the tiles -- ragged tiles, windows that wrap or
mirror, interior tiles beside edge tiles, every filter radius, bf16 words --
must record no access outside, and give the release library's fields."""
import os

import numpy as np
import pytest

from paper_1812_02459_gb300 import build, inputs, lbm

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, periodic x, periodic y, precision, extra parameters
    (64, 48, 1, 0, "fp32", {}),            # node-pair collide, TMA stencil passes, walls in y
    (300, 70, 0, 1, "fp32", {}),           # walls in x (one-node collide), interior and edge TMA tiles
    (392, 136, 1, 0, "fp32", {}),          # several interior tiles per row
    (46, 37, 1, 0, "fp32", {}),            # even width not a multiple of 4: column-pair strips
    (46, 38, 0, 0, "fp32", {"filter_order": 5, "picard_iters": 3}),
    (64, 48, 1, 0, "fp32", {"filter_order": 7}),
    (64, 48, 1, 0, "fp32", {"filter_order": 9}),
    (64, 48, 1, 0, "mix_bf16", {}),        # 16-bit words through the same kernels
    (12, 12, 1, 1, "fp32", {}),            # windows that wrap more than once
]


@pytest.mark.parametrize("nx,ny,px,py,precision,extra", CASES)
def test_no_shared_memory_access_out_of_bounds(nx, ny, px, py, precision, extra):
    assert os.path.exists(build.DEBUG_LIB), "liblbm_debug.so is built beside liblbm.so"
    Ld = lbm.load(path=build.DEBUG_LIB)
    assert Ld.lbm_debug_violations() == 0   # and cleared
    prm = inputs.base_params(rho_H=20.0, sigma=5e-3, gy=-2e-6 if py == 0 else 0.0, periodic_x=px,
                             periodic_y=py, **extra)
    R = max(min(nx, ny) / 4.0, 3.0)
    phi = inputs.drop(nx, ny, R, nx / 2 + 0.3, ny / 2 - 0.2, prm["W"])
    z = np.zeros_like(phi)
    fields = (phi, z, np.full_like(phi, 1e-3), z)
    d = lbm.Sim(prm, *fields, precision=precision, lib=Ld)
    r = lbm.Sim(prm, *fields, precision=precision)
    d.step(20)
    r.step(20)
    v = Ld.lbm_debug_violations()
    assert v == 0, f"shared-memory access out of bounds: block {v >> 32}, offset {(v & 0x7fffffff) - 1}"
    for a, b in zip(d.fields(), r.fields()):
        assert np.abs(a - b).max() <= 1e-6 * max(np.abs(b).max(), 1e-30)
    d.close()
    r.close()
