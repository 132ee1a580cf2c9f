"""The C ABI library: it loads, exports every declared entry point, its
struct layouts match the binding, and parameter validation (host logic, no
CUDA call) rejects what the paper's constraints exclude."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1812_02459_gb300 import inputs, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = lbm.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(lbm.EXPORTS)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in lbm.LbmParams._fields_]
    cf = {"lambda_": "lambda"}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(lbm_grid), sizeof(lbm_params));']
    for f in fields:
        lines.append(f'printf("%zu\\n", offsetof(lbm_params, {cf.get(f, f)}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(prog)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == C.sizeof(lbm.LbmGrid)
    assert int(out[1]) == C.sizeof(lbm.LbmParams)
    for f, off in zip(fields, out[2:]):
        assert int(off) == getattr(lbm.LbmParams, f).offset, f


@pytest.mark.parametrize("change,msg", [
    (dict(filter_order=6), "filter_order"),
    (dict(filter_a=1.5), "filter_a"),
    (dict(M=0.0), "tau_f"),
    (dict(rho_L=0.0), "densities"),
    (dict(nu_H=-1.0), "viscosities"),
    (dict(W=0.0), "W must"),
    (dict(picard_iters=0), "picard_iters"),
    (dict(picard_zeta=1e-3), "picard_zeta"),
    (dict(grad_eps=0.0), "grad_eps"),
    (dict(flags=2), "flags"),
])
def test_invalid_parameters_rejected(change, msg):
    prm, fields = inputs.static_drop(n=16, R=4.0)
    prm.update(change)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Sim(prm, *fields)
    assert e.value.status == 1 and msg in str(e.value)


@pytest.mark.parametrize("precision", ["mix_bf16", "mix_fp16"])
def test_strain_moments_flag_needs_full_precision(precision):
    prm, fields = inputs.static_drop(n=16, R=4.0)
    prm["flags"] = 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.Sim(prm, *fields, precision=precision)
    assert e.value.status == 1 and "STRAIN_MOMENTS" in str(e.value)


def test_invalid_rates_and_sizes_rejected():
    prm, fields = inputs.static_drop(n=16, R=4.0)
    prm["s_g"] = list(prm["s_g"])
    prm["s_g"][4] = 2.5
    with pytest.raises(lbm.LbmError) as e:
        lbm.Sim(prm, *fields)
    assert e.value.status == 1
    prm, fields = inputs.static_drop(n=8, R=2.0)
    with pytest.raises(lbm.LbmError) as e:
        lbm.Sim(prm, *fields)
    assert e.value.status == 1 and "12" in str(e.value)
    prm, fields = inputs.static_drop(n=16, R=4.0)
    with pytest.raises(KeyError):
        lbm.Sim(prm, *fields, precision="fp8")


def test_null_handle_rejected_without_cuda():
    """Every entry point given a NULL handle (or a NULL required pointer)
    returns LBM_ERR_ARG -- or -1 / nothing where that is its documented
    answer -- before any CUDA call, so this runs without a GPU."""
    L = lbm.load()
    ARG = 1
    d = np.zeros(lbm.LBM_NDIAG)
    pd = d.ctypes.data_as(C.POINTER(C.c_double))
    assert L.lbm_step(None, 1) == ARG
    assert L.lbm_step_ch(None, 1, pd, pd, None) == ARG
    assert L.lbm_set_check(None, 2, C.c_double(0.01)) == ARG
    assert L.lbm_diagnostics(None, pd) == ARG
    assert L.lbm_diagnostics_async(None, pd) == ARG
    assert L.lbm_check(None, C.c_double(0.01)) == ARG
    assert L.lbm_fields(None, pd, pd, pd, pd) == ARG
    assert L.lbm_dynamic_pressure(None, pd) == ARG
    assert L.lbm_set_fields(None, pd, pd, pd, pd) == ARG
    assert L.lbm_adjoint_begin(None, 4, 2) == ARG
    assert L.lbm_adjoint_end(None, pd, pd, pd, pd) == ARG
    assert L.lbm_adjoint_engine(None) == -1
    assert L.lbm_profile(None, 1) == ARG
    assert L.lbm_debug_violations() == 0   # release build: nothing is checked
    L.lbm_destroy(None)
    assert L.lbm_diagnostics_async(None, pd) == ARG
    assert L.lbm_last_error(None) == b"NULL handle"
