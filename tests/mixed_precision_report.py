"""Accuracy report of the reduced-precision population storage (not a test).

    python tests/mixed_precision_report.py [--oracle-steps 2000] [--steps 50000] [--out FILE]

Part A: rising bubble 256 x 512 (R = 32, density ratio 1000), advanced by
the FP64 oracle and by the GPU in fp64, fp32, mix_bf16 and mix_fp16 for the
same number of steps; errors of phi, of the bubble centroid and of the rise
velocity against the oracle.  Part B: the same bubble on 1024 x 2048
(R = 128) for 50000 steps on the GPU; mix_bf16 and mix_fp16 against fp32,
with the throughput of each.  Writes one JSON document.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1812_02459_gb300 import inputs, lbm  # noqa: E402


def centroid(d):
    """Indicator centroid, smooth (1-phi)/2 centroid, smooth rise velocity."""
    return {"yc_indicator": d[3] / d[2], "yc": d[6] / d[5], "vc": d[7] / d[5], "volume": d[0]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--oracle-steps", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--out", default=os.path.join(ROOT, "gpurun_out", "mixed_precision_report.json"))
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    rep = {"part_a": {}, "part_b": {}}

    prm, fields = inputs.rising_bubble()
    t0 = time.time()
    o = oracle.Sim(prm, *fields)
    o.step(a.oracle_steps)
    of = o.fields()
    oc = centroid(np.concatenate([o.diagnostics(), [0.0]]))
    rep["part_a"]["oracle"] = dict(oc, seconds=time.time() - t0, steps=a.oracle_steps)
    for prec in ("fp64", "fp32", "mix_bf16", "mix_fp16"):
        g = lbm.Sim(prm, *fields, precision=prec)
        g.step(a.oracle_steps)
        gf = g.fields()
        gc = centroid(g.diagnostics())
        errs = {n: float(np.abs(x - y).max() / max(np.abs(y).max(), 1e-300))
                for n, x, y in zip(("phi", "p", "ux", "uy"), gf, of)}
        rep["part_a"][prec] = dict(field_rel_err=errs, centroid=gc,
                                   yc_err=gc["yc"] - oc["yc"], vc_err=gc["vc"] - oc["vc"],
                                   yc_err_over_D=(gc["yc"] - oc["yc"]) / 64.0)
        print(prec, json.dumps(rep["part_a"][prec]), flush=True)
        g.close()

    prm, fields = inputs.rising_bubble_large()
    nx, ny = fields[0].shape[1], fields[0].shape[0]
    res = {}
    for prec in ("fp32", "mix_bf16", "mix_fp16"):
        g = lbm.Sim(prm, *fields, precision=prec)
        d0 = g.diagnostics()
        torch.cuda.synchronize()
        t = time.time()
        g.step(a.steps)
        torch.cuda.synchronize()
        dt = time.time() - t
        d = g.diagnostics()
        res[prec] = dict(centroid(d), seconds=dt, mlups=nx * ny * a.steps / dt / 1e6,
                         volume_drift=float(d[0] - d0[0]), phi_max=d[8], phi_min=d[9], nonfinite=d[10],
                         fields=g.fields())
        g.close()
    for prec, r in res.items():
        out = {k: v for k, v in r.items() if k != "fields"}
        if prec != "fp32":
            f32 = res["fp32"]
            out["yc_diff_vs_fp32"] = r["yc"] - f32["yc"]
            out["yc_diff_over_D"] = (r["yc"] - f32["yc"]) / 256.0
            out["vc_diff_vs_fp32"] = r["vc"] - f32["vc"]
            out["phi_max_abs_diff_vs_fp32"] = float(np.abs(r["fields"][0] - f32["fields"][0]).max())
            out["u_rel_diff_vs_fp32"] = float(max(np.abs(r["fields"][k] - f32["fields"][k]).max()
                                                  for k in (2, 3)) /
                                              max(np.abs(f32["fields"][k]).max() for k in (2, 3)))
        rep["part_b"][prec] = out
        print(prec, json.dumps(out), flush=True)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    json.dump(rep, open(a.out, "w"), indent=1, default=float)


if __name__ == "__main__":
    main()
