"""Planted mistakes in the FP64 oracle, against its CPU pins (test
infrastructure; runs on the CPU only).

Each entry of MISTAKES is a plausible slip in oracle/lbm_oracle.c: a dropped
term, a wrong sign, a transposed index, a swapped coefficient or parity. For
each one the script copies the repository into a scratch directory, plants
the slip in the copy's oracle, rebuilds it there, and runs the pins that
check the oracle against the paper and the mathematics (no GPU, no
comparison with the CUDA path). A slip counts as caught when a pin fails.

    python oracle/planted_mistakes.py [--workdir DIR] [--jobs N]

The repository itself is never modified. An anchor that no longer occurs
exactly once in the oracle is reported, so the list follows the source.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_ch_only.py", "tests/test_capillary_wave.py",
        "tests/test_fp32_floor.py"]

# (what the slip is, text in lbm_oracle.c, the slipped text)
MISTAKES = [
 ("feq rest: sign of (w0-1) eta mu", "out[i] = phi + (g_w[0] - 1.0) * eta * mu", "out[i] = phi + (g_w[0] + 1.0) * eta * mu"),
 ("feq: dropped (c.u)^2 term", "+ g_w[i] * phi * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - u2 / (2 * CS2));", "+ g_w[i] * phi * (cu / CS2 - u2 / (2 * CS2));"),
 ("geq: sign of c.u", "out[i] = g_w[i] * (p / CS2 + cu / CS2", "out[i] = g_w[i] * (p / CS2 - cu / CS2"),
 ("F_i: half", "out[i] = g_w[i] * phi * (g_c[2 * i] * ax + g_c[2 * i + 1] * ay) / CS2;", "out[i] = g_w[i] * phi * (g_c[2 * i] * ax + g_c[2 * i + 1] * ay) / CS2 * 0.5;"),
 ("F_i: ax, ay swapped", "out[i] = g_w[i] * phi * (g_c[2 * i] * ax + g_c[2 * i + 1] * ay) / CS2;", "out[i] = g_w[i] * phi * (g_c[2 * i] * ay + g_c[2 * i + 1] * ax) / CS2;"),
 ("G_i: b = F/rho + grad p", "double bx = Fx / rho - dpx, by = Fy / rho - dpy;", "double bx = Fx / rho + dpx, by = Fy / rho + dpy;"),
 ("G_i: first order without 1/rho", "double first = (c[0] * Fx + c[1] * Fy) / (rho * CS2);", "double first = (c[0] * Fx + c[1] * Fy) / (CS2);"),
 ("collide f: no (1 - s/2) on the source", "ms[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * mF[k];", "ms[k] = m[k] - s[k] * (m[k] - meq[k]) + mF[k];"),
 ("collide g: no (1 - s/2) on the source", "ms[k] = mf[k] + (1.0 - s[k]) * (m[k] - mh[k]) + (1.0 - 0.5 * s[k]) * mG[k];", "ms[k] = mf[k] + (1.0 - s[k]) * (m[k] - mh[k]) + mG[k];"),
 ("iso laplacian: half", "s += 2.0 * g_w[q] * (*PA(in, i + g_c[2 * q], j + g_c[2 * q + 1]) - c0) / CS2;", "s += g_w[q] * (*PA(in, i + g_c[2 * q], j + g_c[2 * q + 1]) - c0) / CS2;"),
 ("iso gradient: sign of y", "sy += g_w[q] * g_c[2 * q + 1] * v / CS2;", "sy -= g_w[q] * g_c[2 * q + 1] * v / CS2;"),
 ("FD4 gradient x: 7 for 8", "*PA(gx, i, j) = (*PA(in, i - 2, j) - 8.0 * *PA(in, i - 1, j)", "*PA(gx, i, j) = (*PA(in, i - 2, j) - 7.0 * *PA(in, i - 1, j)"),
 ("FD4 laplacian x: sign of outer tap", "double dxx = (-*PA(in, i - 2, j) + 16.0", "double dxx = (*PA(in, i - 2, j) + 16.0"),
 ("filter: + a s", "out[(size_t)j * nx + i] = *PA(&c, i, j) - a * s;", "out[(size_t)j * nx + i] = *PA(&c, i, j) + a * s;"),
 ("stream: wall returns same direction", "if (out_x || out_y) v = fstar[opp * N", "if (out_x || out_y) v = fstar[q * N"),
 ("FD mu: + kappa lap", "*PA(&mu, i, j) = 4.0 * beta * (v * v * v - v) - kappa * *PA(&lap, i, j);", "*PA(&mu, i, j) = 4.0 * beta * (v * v * v - v) + kappa * *PA(&lap, i, j);"),
 ("J_phi: factor 2 dropped", "double jphi = mag - 2.0 * (1.0 - v * v) / prm->W;", "double jphi = mag - (1.0 - v * v) / prm->W;"),
 ("q: sign in x", "jx += -prm->M * dmn * nxv;", "jx += prm->M * dmn * nxv;"),
 ("RK3: 3/4 and 1/4 swapped", "p2[k] = 0.75 * phibar[k] + 0.25 * (p1[k] + Lv[k]);", "p2[k] = 0.25 * phibar[k] + 0.75 * (p1[k] + Lv[k]);"),
 ("RK3: last stage 1/2, 1/2", "out[k] = phibar[k] / 3.0 + 2.0 / 3.0 * (p2[k] + Lv[k]);", "out[k] = phibar[k] / 2.0 + 1.0 / 2.0 * (p2[k] + Lv[k]);"),
 ("LBE mu: phi^3 + phi", "*PA(&MU, i, j) = 4.0 * s->beta * (v * v * v - v) - s->kappa * *PA(&lap, i, j);", "*PA(&MU, i, j) = 4.0 * s->beta * (v * v * v + v) - s->kappa * *PA(&lap, i, j);"),
 ("tensor: + a b", "*PA(&Txy, i, j) = -a * b;", "*PA(&Txy, i, j) = a * b;"),
 ("F_s: d_x Txy for d_y Txy", "F->Fsx[k] = s->kappa * (*PA(&dTxx_x, i, j) + *PA(&dTxy_y, i, j));", "F->Fsx[k] = s->kappa * (*PA(&dTxx_x, i, j) + *PA(&dTxy_x, i, j));"),
 ("J: without drho", "F->Jx[k] = drho * q->M * *PA(&gmx, i, j);", "F->Jx[k] = q->M * *PA(&gmx, i, j);"),
 ("F_p: sign", "double Fpx = -p[k] * F->grx[k], Fpy = -p[k] * F->gry[k];", "double Fpx = p[k] * F->grx[k], Fpy = p[k] * F->gry[k];"),
 ("F_nu: grx for gry", "double Fnx = F->nu[k] * (Sxx * F->grx[k] + Sxy * F->gry[k]);", "double Fnx = F->nu[k] * (Sxx * F->grx[k] + Sxy * F->grx[k]);"),
 ("F_m: transposed index", "double Fmx = F->Jx[k] * dxux[k] + F->Jy[k] * dyux[k];", "double Fmx = F->Jx[k] * dxux[k] + F->Jy[k] * dxuy[k];"),
 ("F_g: rho + rho_ref in y", "Fgy = (F->rho[k] - q->g_rho_ref) * q->gy;", "Fgy = (F->rho[k] + q->g_rho_ref) * q->gy;"),
 ("tau_g: nu without 1/cs2", "double tau_g = F.nu[k] / CS2 + 0.5;", "double tau_g = F.nu[k] + 0.5;"),
 ("Picard: F/rho for F/(2 rho)", "unx[k] = jx[k] + Fx / (2.0 * F.rho[k]);", "unx[k] = jx[k] + Fx / (F.rho[k]);"),
 ("p_hat without cs2", "phibar[k] = sp; phat[k] = CS2 * sgv;", "phibar[k] = sp; phat[k] = sgv;"),
 ("a: u.grad u transposed", "double ax = (ux - s->upx[k]) + ux * dxux[k] + uy * dyux[k];", "double ax = (ux - s->upx[k]) + ux * dxux[k] + uy * dxuy[k];"),
 ("a: u.grad u dropped", "double ay = (uy - s->upy[k]) + ux * dxuy[k] + uy * dyuy[k];", "double ay = (uy - s->upy[k]);"),
 ("rho(phi): densities swapped", "return p->rho_H * (1.0 + c) / 2.0 + p->rho_L * (1.0 - c) / 2.0;", "return p->rho_L * (1.0 + c) / 2.0 + p->rho_H * (1.0 - c) / 2.0;"),
 ("viscosity: nu_H and nu_L swapped", "return p->rho_H * p->nu_H * (1.0 + c) / 2.0 + p->rho_L * p->nu_L * (1.0 - c) / 2.0;", "return p->rho_H * p->nu_L * (1.0 + c) / 2.0 + p->rho_L * p->nu_H * (1.0 - c) / 2.0;"),
 ("u gradients even at walls", "orc_grad_iso(q->nx, q->ny, q->periodic_x, q->periodic_y, -1, ux, dxux, dyux);", "orc_grad_iso(q->nx, q->ny, q->periodic_x, q->periodic_y, +1, ux, dxux, dyux);"),
 ("filter of u_x even at walls", "orc_filter(nx, ny, q->periodic_x, q->periodic_y, -1, q->filter_order, q->filter_a, ukx, s->uxf);", "orc_filter(nx, ny, q->periodic_x, q->periodic_y, +1, q->filter_order, q->filter_a, ukx, s->uxf);"),
 ("c12: equilibrium part at (p_hat, u_hat)", "ms[k] = mf[k] + (1.0 - s[k]) * (m[k] - mh[k]) + (1.0 - 0.5 * s[k]) * mG[k];", "ms[k] = mh[k] + (1.0 - s[k]) * (m[k] - mh[k]) + (1.0 - 0.5 * s[k]) * mG[k];"),
]


def _copy(workdir, k):
    d = os.path.join(workdir, f"copy{k}")
    if os.path.exists(d):
        shutil.rmtree(d)
    shutil.copytree(ROOT, d, ignore=shutil.ignore_patterns(".git", "_work", "gpurun_out", "*.ncu-rep", "*.so"))
    return d


def _try(d, mistake, original):
    name, old, new = mistake
    if original.count(old) != 1:
        return name, None, "anchor missing"
    with open(os.path.join(d, "oracle", "lbm_oracle.c"), "w") as f:
        f.write(original.replace(old, new))
    subprocess.run([sys.executable, "oracle/build.py", "--force"], cwd=d, check=True, capture_output=True)
    # the anchor check of this list fails on any planted copy by construction
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-m", "not gpu", "-x", "-q", "-p", "no:cacheprovider",
                        "--deselect", "tests/test_oracle_pins.py::test_planted_mistake_anchors_present"],
                       cwd=d, capture_output=True, text=True)
    failed = [l for l in r.stdout.splitlines() if l.startswith("FAILED")]
    return name, r.returncode != 0, failed[0] if failed else ""


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workdir", default=None, help="scratch directory for the copies (default: a temporary one)")
    ap.add_argument("--jobs", type=int, default=4)
    a = ap.parse_args()
    workdir = a.workdir or tempfile.mkdtemp(prefix="planted_mistakes_")
    os.makedirs(workdir, exist_ok=True)
    with open(os.path.join(ROOT, "oracle", "lbm_oracle.c")) as f:
        original = f.read()
    copies = [_copy(workdir, k) for k in range(a.jobs)]
    lanes = [[m for i, m in enumerate(MISTAKES) if i % a.jobs == k] for k in range(a.jobs)]
    with ThreadPoolExecutor(a.jobs) as ex:
        results = [r for rs in ex.map(lambda k: [_try(copies[k], m, original) for m in lanes[k]], range(a.jobs))
                   for r in rs]
    caught = 0
    for name, hit, first in results:
        caught += bool(hit)
        tag = "CAUGHT  " if hit else ("MISSING " if hit is None else "SURVIVED")
        print(tag, name, "|", first[:100])
    print(f"{caught} of {len(results)} planted mistakes fail a pin")
    if not a.workdir:
        shutil.rmtree(workdir, ignore_errors=True)


if __name__ == "__main__":
    main()
