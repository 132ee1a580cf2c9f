"""The GPU discrete adjoint (lbm_adjoint_begin / lbm_adjoint_end) against the
FP64 oracle adjoint (torch autograd of oracle/torch_ref.py, itself pinned to
finite differences of the C oracle) and against central finite differences of
the GPU forward.  Loss: L = 1/2 sum (phi_T - phi_target)^2."""
import time

import numpy as np
import pytest
import torch

from oracle import torch_ref as tr
from paper_1812_02459_gb300 import inputs, lbm
from paper_1812_02459_gb300.autograd import LbmTrajectory

pytestmark = pytest.mark.gpu
T = lambda a: torch.tensor(a, dtype=torch.float64)


def case(n=20, R=5.0):
    prm, fields = inputs.translating_drop(n=n, R=R, U0=0.01)
    prm["sigma"] = 5e-3
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    target = np.tanh(2.0 * (R + 0.5 - np.hypot(xx - n / 2 - 0.7, yy - n / 2)) / prm["W"])
    return prm, fields, target


def gpu_grad(prm, fields, target, steps, every, precision, engine=1):
    s = lbm.Sim(prm, *fields, precision=precision)
    s.adjoint_begin(steps, every)
    phiT = s.fields()[0]
    g, ds, dm = s.adjoint_end(phiT - target)
    assert s.adjoint_engine() == engine   # 1: compiled level kernels, 0: tape interpreter
    loss = 0.5 * float(((phiT - target) ** 2).sum())
    s.close()
    return loss, g, ds, dm


def gpu_loss(prm, fields, target, steps, precision="fp64"):
    s = lbm.Sim(prm, *fields, precision=precision)
    s.step(steps)
    phiT = s.fields()[0]
    s.close()
    return 0.5 * float(((phiT - target) ** 2).sum())


def test_adjoint_fp64_matches_oracle_adjoint():
    prm, fields, target = case()
    steps = 7
    loss, g, ds, dm = gpu_grad(prm, fields, target, steps, 3, "fp64")   # 3 segments, ragged last
    phi0 = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi0, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    lt = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(lt, [phi0, sig, M])
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    assert np.abs(g - gphi.numpy()).max() <= 1e-10 * np.abs(gphi.numpy()).max()
    assert ds == pytest.approx(gs.item(), rel=1e-10)
    assert dm == pytest.approx(gm.item(), rel=1e-10)


def test_adjoint_fp64_matches_oracle_adjoint_32():
    """The adjoint workload's small instance: translating drop 32 x 32 (R = 4,
    U0 = 0.01, density ratio 100), 12 steps in checkpoint segments of 5, a
    seeded target from sigma and M perturbed by 50 % seeded normals."""
    prm, fields = inputs.translating_drop(n=32, R=4.0, U0=0.01)
    rng = np.random.default_rng(0)
    xi = rng.standard_normal(2)
    steps = 12
    tp = dict(prm, sigma=prm["sigma"] * (1 + 0.5 * xi[0]), M=prm["M"] * (1 + 0.5 * xi[1]))
    target = tr.run(tp, *(T(a) for a in fields), T(tp["sigma"]), T(tp["M"]), steps)["phi"].numpy()
    loss, g, ds, dm = gpu_grad(prm, fields, target, steps, 5, "fp64")
    phi0 = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi0, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    lt = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(lt, [phi0, sig, M])
    assert loss == pytest.approx(lt.item(), rel=1e-10)
    assert np.abs(g - gphi.numpy()).max() <= 1e-10 * np.abs(gphi.numpy()).max()
    assert ds == pytest.approx(gs.item(), rel=1e-10)
    assert dm == pytest.approx(gm.item(), rel=1e-10)


# Tape structures other than the default one: each compiles its own level
# kernels (the source depends on the flux correction, the number of Picard
# sweeps, the filter order); gravity adds terms to the force.
STRUCTURES = {
    "no_flux_correction": dict(flux_correction=0),
    "picard1_no_filter": dict(picard_iters=1, filter_order=0),
    "picard3_sf5": dict(picard_iters=3, filter_order=5),
    "sf7_gravity": dict(filter_order=7, gx=2e-6, gy=-3e-6, g_rho_ref=1.0),
}


@pytest.mark.parametrize("name", sorted(STRUCTURES))
def test_compiled_levels_other_tape_structures(name):
    """A 24 x 20 (non-square) drop carried by a uniform flow, 5 steps in
    checkpoint segments of 2: the compiled FP64 sweep against the oracle
    adjoint for each tape structure."""
    nx, ny, R = 24, 20, 5.0
    prm = inputs.base_params(M=0.1, sigma=5e-3, rho_H=100.0, rho_L=1.0, **STRUCTURES[name])
    phi0 = inputs.drop(nx, ny, R, nx / 2, ny / 2, prm["W"])
    fields = (phi0, np.zeros((ny, nx)), np.full((ny, nx), 0.01), np.zeros((ny, nx)))
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    target = np.tanh(2.0 * (R + 0.5 - np.hypot(xx - nx / 2 - 0.7, yy - ny / 2)) / prm["W"])
    steps = 5
    loss, g, ds, dm = gpu_grad(prm, fields, target, steps, 2, "fp64")
    phi = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    lt = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(lt, [phi, sig, M])
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    assert np.abs(g - gphi.numpy()).max() <= 1e-10 * np.abs(gphi.numpy()).max()
    assert ds == pytest.approx(gs.item(), rel=1e-10)
    assert dm == pytest.approx(gm.item(), rel=1e-10)


def test_adjoint_fp64_matches_gpu_finite_differences():
    prm, fields, target = case(n=24, R=6.0)
    steps = 10
    _, g, ds, dm = gpu_grad(prm, fields, target, steps, 4, "fp64")
    hs = 1e-4 * prm["sigma"]
    fd_s = (gpu_loss(dict(prm, sigma=prm["sigma"] + hs), fields, target, steps)
            - gpu_loss(dict(prm, sigma=prm["sigma"] - hs), fields, target, steps)) / (2 * hs)
    hm = 1e-4 * prm["M"]
    fd_m = (gpu_loss(dict(prm, M=prm["M"] + hm), fields, target, steps)
            - gpu_loss(dict(prm, M=prm["M"] - hm), fields, target, steps)) / (2 * hm)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(fields[0].shape) * (np.abs(fields[0]) < 0.95)
    he = 1e-5
    fp = list(fields); fm = list(fields)
    fp[0] = fields[0] + he * v
    fm[0] = fields[0] - he * v
    fd_v = (gpu_loss(prm, fp, target, steps) - gpu_loss(prm, fm, target, steps)) / (2 * he)
    assert ds == pytest.approx(fd_s, rel=1e-6)
    assert dm == pytest.approx(fd_m, rel=1e-6)
    assert float((g * v).sum()) == pytest.approx(fd_v, rel=1e-6)


def test_segments_in_several_batches(monkeypatch):
    """Segments of 3 steps reversed in batches of at most 2 steps (the path
    with a segment buffer, taken when the value planes of a whole segment do
    not fit): the same gradients as whole-segment batches -- the phi0
    gradient bit for bit, sigma and M up to the order of their FP64 atomic
    sums."""
    prm, fields, target = case()
    ref = gpu_grad(prm, fields, target, 7, 3, "fp64")
    monkeypatch.setenv("LBM_ADJOINT_BATCH", "2")
    got = gpu_grad(prm, fields, target, 7, 3, "fp64")
    assert got[0] == ref[0]
    assert np.array_equal(got[1], ref[1])
    assert got[2] == pytest.approx(ref[2], rel=1e-12)
    assert got[3] == pytest.approx(ref[3], rel=1e-12)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_interpreter_matches_compiled_levels(monkeypatch, precision, tol):
    """The tape interpreter (the fallback when run-time compilation is not
    available) and the compiled level kernels apply the same
    vector-Jacobian products; only the rounding order differs."""
    prm, fields, target = case()
    comp = gpu_grad(prm, fields, target, 7, 3, precision, engine=1)
    monkeypatch.setenv("LBM_ADJOINT_COMPILED", "0")
    interp = gpu_grad(prm, fields, target, 7, 3, precision, engine=0)
    assert interp[0] == comp[0]   # same forward trajectory
    assert np.abs(interp[1] - comp[1]).max() <= tol * np.abs(comp[1]).max()
    assert interp[2] == pytest.approx(comp[2], rel=tol)
    assert interp[3] == pytest.approx(comp[3], rel=tol)


def test_autograd_function_and_fp32():
    prm, fields, target = case()
    for precision, tol in (("fp64", 1e-10), ("fp32", 1e-3)):
        phi0 = T(fields[0]).requires_grad_(True)
        sig = T(prm["sigma"]).requires_grad_(True)
        M = T(prm["M"]).requires_grad_(True)
        phiT = LbmTrajectory.apply(phi0, sig, M, prm, fields[1], fields[2], fields[3], 6, 4, precision)
        loss = 0.5 * ((phiT - T(target)) ** 2).sum()
        loss.backward()
        if precision == "fp64":
            ref = (phi0.grad.clone(), sig.grad.item(), M.grad.item())
        else:
            assert np.abs(phi0.grad.numpy() - ref[0].numpy()).max() <= tol * np.abs(ref[0].numpy()).max()
            assert sig.grad.item() == pytest.approx(ref[1], rel=tol)
            assert M.grad.item() == pytest.approx(ref[2], rel=tol)


@pytest.mark.slow
def test_adjoint_translating_drop_256():
    """Drop in a uniform flow, 256^2, rho ratio 100, 500 steps, checkpoint
    every 22 steps.  The target is the final phi of an FP64 run with sigma and
    M perturbed by 5 % seeded normals.  The FP32 adjoint, seeded with the same
    residual as the FP64 one, must reproduce the FP64 gradients (its reverse
    sweep linearises about the FP32 trajectory)."""
    prm, fields = inputs.translating_drop(n=256, R=32.0, U0=0.01)
    rng = np.random.default_rng(0)
    xi = rng.standard_normal(2)
    tp = dict(prm, sigma=prm["sigma"] * (1 + 0.05 * xi[0]), M=prm["M"] * (1 + 0.05 * xi[1]))
    s = lbm.Sim(tp, *fields, precision="fp64")
    s.step(500)
    target = s.fields()[0]
    s.close()
    out = {}
    seed = None
    for precision in ("fp64", "fp32"):
        s = lbm.Sim(prm, *fields, precision=precision)
        torch.cuda.synchronize()
        t0 = time.time()
        s.adjoint_begin(500, 22)
        t1 = time.time()
        phiT = s.fields()[0]
        if seed is None:
            seed = phiT - target
        g, ds, dm = s.adjoint_end(seed)
        t2 = time.time()
        out[precision] = (g, ds, dm, phiT)
        s.close()
        print(precision, "dsigma", ds, "dM", dm, "forward s", round(t1 - t0, 3), "reverse s", round(t2 - t1, 3),
              "residual", float(np.abs(seed).max()), "traj diff", float(np.abs(phiT - out["fp64"][3]).max()))
    g64, ds64, dm64 = out["fp64"][:3]
    g32, ds32, dm32 = out["fp32"][:3]
    assert np.isfinite(g32).all()
    assert dm32 == pytest.approx(dm64, rel=1e-2)
    assert abs(ds32 - ds64) <= 1e-2 * (abs(ds64) + abs(dm64))
    assert np.abs(g32 - g64).max() <= 1e-2 * np.abs(g64).max()


def test_adjoint_fp32_against_finite_differences_256():
    """FP32 adjoint on the 256^2 translating drop (rho ratio 100, 500 steps,
    checkpoint every 22) against central differences of the FP64 forward
    (h = 1e-4 relative; the FP64 adjoint meets them to 1e-6).  The FP32
    reverse sweep is seeded with the FP64 residual phi_T - target: it then
    differentiates the FP64 loss, linearised about the FP32 trajectory.
    Measured: dL/dM within 1.1e-5 of the difference, dL/dsigma within 3.3e-5
    of |dL/dsigma| + |dL/dM| (8.7e-4 of itself: dL/dsigma is a small difference
    of large surface-tension terms, each rounded in FP32), and dL/dphi0 . v for
    a random direction v within 1.2e-4 (gated at 2e-4): the FP32 trajectory
    about which the sweep linearises departs from the FP64 one by 1.8e-5 in
    phi over the 500 steps, and the projection on a random direction sums
    gradient components of both signs.  Seeded with its own
    residual instead, the FP32 gradient differs by the FP32 trajectory's
    departure from the FP64 one relative to the residual (here 1.8e-5 against
    2.8e-4 after 500 steps: a few per cent), a floor of the FP32 forward, not
    of the reverse sweep."""
    n, steps = 256, 500
    prm, fields = inputs.translating_drop(n=n, R=n / 8.0, U0=0.01)
    rng = np.random.default_rng(0)
    xi = rng.standard_normal(2)
    tp = dict(prm, sigma=prm["sigma"] * (1 + 0.05 * xi[0]), M=prm["M"] * (1 + 0.05 * xi[1]))
    s = lbm.Sim(tp, *fields, precision="fp64")
    s.step(steps)
    target = s.fields()[0]
    s.close()
    hs, hm, he = 1e-4 * prm["sigma"], 1e-4 * prm["M"], 1e-5
    fd_s = (gpu_loss(dict(prm, sigma=prm["sigma"] + hs), fields, target, steps)
            - gpu_loss(dict(prm, sigma=prm["sigma"] - hs), fields, target, steps)) / (2 * hs)
    fd_m = (gpu_loss(dict(prm, M=prm["M"] + hm), fields, target, steps)
            - gpu_loss(dict(prm, M=prm["M"] - hm), fields, target, steps)) / (2 * hm)
    v = rng.standard_normal(fields[0].shape) * (np.abs(fields[0]) < 0.95)
    fp = list(fields); fm = list(fields)
    fp[0] = fields[0] + he * v
    fm[0] = fields[0] - he * v
    fd_v = (gpu_loss(prm, fp, target, steps) - gpu_loss(prm, fm, target, steps)) / (2 * he)
    seed = None
    res = {}
    for precision in ("fp64", "fp32"):
        s = lbm.Sim(prm, *fields, precision=precision)
        s.adjoint_begin(steps, 22)
        phiT = s.fields()[0]
        if seed is None:
            seed, phi64 = phiT - target, phiT
        res[precision] = s.adjoint_end(seed)
        if precision == "fp32":
            drift = float(np.abs(phiT - phi64).max())
        s.close()
    g, ds, dm = res["fp32"]
    gv = float((g * v).sum())
    scale = abs(fd_s) + abs(fd_m)
    print("fp32 adjoint vs fd: dsigma", abs(ds - fd_s) / abs(fd_s), "of scale", abs(ds - fd_s) / scale,
          "dM", abs(dm - fd_m) / abs(fd_m), "dphi0.v", abs(gv - fd_v) / abs(fd_v),
          "trajectory drift", drift, "residual", float(np.abs(seed).max()))
    g64, ds64, dm64 = res["fp64"]
    assert ds64 == pytest.approx(fd_s, rel=1e-5)
    assert dm64 == pytest.approx(fd_m, rel=1e-5)
    assert abs(ds - fd_s) <= 1e-4 * scale
    assert dm == pytest.approx(fd_m, rel=1e-4)
    assert gv == pytest.approx(fd_v, rel=2e-4)


def wall_case(px, py, nx=24, ny=20):
    """A wavy interface tilted by 35 degrees, crossing the walls y = -1/2,
    ny - 1/2 (and x = -1/2, nx - 1/2 when that axis is walled too), in a flow
    along x, with gravity: the stencils of the step read interface values
    through mirrored ghosts, and bounce-back acts on moving fluid."""
    prm = inputs.base_params(M=0.1, sigma=5e-3, rho_H=100.0, rho_L=1.0, gy=-1e-5, periodic_x=px, periodic_y=py)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(float)
    ang = np.deg2rad(35.0)
    d = (xx - 11.3) * np.cos(ang) + (yy - 9.6) * np.sin(ang) + np.sin(2 * np.pi * xx / nx)
    phi0 = np.tanh(2.0 * d / prm["W"])
    fields = (phi0, np.zeros((ny, nx)), np.full((ny, nx), 0.01), np.zeros((ny, nx)))
    target = np.tanh(2.0 * (d + 0.5) / prm["W"])
    return prm, fields, target


@pytest.mark.parametrize("px,py", [(1, 0), (0, 1), (0, 0)])
def test_adjoint_walls_fp64_matches_oracle_adjoint(px, py):
    """Walls: the FP64 adjoint (bounce-back masks and mirrored-ghost
    transposes in the compiled level kernels) against the oracle adjoint with
    walls, 5 steps in checkpoint segments of 2."""
    prm, fields, target = wall_case(px, py)
    steps = 5
    loss, g, ds, dm = gpu_grad(prm, fields, target, steps, 2, "fp64")
    phi = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    lt = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(lt, [phi, sig, M])
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    assert np.abs(g - gphi.numpy()).max() <= 1e-10 * np.abs(gphi.numpy()).max()
    assert ds == pytest.approx(gs.item(), rel=1e-10)
    assert dm == pytest.approx(gm.item(), rel=1e-10)


@pytest.mark.parametrize("px,py", [(1, 0), (0, 0)])
def test_adjoint_walls_fp64_matches_gpu_finite_differences(px, py):
    prm, fields, target = wall_case(px, py)
    steps = 10
    _, g, ds, dm = gpu_grad(prm, fields, target, steps, 4, "fp64")
    hs, hm, he = 1e-4 * prm["sigma"], 1e-4 * prm["M"], 1e-5
    fd_s = (gpu_loss(dict(prm, sigma=prm["sigma"] + hs), fields, target, steps)
            - gpu_loss(dict(prm, sigma=prm["sigma"] - hs), fields, target, steps)) / (2 * hs)
    fd_m = (gpu_loss(dict(prm, M=prm["M"] + hm), fields, target, steps)
            - gpu_loss(dict(prm, M=prm["M"] - hm), fields, target, steps)) / (2 * hm)
    v = np.random.default_rng(2).standard_normal(fields[0].shape) * (np.abs(fields[0]) < 0.95)
    fp = list(fields); fm = list(fields)
    fp[0] = fields[0] + he * v
    fm[0] = fields[0] - he * v
    fd_v = (gpu_loss(prm, fp, target, steps) - gpu_loss(prm, fm, target, steps)) / (2 * he)
    assert ds == pytest.approx(fd_s, rel=1e-6)
    assert dm == pytest.approx(fd_m, rel=1e-6)
    assert float((g * v).sum()) == pytest.approx(fd_v, rel=1e-6)


def test_adjoint_walls_capillary_wave_fp32():
    """The capillary wave (density ratio 1000, walls in y) through the FP32
    adjoint, 40 steps with checkpoints every 22 (64 x 64): the FP32 gradients
    against the FP64 ones seeded with the same residual (measured 2.4e-6 for
    dL/dphi0, below 1e-6 for sigma and M)."""
    prm, fields = inputs.capillary_wave(n=64)
    s = lbm.Sim(dict(prm, sigma=prm["sigma"] * 1.05), *fields, precision="fp64")
    s.step(40)
    target = s.fields()[0]
    s.close()
    seed = None
    res = {}
    for precision in ("fp64", "fp32"):
        s = lbm.Sim(prm, *fields, precision=precision)
        s.adjoint_begin(40, 22)
        phiT = s.fields()[0]
        if seed is None:
            seed = phiT - target
        res[precision] = s.adjoint_end(seed)
        assert s.adjoint_engine() == 1
        s.close()
    (g64, ds64, dm64), (g32, ds32, dm32) = res["fp64"], res["fp32"]
    print("capillary wave adjoint fp32 vs fp64: dphi0", np.abs(g32 - g64).max() / np.abs(g64).max(),
          "dsigma", abs(ds32 - ds64) / abs(ds64), "dM", abs(dm32 - dm64) / abs(dm64))
    assert np.isfinite(g32).all()
    assert np.abs(g32 - g64).max() <= 2e-5 * np.abs(g64).max()
    assert abs(ds32 - ds64) <= 2e-5 * (abs(ds64) + abs(dm64))
    assert abs(dm32 - dm64) <= 2e-5 * (abs(ds64) + abs(dm64))


def test_adjoint_walls_refused_by_the_interpreter(monkeypatch):
    prm, fields, target = wall_case(1, 0)
    monkeypatch.setenv("LBM_ADJOINT_COMPILED", "0")
    s = lbm.Sim(prm, *fields, precision="fp64")
    s.adjoint_begin(2, 2)
    with pytest.raises(lbm.LbmError) as e:
        s.adjoint_end(s.fields()[0] - target)
    assert e.value.status == 1 and "walls" in str(e.value)
    s.close()


@pytest.mark.parametrize("steps,every", [(1, 1), (3, 1), (2, 5)])
def test_adjoint_degenerate_segments(steps, every):
    """One step, a checkpoint at every step, and a segment longer than the
    run: the FP64 sweep against the oracle adjoint."""
    prm, fields, target = case()
    loss, g, ds, dm = gpu_grad(prm, fields, target, steps, every, "fp64")
    phi0 = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi0, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    lt = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(lt, [phi0, sig, M])
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    assert np.abs(g - gphi.numpy()).max() <= 1e-10 * np.abs(gphi.numpy()).max()
    assert ds == pytest.approx(gs.item(), rel=1e-10)
    assert dm == pytest.approx(gm.item(), rel=1e-10)
