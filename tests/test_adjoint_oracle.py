"""The FP64 oracle adjoint (torch autograd of oracle/torch_ref.py) pinned to
the C oracle: its forward equals lbm_oracle.c to round-off, and its
reverse-mode gradients equal central finite differences of lbm_oracle.c (an
independent implementation), for sigma, M and a direction in phi0."""
import numpy as np
import pytest
import torch

import oracle
from oracle import torch_ref as tr
from paper_1812_02459_gb300 import inputs

T = lambda a: torch.tensor(a, dtype=torch.float64)


def drop_case(n=20, steps=6):
    prm, (phi, p, ux, uy) = inputs.translating_drop(n=n, R=5.0, U0=0.01)
    prm["sigma"] = 5e-3
    rng = np.random.default_rng(0)
    target = np.tanh(2.0 * (5.5 - np.hypot(*np.meshgrid(np.arange(n) - n / 2 - 0.7, np.arange(n) - n / 2)))
                     / prm["W"])
    return prm, (phi, p, ux, uy), steps, target, rng


def c_loss(prm, fields, steps, target, sigma=None, M=None, phi0=None):
    q = dict(prm)
    if sigma is not None:
        q["sigma"] = sigma
    if M is not None:
        q["M"] = M
    f = list(fields)
    if phi0 is not None:
        f[0] = phi0
    s = oracle.Sim(q, *f)
    s.step(steps)
    return 0.5 * float(((s.fields()[0] - target) ** 2).sum())


def test_torch_forward_equals_c_oracle():
    prm, fields, steps, _, _ = drop_case()
    s = oracle.Sim(prm, *fields)
    s.step(steps)
    r = tr.run(prm, *(T(a) for a in fields), T(prm["sigma"]), T(prm["M"]), steps)
    for a, b in zip(s.fields(), (r["phi"], r["p"], r["ux"], r["uy"])):
        assert np.abs(a - b.numpy()).max() <= 1e-12 * max(np.abs(a).max(), 1e-30)


def test_torch_adjoint_matches_c_oracle_finite_differences():
    prm, fields, steps, target, rng = drop_case()
    phi0 = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi0, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    loss = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(loss, [phi0, sig, M])
    # central differences of the independent C oracle
    hs = 1e-4 * prm["sigma"]
    fd_s = (c_loss(prm, fields, steps, target, sigma=prm["sigma"] + hs)
            - c_loss(prm, fields, steps, target, sigma=prm["sigma"] - hs)) / (2 * hs)
    hm = 1e-4 * prm["M"]
    fd_m = (c_loss(prm, fields, steps, target, M=prm["M"] + hm)
            - c_loss(prm, fields, steps, target, M=prm["M"] - hm)) / (2 * hm)
    # a direction inside the interface only: a perturbation of the bulk
    # (phi0 = -1 + 1e-9) would cross the kink of the clamp in rho(phi)
    v = rng.standard_normal(fields[0].shape) * (np.abs(fields[0]) < 0.95)
    he = 1e-5
    fd_v = (c_loss(prm, fields, steps, target, phi0=fields[0] + he * v)
            - c_loss(prm, fields, steps, target, phi0=fields[0] - he * v)) / (2 * he)
    assert gs.item() == pytest.approx(fd_s, rel=1e-6)
    assert gm.item() == pytest.approx(fd_m, rel=1e-6)
    assert float((gphi.numpy() * v).sum()) == pytest.approx(fd_v, rel=1e-6)


def test_torch_adjoint_every_component_on_a_small_grid():
    """Brute force on a 12 x 12 grid: every component of dL/dphi0 from the
    oracle adjoint against a central difference of the C oracle at that node
    (all nodes lie strictly inside (-1, 1), away from the clamp's kink)."""
    n, steps = 12, 3
    prm, (phi, p, ux, uy) = inputs.translating_drop(n=n, R=3.0, U0=0.01)
    prm["sigma"] = 5e-3
    fields = (phi, p, ux, uy)
    assert np.abs(phi).max() < 0.999
    target = np.roll(phi, 1, axis=1)
    phi0 = T(phi).requires_grad_(True)
    r = tr.run(prm, phi0, T(p), T(ux), T(uy), T(prm["sigma"]), T(prm["M"]), steps)
    loss = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    (g,) = torch.autograd.grad(loss, [phi0])
    g = g.numpy()
    # where grad phi nearly vanishes the regularised normal
    # grad phi / sqrt(|grad phi|^2 + eps^2), eps = 1e-4, is strongly curved:
    # the central difference's O(he^2) error there is 8e-7 at he = 1e-5 and
    # 8e-9 at he = 1e-6, and rounding stays near 1e-10
    he = 1e-6
    fd = np.empty_like(phi)
    for j in range(n):
        for i in range(n):
            e = np.zeros_like(phi)
            e[j, i] = he
            fd[j, i] = (c_loss(prm, fields, steps, target, phi0=phi + e)
                        - c_loss(prm, fields, steps, target, phi0=phi - e)) / (2 * he)
    assert np.abs(fd - g).max() <= 1e-6 * np.abs(g).max()
    assert np.abs(g).max() > 0


@pytest.mark.parametrize("px,py", [(1, 0), (0, 0)])
def test_torch_walls_forward_and_adjoint_match_c_oracle(px, py):
    """Walls on one or both axes (halfway bounce-back, mirrored ghosts with
    each field's parity): the torch restatement's forward equals the C oracle
    to round-off, and its gradients equal central differences of the C oracle."""
    prm, fields, steps, target, rng = drop_case(n=20, steps=5)
    prm = dict(prm, periodic_x=px, periodic_y=py, gy=-1e-5)
    # the drop straddles the wall y = -1/2 (and x = -1/2): every stencil
    # reads interface values through the mirrored ghosts
    fields = (inputs.drop(20, 20, 6.0, 5.0, 3.0, prm["W"]),) + tuple(fields[1:])
    s = oracle.Sim(prm, *fields)
    s.step(steps)
    r = tr.run(prm, *(T(a) for a in fields), T(prm["sigma"]), T(prm["M"]), steps)
    for a, b in zip(s.fields(), (r["phi"], r["p"], r["ux"], r["uy"])):
        assert np.abs(a - b.numpy()).max() <= 1e-12 * max(np.abs(a).max(), 1e-30)
    phi0 = T(fields[0]).requires_grad_(True)
    sig = T(prm["sigma"]).requires_grad_(True)
    M = T(prm["M"]).requires_grad_(True)
    r = tr.run(prm, phi0, T(fields[1]), T(fields[2]), T(fields[3]), sig, M, steps)
    loss = 0.5 * ((r["phi"] - T(target)) ** 2).sum()
    gphi, gs, gm = torch.autograd.grad(loss, [phi0, sig, M])
    hs, hm, he = 1e-4 * prm["sigma"], 1e-4 * prm["M"], 1e-5
    fd_s = (c_loss(prm, fields, steps, target, sigma=prm["sigma"] + hs)
            - c_loss(prm, fields, steps, target, sigma=prm["sigma"] - hs)) / (2 * hs)
    fd_m = (c_loss(prm, fields, steps, target, M=prm["M"] + hm)
            - c_loss(prm, fields, steps, target, M=prm["M"] - hm)) / (2 * hm)
    v = rng.standard_normal(fields[0].shape) * (np.abs(fields[0]) < 0.95)
    fd_v = (c_loss(prm, fields, steps, target, phi0=fields[0] + he * v)
            - c_loss(prm, fields, steps, target, phi0=fields[0] - he * v)) / (2 * he)
    assert gs.item() == pytest.approx(fd_s, rel=1e-6)
    assert gm.item() == pytest.approx(fd_m, rel=1e-6)
    assert float((gphi.numpy() * v).sum()) == pytest.approx(fd_v, rel=1e-6)
