"""FP64 PyTorch-CPU restatement of one lattice step, for the adjoint -- TEST INFRASTRUCTURE.

A second plain implementation of the step of lbm_oracle.c, written with
whole-array torch operations so that torch.autograd can differentiate it.
Walls (an axis that is not periodic) follow lbm_oracle.c: halfway bounce-back
for the populations, and for the stencils a ghost across a wall is the mirror
image about the halfway wall times the field's parity along that axis --
+1 for phi, p and the quantities even in the wall-normal coordinate, -1 for
u (no slip) and for the odd ones (the normal component of a gradient).  Its reverse-mode gradients are the oracle adjoint against
which the GPU adjoint is checked.  It is pinned to the C oracle (forward
fields equal to round-off) and to central finite differences of the C oracle
(gradients), both in tests/test_adjoint_oracle.py.  It follows the same
readings as lbm_oracle.c; every function names the passage it restates.

Arrays are torch.float64 tensors shaped [ny, nx] (populations [9, ny, nx]).
"""
import torch

CS2 = 1.0 / 3.0
# Sec. III.A Eq. (D2Q9) and the weights below it
CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
WQ = (4.0 / 9,) + (1.0 / 9,) * 4 + (1.0 / 36,) * 4
# Sec. III.A Eq. (D2Q9MRT)
MROWS = ((1, 1, 1, 1, 1, 1, 1, 1, 1),
         (-4, -1, -1, -1, -1, 2, 2, 2, 2),
         (4, -2, -2, -2, -2, 1, 1, 1, 1),
         (0, 1, 0, -1, 0, 1, -1, -1, 1),
         (0, -2, 0, 2, 0, 1, -1, -1, 1),
         (0, 0, 1, 0, -1, 1, 1, -1, -1),
         (0, 0, -2, 0, 2, 1, 1, -1, -1),
         (0, 1, -1, 1, -1, 0, 0, 0, 0),
         (0, 0, 0, 0, 0, 1, -1, 1, -1))
# App. B, SF-5/7/9/11
FILTERS = {5: (6 / 16, -4 / 16, 1 / 16), 7: (5 / 16, -15 / 64, 3 / 32, -1 / 64),
           9: (0.243527493120, -0.204788880640, 0.120007591680, -0.045211119360, 0.008228661760),
           11: (0.215044884112, -0.187772883589, 0.123755948787, -0.059227575576, 0.018721609157,
                -0.002999540835)}

DT = torch.float64
MMAT = torch.tensor(MROWS, dtype=DT)
MINV = torch.linalg.inv(MMAT)


# Which axes are periodic, set from the parameters by init_state() and step().
AXES = {"px": True, "py": True}
EVEN, ODD = (1.0, 1.0), (-1.0, -1.0)
OPP = tuple(next(r for r in range(9) if CX[r] == -CX[q] and CY[r] == -CY[q]) for q in range(9))


def set_axes(prm):
    AXES["px"] = bool(prm.get("periodic_x", 1))
    AXES["py"] = bool(prm.get("periodic_y", 1))


def _axis(n, d, periodic):
    """Source index of x + d along an axis of n nodes, and whether it crossed a wall."""
    i = torch.arange(n) + d
    if periodic:
        return i % n, torch.zeros(n, dtype=torch.bool)
    crossed = (i < 0) | (i >= n)
    return torch.where(i < 0, -1 - i, torch.where(i >= n, 2 * n - 1 - i, i)), crossed


def at(a, dx, dy, par=EVEN):
    """a(x + dx, y + dy): periodic axes wrap; across a wall the ghost is the
    mirror image about the halfway wall times par = (parity along x, along y)
    (a parity 0 makes the ghost zero)."""
    if AXES["px"] and AXES["py"]:
        return torch.roll(a, shifts=(-dy, -dx), dims=(-2, -1))
    ny, nx = a.shape[-2:]
    ix, cx = _axis(nx, dx, AXES["px"])
    iy, cy = _axis(ny, dy, AXES["py"])
    sx = torch.where(cx, torch.tensor(float(par[0]), dtype=DT), torch.tensor(1.0, dtype=DT))
    sy = torch.where(cy, torch.tensor(float(par[1]), dtype=DT), torch.tensor(1.0, dtype=DT))
    return a[..., iy, :][..., ix] * (sy[:, None] * sx[None, :])


def grad_iso(a, par=EVEN):
    """Isotropic gradient, Sec. III.B Eq. (dicretized)."""
    gx = sum(WQ[q] * CX[q] * at(a, CX[q], CY[q], par) for q in range(1, 9)) / CS2
    gy = sum(WQ[q] * CY[q] * at(a, CX[q], CY[q], par) for q in range(1, 9)) / CS2
    return gx, gy


def lap_iso(a, par=EVEN):
    """Isotropic Laplacian, Sec. III.B Eq. (dicretized)."""
    return sum(2.0 * WQ[q] * (at(a, CX[q], CY[q], par) - a) for q in range(1, 9)) / CS2


def d1(a, axis, par=EVEN):
    """Fourth-order central first derivative, Sec. III.A Eq. (fourOrder_FDM)."""
    s = (lambda k: at(a, k, 0, par)) if axis == 0 else (lambda k: at(a, 0, k, par))
    return (s(-2) - 8.0 * s(-1) + 8.0 * s(1) - s(2)) / 12.0


def d2(a, axis, par=EVEN):
    """Five-point fourth-order second derivative."""
    s = (lambda k: at(a, k, 0, par)) if axis == 0 else (lambda k: at(a, 0, k, par))
    return (-s(-2) + 16.0 * s(-1) - 30.0 * a + 16.0 * s(1) - s(2)) / 12.0


def selective_filter(a, order, alpha, par=EVEN):
    """Explicit selective filter, Sec. III.B Eq. (filter), App. B."""
    if not order:
        return a
    d = FILTERS[order]
    acc = 2.0 * d[0] * a
    for m in range(1, len(d)):
        acc = acc + d[m] * (at(a, m, 0, par) + at(a, -m, 0, par) + at(a, 0, m, par) + at(a, 0, -m, par))
    return a - alpha * acc


def coefficients(prm, sigma, M):
    """kappa, beta (Sec. II.A) and 1/tau_f (Eq. mobility) as tensors of sigma, M."""
    kappa = 3.0 * sigma * prm["W"] / 8.0
    beta = 3.0 * sigma / (4.0 * prm["W"])
    stau = 1.0 / (0.5 + M / (prm["eta"] * CS2))
    return kappa, beta, stau


def chem(phi, kappa, beta):
    """Chemical potential, Sec. II.A Eq. (chemical), isotropic Laplacian."""
    return 4.0 * beta * (phi ** 3 - phi) - kappa * lap_iso(phi)


def rho_nu(prm, phi):
    """Density and kinematic viscosity, Eqs. (rho), (dynamic_vis); phi clamped here only."""
    c = torch.clamp(phi, -1.0, 1.0)
    rho = prm["rho_H"] * (1 + c) / 2 + prm["rho_L"] * (1 - c) / 2
    mu = prm["rho_H"] * prm["nu_H"] * (1 + c) / 2 + prm["rho_L"] * prm["nu_L"] * (1 - c) / 2
    return rho, mu / rho


def u_independent_forces(prm, phi, p, kappa, beta, M):
    """rho, nu, grad rho, J = (d rho/d phi) M grad mu, F_s, grad p, mu (Sec. II.B)."""
    drho = (prm["rho_H"] - prm["rho_L"]) / 2.0
    rho, nu = rho_nu(prm, phi)
    mu = chem(phi, kappa, beta)
    gx, gy = grad_iso(phi)
    txx, txy, tyy = gx * gx + gy * gy - gx * gx, -gx * gy, gx * gx + gy * gy - gy * gy
    dtxx, _ = grad_iso(txx)
    dtxy_x, dtxy_y = grad_iso(txy, ODD)   # -gx gy: odd along both axes
    _, dtyy = grad_iso(tyy)
    fsx, fsy = kappa * (dtxx + dtxy_y), kappa * (dtxy_x + dtyy)
    mx, my = grad_iso(mu)
    gpx, gpy = grad_iso(p)
    return dict(rho=rho, nu=nu, mu=mu, grx=drho * gx, gry=drho * gy, Jx=drho * M * mx, Jy=drho * M * my,
                Fsx=fsx, Fsy=fsy, gpx=gpx, gpy=gpy)


def total_force(prm, F, p, ux, uy):
    """F = F_p + F_s + F_nu + F_m + F_g of Sec. II.B Eq. (reformNS), F_g = (rho - rho_ref) g."""
    dxux, dyux = grad_iso(ux, ODD)
    dxuy, dyuy = grad_iso(uy, ODD)
    sxx, sxy, syy = 2 * dxux, dyux + dxuy, 2 * dyuy
    g_rel = F["rho"] - prm.get("g_rho_ref", 0.0)
    fx = (-p * F["grx"] + F["Fsx"] + F["nu"] * (sxx * F["grx"] + sxy * F["gry"])
          + (F["Jx"] * dxux + F["Jy"] * dyux) + g_rel * prm.get("gx", 0.0))
    fy = (-p * F["gry"] + F["Fsy"] + F["nu"] * (sxy * F["grx"] + syy * F["gry"])
          + (F["Jx"] * dxuy + F["Jy"] * dyuy) + g_rel * prm.get("gy", 0.0))
    return fx, fy, (dxux, dyux, dxuy, dyuy)


def feq(phi, mu, ux, uy, eta):
    """CH equilibrium, Sec. III.A Eq. (feq_CH), stacked [9, ny, nx]."""
    u2 = ux * ux + uy * uy
    out = []
    for q in range(9):
        cu = CX[q] * ux + CY[q] * uy
        if q == 0:
            out.append(phi + (WQ[0] - 1.0) * eta * mu - WQ[0] * phi * u2 / (2 * CS2))
        else:
            out.append(WQ[q] * eta * mu + WQ[q] * phi * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - u2 / (2 * CS2)))
    return torch.stack(out)


def geq(p, ux, uy):
    """NS equilibrium, Sec. III.B Eq. (geq)."""
    u2 = ux * ux + uy * uy
    out = []
    for q in range(9):
        cu = CX[q] * ux + CY[q] * uy
        out.append(WQ[q] * (p / CS2 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - u2 / (2 * CS2)))
    return torch.stack(out)


def src_ch(phi, ax, ay):
    """CH source, Sec. III.A Eq. (Fi)."""
    return torch.stack([WQ[q] * phi * (CX[q] * ax + CY[q] * ay) / CS2 for q in range(9)])


def src_ns(rho, fx, fy, ux, uy, dpx, dpy):
    """NS source, Sec. III.B Eq. (Gi) with u(F/rho - grad p)."""
    bx, by = fx / rho - dpx, fy / rho - dpy
    out = []
    for q in range(9):
        c = (CX[q], CY[q])
        u = (ux, uy)
        b = (bx, by)
        second = 0
        for a in range(2):
            for k in range(2):
                second = second + u[a] * b[k] * (c[a] * c[k] - (CS2 if a == k else 0.0))
        out.append(WQ[q] * ((CX[q] * fx + CY[q] * fy) / (rho * CS2) + second / (CS2 * CS2)))
    return torch.stack(out)


def mom(x):
    return torch.einsum("kq,q...->k...", MMAT, x)


def unmom(m):
    return torch.einsum("qk,k...->q...", MINV, m)


def stream(fs):
    """Pull streaming f_i(x) = f*_i(x - c_i); a source across a wall returns
    the node's own opposite population (halfway bounce-back)."""
    if AXES["px"] and AXES["py"]:
        return torch.stack([at(fs[q], -CX[q], -CY[q]) for q in range(9)])
    ny, nx = fs.shape[-2:]
    out = []
    for q in range(9):
        _, cx = _axis(nx, -CX[q], AXES["px"])
        _, cy = _axis(ny, -CY[q], AXES["py"])
        crossed = (cy[:, None] | cx[None, :]).to(DT)
        out.append(at(fs[q], -CX[q], -CY[q], (0.0, 0.0)) + crossed * fs[OPP[q]])
    return torch.stack(out)


def fd_rhs(prm, psi, kappa, beta, M):
    """L(psi) = div(lambda J_phi + q), Sec. II.A Eq. (step2) with Eq. (fourOrder_FDM)."""
    gx, gy = d1(psi, 0), d1(psi, 1)
    mu = 4.0 * beta * (psi ** 3 - psi) - kappa * (d2(psi, 0) + d2(psi, 1))
    mag = torch.sqrt(gx * gx + gy * gy + prm["grad_eps"] ** 2)
    nx, ny = gx / mag, gy / mag
    jphi = mag - 2.0 * (1.0 - psi * psi) / prm["W"]
    jx, jy = prm["lambda"] * jphi * nx, prm["lambda"] * jphi * ny
    if prm.get("flux_correction", 1):
        dmn = d1(mu, 0) * nx + d1(mu, 1) * ny
        jx = jx - M * dmn * nx
        jy = jy - M * dmn * ny
    # J_x is odd along x and even along y, J_y the reverse
    return d1(jx, 0, (-1.0, 1.0)) + d1(jy, 1, (1.0, -1.0))


def init_state(prm, phi0, p0, ux0, uy0, sigma, M):
    """f = f_eq(phi0, mu(phi0), u0), g = g_eq(p0, u0) (initial populations)."""
    set_axes(prm)
    kappa, beta, _ = coefficients(prm, sigma, M)
    mu = chem(phi0, kappa, beta)
    return dict(f=feq(phi0, mu, ux0, uy0, prm["eta"]), g=geq(p0, ux0, uy0), phi=phi0, p=p0,
                ux=ux0, uy=uy0, uhx=ux0, uhy=uy0, upx=ux0, upy=uy0)


def step(prm, s, sigma, M):
    """One time step in the order of lbm_oracle.c: fields at t^n, collision,
    streaming, moments, TVD-RK3 correction, Picard sweeps, filter."""
    set_axes(prm)
    kappa, beta, stau = coefficients(prm, sigma, M)
    F = u_independent_forces(prm, s["phi"], s["p"], kappa, beta, M)
    fx, fy, (dxux, dyux, dxuy, dyuy) = total_force(prm, F, s["p"], s["ux"], s["uy"])
    ux, uy = s["ux"], s["uy"]
    ax = (ux - s["upx"]) + ux * dxux + uy * dyux
    ay = (uy - s["upy"]) + ux * dxuy + uy * dyuy
    # CH collision, Sec. III.A Eqs. (distribution_CH), (collison)
    sf = [torch.as_tensor(v, dtype=DT) for v in prm["s_f"]]
    sf[3] = stau
    sf[5] = stau
    m = mom(s["f"])
    meq = mom(feq(s["phi"], F["mu"], ux, uy, prm["eta"]))
    mF = mom(src_ch(s["phi"], ax, ay))
    ms = torch.stack([m[k] - sf[k] * (m[k] - meq[k]) + (1 - 0.5 * sf[k]) * mF[k] for k in range(9)])
    fstar = unmom(ms)
    # NS collision, Sec. III.B Eq. (distribution_NS), filtered equilibrium
    phat_old = CS2 * s["g"].sum(0)
    tau_g = F["nu"] / CS2 + 0.5
    sg = [torch.full_like(tau_g, v) for v in prm["s_g"]]
    sg[7] = 1.0 / tau_g
    sg[8] = 1.0 / tau_g
    mg = mom(s["g"])
    mef = mom(geq(s["p"], ux, uy))
    meh = mom(geq(phat_old, s["uhx"], s["uhy"]))
    mG = mom(src_ns(F["rho"], fx, fy, ux, uy, F["gpx"], F["gpy"]))
    mgs = torch.stack([mef[k] + (1 - sg[k]) * (mg[k] - meh[k]) + (1 - 0.5 * sg[k]) * mG[k] for k in range(9)])
    gstar = unmom(mgs)
    f = stream(fstar)
    g = stream(gstar)
    phibar = f.sum(0)
    phat = CS2 * g.sum(0)
    jx = sum(CX[q] * g[q] for q in range(9))
    jy = sum(CY[q] * g[q] for q in range(9))
    # TVD-RK3, Sec. III.A Eq. (TVD-3order)
    p1 = phibar + fd_rhs(prm, phibar, kappa, beta, M)
    p2 = 0.75 * phibar + 0.25 * (p1 + fd_rhs(prm, p1, kappa, beta, M))
    phin = phibar / 3.0 + 2.0 / 3.0 * (p2 + fd_rhs(prm, p2, kappa, beta, M))
    # implicit velocity by Picard sweeps, Sec. III.B Eq. (u)
    Fn = u_independent_forces(prm, phin, phat, kappa, beta, M)
    ukx, uky = ux, uy
    for _ in range(prm["picard_iters"]):
        fx, fy, _ = total_force(prm, Fn, phat, ukx, uky)
        ukx, uky = jx + fx / (2.0 * Fn["rho"]), jy + fy / (2.0 * Fn["rho"])
    # selective filter, Sec. III.B Eq. (filter)
    fo, fa = prm["filter_order"], prm["filter_a"]
    return dict(f=f, g=g, phi=phin, p=selective_filter(phat, fo, fa),
                ux=selective_filter(ukx, fo, fa, ODD), uy=selective_filter(uky, fo, fa, ODD),
                uhx=ukx, uhy=uky, upx=ux, upy=uy)


def run(prm, phi0, p0, ux0, uy0, sigma, M, steps):
    s = init_state(prm, phi0, p0, ux0, uy0, sigma, M)
    for _ in range(steps):
        s = step(prm, s, sigma, M)
    return s
