"""torch.autograd.Function over the C ABI's discrete adjoint (argument marshalling only).

    phi_T = LbmTrajectory.apply(phi0, sigma, M, prm, p0, ux0, uy0, nsteps, every, precision)

phi0 (float64 tensor [ny, nx]), sigma and M (0-dim float64 tensors) are the
differentiable inputs; the forward runs nsteps lattice steps on the GPU
keeping a checkpoint every `every` steps (lbm_adjoint_begin), the backward
runs the hand-written reverse sweep (lbm_adjoint_end) and returns
dL/dphi0, dL/dsigma, dL/dM.  Tensors live on the host; the library moves
them.
"""
import numpy as np
import torch

from . import lbm


class LbmTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, sigma, M, prm, p0, ux0, uy0, nsteps, every, precision="fp32"):
        q = dict(prm)
        q["sigma"] = float(sigma)
        q["M"] = float(M)
        sim = lbm.Sim(q, phi0.detach().cpu().numpy(), np.asarray(p0), np.asarray(ux0), np.asarray(uy0),
                      precision=precision)
        sim.adjoint_begin(nsteps, every)
        phiT = sim.fields()[0]
        ctx.sim = sim
        return torch.from_numpy(phiT)

    @staticmethod
    def backward(ctx, grad_phiT):
        sim = ctx.sim
        g, ds, dm = sim.adjoint_end(grad_phiT.detach().cpu().numpy())
        sim.close()
        ctx.sim = None
        return (torch.from_numpy(g), torch.tensor(ds, dtype=torch.float64),
                torch.tensor(dm, dtype=torch.float64), None, None, None, None, None, None, None)
