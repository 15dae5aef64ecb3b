"""torch.autograd.Function around the discrete adjoint of the C ABI.

FluxObjective.apply(amp, gshift, sim, phi, gbody, n_init, nsteps, ckpt_every, axis, plane) returns
the flux through a plane averaged over nsteps DD-TR steps started from the rest state of the
densities n_init [M][N], as a function of the wall-potential amplitude amp [N] (V += amp * phi for
every species, with the wall shape phi [N]) and a body force gshift [3] added to every species' base
body force gbody [M][3].  sim is an lbe.Simulation with its geometry, species and potentials set.
The forward pass runs lbe_adjoint_flux_gradient once (forward sweep with checkpoints plus the
reverse sweep) and keeps the gradients; backward scales them by the incoming gradient.
"""
import numpy as np
import torch

from . import lbe


class FluxObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amp, gshift, sim, phi, gbody, n_init, nsteps, ckpt_every, axis, plane):
        a = amp.detach().to("cpu", torch.float64).numpy().reshape(-1)
        gs = gshift.detach().to("cpu", torch.float64).numpy().reshape(3)
        sim.set_wall_potential(phi, a)
        for s in range(sim.M):
            sim.set_body_force(s, np.asarray(gbody[s], dtype=np.float64) + gs)
        for s in range(sim.M):
            sim.init_density(s, n_init[s])
        Phi, dA, dG = sim.adjoint_flux_gradient(nsteps, ckpt_every, axis, plane)
        ctx.save_for_backward(torch.from_numpy(dA).to(amp.device, amp.dtype),
                              torch.from_numpy(dG).to(gshift.device, gshift.dtype))
        return torch.tensor(Phi, dtype=amp.dtype, device=amp.device)

    @staticmethod
    def backward(ctx, grad_out):
        dA, dG = ctx.saved_tensors
        return grad_out * dA, grad_out * dG, None, None, None, None, None, None, None, None
