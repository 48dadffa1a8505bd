"""End-to-end gradients of a wall loss with respect to the porous-wall parameters.

The paper's motivation (Section 1, Section 3.2) is end-to-end optimisation through the
differentiable "Disturbance Wall" boundary condition.  Here the gradient comes from the library's
hand-written discrete adjoint (fluid_adjoint_step), wrapped as a torch.autograd.Function:

  forward   phi -> run N RK3 steps with a frozen dt from U0 -> J = integrated wall heat flux;
            the state is checkpointed every K steps
  backward  lambda_N = dJ/dU_N; for each segment, last first: replay the segment from its
            checkpoint keeping every step's state and stage states, then apply the step adjoint
            from the last step back to the checkpoint, accumulating dJ/dphi

Memory: N / K checkpoints plus 3 K states of one segment.  All arithmetic runs in the CUDA
library; this module only orders the calls.
"""
import torch


class WallHeatLoss(torch.autograd.Function):
    """J(phi) = wall heat flux of face (axis, side) after `nsteps` steps from U0."""

    @staticmethod
    def forward(ctx, phi, solver, U0, nsteps, K, axis, side):
        if not solver.cfg.adjoint or solver.cfg.dt_fixed <= 0:
            raise ValueError("the solver needs adjoint=True and a frozen dt (dt_fixed > 0)")
        phi = phi.detach().contiguous()
        solver.set_wall_params(phi)
        U = U0.detach().clone()
        checkpoints = []
        for k in range(nsteps):
            if k % K == 0:
                checkpoints.append(U.clone())
            solver.step(U, 1)
        J = solver.wall_heat_loss(U, axis, side)
        ctx.solver, ctx.nsteps, ctx.K, ctx.axis, ctx.side = solver, nsteps, K, axis, side
        ctx.checkpoints = checkpoints
        ctx.UN = U
        ctx.phi = phi
        return J[0].clone()

    @staticmethod
    def backward(ctx, gJ):
        s = ctx.solver
        s.set_wall_params(ctx.phi)
        _, lam = s.wall_heat_loss(ctx.UN, ctx.axis, ctx.side, grad=True)
        lam.mul_(gJ)
        gphi = torch.zeros_like(ctx.phi)
        nseg = len(ctx.checkpoints)
        for seg in reversed(range(nseg)):
            first = seg * ctx.K
            count = min(ctx.K, ctx.nsteps - first)
            U = ctx.checkpoints[seg].clone()
            states = []
            for _ in range(count):
                Un = U.clone()
                U1, U2 = torch.zeros_like(U), torch.zeros_like(U)
                s.step_stages(U, U1, U2)
                states.append((Un, U1, U2))
            for Un, U1, U2 in reversed(states):
                s.adjoint_step(Un, lam, gphi, U1, U2)
        return gphi, None, None, None, None, None, None


def wall_heat_loss(phi, solver, U0, nsteps, K=20, axis=1, side=0):
    return WallHeatLoss.apply(phi, solver, U0, nsteps, K, axis, side)
