"""torch.autograd front end of the discrete adjoint.

``PFLRollout.apply(M, xi, sigma, setup)`` runs n steps of the PFLBM from the
set-up's initial state with the given mobility, interface width and surface
tension (0-d float64 tensors) and returns J = sum_o sum_x W_o(x) phi(x, t_o)
as a 0-d tensor.  The forward call runs the library's adjoint directly (its
forward sweep computes J and its reverse sweep the gradient in the same call,
with sqrt(n) checkpointing); backward scales that gradient by the incoming one.

``ObjectiveRollout.apply(M, xi, sigma, setup, objective)`` does the same for a
nonlinear objective of phi at chosen steps (``objectives.WaveFrequency``: the
fitted capillary-wave frequency): a forward run records phi at the
objective's steps, the objective gives J and its seed fields dJ / dphi(t_o),
and the library's adjoint of those seeds gives dJ / d(M, xi, sigma).
"""
import copy

import torch

from .pflbm import Simulation


class RolloutSetup:
    """Lattice, initial fields, step count and observations of one rollout."""

    def __init__(self, params, phi0, n_steps, observations, u0=None, p0=None, precision="fp32", device=None):
        self.params = params
        self.phi0, self.u0, self.p0 = phi0, u0, p0
        self.n_steps = int(n_steps)
        self.observations = observations
        self.precision = precision
        self.device = device


class PFLRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, xi, sigma, setup):
        p = copy.copy(setup.params)
        p.mobility, p.xi, p.sigma = float(M), float(xi), float(sigma)
        sim = Simulation(p, setup.phi0, setup.u0, setup.p0, precision=setup.precision, device=setup.device)
        J, grad = sim.adjoint(setup.n_steps, setup.observations)
        sim.close()
        g = torch.tensor(grad, dtype=torch.float64)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        gout = gout.to(torch.float64)
        return gout * g[0], gout * g[1], gout * g[2], None


def rollout(M, xi, sigma, setup):
    return PFLRollout.apply(M, xi, sigma, setup)


class ObjectiveRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, xi, sigma, setup, objective):
        p = copy.copy(setup.params)
        p.mobility, p.xi, p.sigma = float(M), float(xi), float(sigma)
        sim = Simulation(p, setup.phi0, setup.u0, setup.p0, precision=setup.precision, device=setup.device)
        for s in sorted(set(objective.steps)):
            sim.step(s - sim.time)
            objective.record(s, sim.phi())
        sim.close()
        J = objective.value()
        seeds = objective.seeds((p.nz, p.ny, p.nx))
        sim = Simulation(p, setup.phi0, setup.u0, setup.p0, precision=setup.precision, device=setup.device)
        _, grad = sim.adjoint(max(objective.steps), seeds)
        sim.close()
        ctx.save_for_backward(torch.tensor(grad, dtype=torch.float64))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout):
        (g,) = ctx.saved_tensors
        gout = gout.to(torch.float64)
        return gout * g[0], gout * g[1], gout * g[2], None, None


def objective_rollout(M, xi, sigma, setup, objective):
    return ObjectiveRollout.apply(M, xi, sigma, setup, objective)
