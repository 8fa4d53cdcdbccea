"""torch.autograd wrapper of the library's discrete adjoint (pic_step_adjoint).

`field_energy_loss(A, u0, spec)` runs a fresh simulation from the particles
of `spec` with initial momenta `u0` and drive amplitude `A`, and returns the
field energy L = 1/2 sum(|E|^2 + |B|^2) dV after `spec.nsteps` steps.  Its
backward uses the gradients the CUDA library computed in the same call:
dL/dA and dL/du0 (the reverse sweep runs in the library's kernels; nothing is
differentiated by torch).
"""
from dataclasses import dataclass, field

import numpy as np
import torch

from . import pic


@dataclass
class RunSpec:
    """A run: grid, shape order, precision, particles (x, y, z, w as float64
    arrays), species charge/mass, drive wavenumber, steps and checkpoint
    spacing."""
    n: tuple
    parts: dict
    nsteps: int
    drive_k: float
    d: tuple = (1.0, 1.0, 1.0)
    dt: float = 0.0
    cfl: float = 0.99
    order: int = 2
    precision: int = pic.FP64
    q: float = -1.0
    m: float = 1.0
    ckpt_every: int = 20
    sort_every: int = 1
    tile: tuple = (0, 0, 0)
    extra: dict = field(default_factory=dict)


def _context(spec: RunSpec):
    return pic.Context(spec.n, d=spec.d, dt=spec.dt, cfl=spec.cfl, precision=spec.precision, order=spec.order,
                       sort_every=spec.sort_every, tile=spec.tile)


class _FieldEnergyLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, u0, spec):
        parts = {k: np.ascontiguousarray(spec.parts[k], dtype=np.float64) for k in ("x", "y", "z", "w")}
        u = u0.detach().to("cpu", torch.float64).numpy()
        for a, key in enumerate(("ux", "uy", "uz")):
            parts[key] = np.ascontiguousarray(u[a])
        with _context(spec) as sim:
            sim.load_particles(spec.q, spec.m, parts)
            sim.set_external_drive(float(A.detach().cpu()), spec.drive_k)
            loss, dA, du = sim.step_adjoint(spec.nsteps, spec.ckpt_every)
        ctx.save_for_backward(torch.tensor(dA, dtype=torch.float64), torch.from_numpy(du))
        ctx.devices = (A.device, u0.device)
        ctx.dtypes = (A.dtype, u0.dtype)
        return torch.tensor(loss, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, g):
        dA, du = ctx.saved_tensors
        g = g.detach().to("cpu", torch.float64)
        gA = (g * dA).to(ctx.devices[0], ctx.dtypes[0]).reshape(())
        gu = (g * du).to(ctx.devices[1], ctx.dtypes[1])
        return gA, gu, None


def field_energy_loss(A: torch.Tensor, u0: torch.Tensor, spec: RunSpec) -> torch.Tensor:
    """L(A, u0) as a differentiable torch scalar (float64).  A: 0-d tensor;
    u0: (3, N) tensor of initial momenta in the order of spec.parts."""
    return _FieldEnergyLoss.apply(A, u0, spec)
