"""Shared helpers of the GPU tests: run the CUDA path and the CPU oracle on
the same seeded inputs and compare them."""
import numpy as np

from oracle import Oracle
from paper_2101_12149_gb300 import inputs, pic

KEYS = pic.PARTICLE_KEYS


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def periodic_diff(a, b, L):
    return (a - b + 0.5 * L) % L - 0.5 * L


def by_id(parts):
    order = np.argsort(parts["id"])
    return {k: np.asarray(v)[order] for k, v in parts.items()}


def compare_particles(gpu, ref, L):
    """Relative L2 of positions (periodic distance) and momenta, matched by id."""
    g = by_id(gpu)
    assert np.array_equal(g["id"], np.arange(g["id"].size)), "ids are not a permutation"
    pos = np.concatenate([periodic_diff(g[k], ref[k], L[a]) for a, k in enumerate(("x", "y", "z"))])
    pos_ref = np.concatenate([ref[k] for k in ("x", "y", "z")])
    mom = np.concatenate([g[k] - ref[k] for k in ("ux", "uy", "uz")])
    mom_ref = np.concatenate([ref[k] for k in ("ux", "uy", "uz")])
    return (np.linalg.norm(pos) / np.linalg.norm(pos_ref),
            np.linalg.norm(mom) / max(np.linalg.norm(mom_ref), 1e-300))


class Case:
    """One workload run side by side on the GPU and in the oracle."""

    def __init__(self, n, order, ppc, sigma_u, seed, precision=pic.FP64, d=(1.0, 1.0, 1.0), cfl=0.99,
                 field_scale=0.0, sort_every=1, tile=(0, 0, 0), stream=None, density=1.0, pert=(0.0, 0.0),
                 q=-1.0, m=1.0, pusher=0, gather=0):
        self.n, self.order, self.d = tuple(n), order, tuple(d)
        self.L = [n[a] * d[a] for a in range(3)]
        self.q, self.m = q, m
        self.dt = inputs.dt_from_cfl(d, cfl)
        self.parts = inputs.uniform_plasma(seed, n, ppc, d=d, sigma_u=sigma_u, density=density,
                                           pert_amp=pert[0], pert_k=pert[1])
        self.F = np.zeros((9,) + self.n)
        if field_scale:
            self.F[:6] = inputs.random_fields(seed + 1000, n, field_scale)[:6]
        self.ctx = pic.Context(n, d=d, dt=self.dt, precision=precision, order=order, sort_every=sort_every,
                               tile=tile, stream=stream)
        self.ctx.set_fields(self.F)
        self.ctx.load_particles(q, m, self.parts)
        self.pusher, self.gather = pusher, gather
        if pusher or gather:
            self.ctx.set_particle_algorithms(pusher, gather)
        self.O = Oracle()
        self.g = self.O.grid(n, d)
        self.ref = {k: v.copy() for k, v in self.parts.items()}
        self.Fref = self.F.copy()
        self.nsteps = 0

    def oracle_steps(self, k, drive=(0.0, 0.0)):
        for _ in range(k):
            self.O.pic_step(self.g, self.order, self.dt, self.q, self.m, self.ref, self.Fref,
                            drive[0], drive[1], self.nsteps * self.dt, pusher=self.pusher, gather=self.gather)
            self.nsteps += 1

    def errors(self):
        F = self.ctx.get_fields()
        parts = self.ctx.get_particles()
        ep, eu = compare_particles(parts, self.ref, self.L)
        return {
            "EB": rel_l2(F[:6], self.Fref[:6]),
            "J": rel_l2(F[6:], self.Fref[6:]),
            "pos": ep,
            "mom": eu,
        }
