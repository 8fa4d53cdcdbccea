"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's tests.

This module holds none of the PIC method's arithmetic: it draws counter-based
random numbers (SplitMix64, see picgen.c) and places particles by the
uniform-plasma recipe.  Both the CUDA library and the CPU oracle receive the
arrays it produces, so neither side has to reproduce the other's random
numbers.

Workload recipes (synthetic stand-ins shaped like the paper's uniform-plasma
scaling runs of Sec. 4.1 and its 2-particle-per-cell wakefield stage of
Sec. 4.2; normalised units, electrons q = -1, m = 1, cell size 1):

  uniform_32    32^3, 2 ppc, order 1, u ~ N(0, 0.01) + 1e-3 sin(2 pi x / 32), n = 1, FP64, 50 steps
  uniform_256   256^3, 8 ppc, order 3, u ~ N(0, 0.05), n = 1, 100 steps, FP64 and FP32-mixed
  wakefield     128 x 128 x 1024, 2 ppc, order 2, moving window, laser a0 = 2
  ensemble      96 boxes with edges in {16,24,32,48,64}, 1-8 ppc, n in [0.1, 10], order 1 or 3
  adjoint_64    64^3, 4 ppc, order 2, external plane-wave drive, 200 steps
  uniform_256_o1  256^3, 2 ppc, order 1, u ~ N(0, 0.05), n = 1 (the memory-bound case)
  WAKEFIELD     128 x 128 x 1024, moving window along z, laser + ramped plasma
  ENSEMBLE      96 independent boxes of uneven sizes
"""
import ctypes as ct
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(HERE, "_build")
_SRC = os.path.join(HERE, "picgen.c")
_lock = threading.Lock()
_lib = None

# Workload recipes.  `cfl` fixes dt = cfl / sqrt(sum 1/d^2).
WORKLOADS = {
    "uniform_32": dict(n=(32, 32, 32), ppc=2, order=1, sigma_u=0.01, density=1.0,
                       pert_amp=1e-3, pert_k=2 * np.pi / 32, cfl=0.99, steps=50, seed=0),
    "uniform_256": dict(n=(256, 256, 256), ppc=8, order=3, sigma_u=0.05, density=1.0,
                        pert_amp=0.0, pert_k=0.0, cfl=0.99, steps=100, seed=1),
    "adjoint_64": dict(n=(64, 64, 64), ppc=4, order=2, sigma_u=0.05, density=1.0,
                       pert_amp=0.0, pert_k=0.0, cfl=0.99, steps=200, seed=4),
    # the 2-particle-per-cell, order-1 case on the full-size grid: the
    # memory-bound end of the method (Sec. 4.2 notes that wakefield runs use
    # about 2 particles per cell)
    "uniform_256_o1": dict(n=(256, 256, 256), ppc=2, order=1, sigma_u=0.05, density=1.0,
                           pert_amp=0.0, pert_k=0.0, cfl=0.99, steps=100, seed=5),
}


def build(force: bool = False) -> str:
    out = os.path.join(_BUILD, "libpicgen.so")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                    _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            P, L, D, I, U = ct.c_void_p, ct.c_int64, ct.c_double, ct.c_int, ct.c_uint64
            lib.pg_uniform.argtypes = [U, L, L, I, P]
            lib.pg_normal.argtypes = [U, L, L, I, P]
            lib.pg_uniform_plasma.argtypes = [U, L, L, L, L, D, D, D, D, D, D, D, L, L,
                                              P, P, P, P, P, P, P]
            for f in (lib.pg_uniform, lib.pg_normal, lib.pg_uniform_plasma):
                f.restype = None
            _lib = lib
        return _lib


def uniform(seed: int, i0: int, n: int, draw: int) -> np.ndarray:
    """U[0,1) draws for counters [i0, i0+n) at one draw index."""
    out = np.empty(n)
    _load().pg_uniform(seed, i0, n, draw, out.ctypes.data_as(ct.c_void_p))
    return out


def normal(seed: int, i0: int, n: int, draw: int) -> np.ndarray:
    out = np.empty(n)
    _load().pg_normal(seed, i0, n, draw, out.ctypes.data_as(ct.c_void_p))
    return out


def dt_from_cfl(d, cfl: float) -> float:
    """dt = cfl * (sum 1/d^2)^(-1/2): the Courant number of the Yee scheme."""
    return float(cfl) / float(np.sqrt(sum(1.0 / (float(a) ** 2) for a in d)))


def uniform_plasma(seed, n, ppc, d=(1.0, 1.0, 1.0), sigma_u=0.0, density=1.0,
                   pert_amp=0.0, pert_k=0.0, cells=None, out=None):
    """Uniform plasma particles (dict of float64 arrays x,y,z,ux,uy,uz,w).

    `cells` = (c0, c1) restricts generation to a range of linear cell ids
    (the same particles a full generation would produce there).  `out` may
    give preallocated arrays (e.g. pinned host memory) to fill."""
    nx, ny, nz = (int(a) for a in n)
    c0, c1 = (0, nx * ny * nz) if cells is None else (int(cells[0]), int(cells[1]))
    npart = (c1 - c0) * int(ppc)
    weight = float(density) * d[0] * d[1] * d[2] / int(ppc)
    keys = ("x", "y", "z", "ux", "uy", "uz", "w")
    if out is None:
        out = {k: np.empty(npart) for k in keys}
    ptrs = []
    for k in keys:
        a = out[k]
        assert a.dtype == np.float64 and a.flags.c_contiguous and a.size >= npart
        ptrs.append(a.ctypes.data_as(ct.c_void_p))
    _load().pg_uniform_plasma(int(seed), nx, ny, nz, int(ppc), float(d[0]), float(d[1]), float(d[2]),
                              float(sigma_u), weight, float(pert_amp), float(pert_k), c0, c1, *ptrs)
    return out


def workload_particles(name: str, cells=None, out=None):
    w = WORKLOADS[name]
    return uniform_plasma(w["seed"], w["n"], w["ppc"], sigma_u=w["sigma_u"], density=w["density"],
                          pert_amp=w["pert_amp"], pert_k=w["pert_k"], cells=cells, out=out)


ENSEMBLE = dict(nboxes=96, edges=(16, 24, 32, 48, 64), ppc=(1, 8), density=(0.1, 10.0), orders=(1, 3),
                sigma_u=0.05, cfl=0.99, steps=200, seed=3)


def ensemble_boxes(seed: int = ENSEMBLE["seed"], nboxes: int = ENSEMBLE["nboxes"], edges=ENSEMBLE["edges"],
                   ppc=ENSEMBLE["ppc"], density=ENSEMBLE["density"], orders=ENSEMBLE["orders"]):
    """Boxes of the batched ensemble: per box b (the counter of each draw)
    each axis extent drawn uniformly from `edges` (draws 0, 1, 2), particles
    per cell uniform in {ppc[0] .. ppc[1]} (draw 3), density log-uniform in
    [density[0], density[1]] (draw 4), shape order orders[0] or orders[1]
    with probability 1/2 (draw 5), and the box's own loader seed."""
    u = [uniform(seed, 0, nboxes, k) for k in range(6)]
    out = []
    for b in range(nboxes):
        n = tuple(int(edges[min(int(u[a][b] * len(edges)), len(edges) - 1)]) for a in range(3))
        p = int(ppc[0] + min(int(u[3][b] * (ppc[1] - ppc[0] + 1)), ppc[1] - ppc[0]))
        dens = float(np.exp(np.log(density[0]) + u[4][b] * (np.log(density[1]) - np.log(density[0]))))
        order = int(orders[0] if u[5][b] < 0.5 else orders[1])
        out.append(dict(n=n, ppc=p, density=dens, order=order, seed=1000 * int(seed) + b + 1))
    return out


def ensemble_particles(boxes, sigma_u: float = ENSEMBLE["sigma_u"]):
    """Particles of all boxes concatenated in box order (box-local
    coordinates, unit cells) and the per-box counts."""
    parts = [uniform_plasma(b["seed"], b["n"], b["ppc"], sigma_u=sigma_u, density=b["density"]) for b in boxes]
    keys = ("x", "y", "z", "ux", "uy", "uz", "w")
    counts = np.array([p["x"].size for p in parts], dtype=np.int64)
    cat = {k: np.concatenate([p[k] for p in parts]) if parts else np.empty(0) for k in keys}
    return cat, counts, parts


# Laser-wakefield-shaped run (moving window along z): 24 cells per laser
# wavelength (omega0 = 2 pi / 24, critical density n_c = omega0^2 in these
# units), a0 = 2 (E0 = a0 omega0), waist 24 cells, 1/e field half-length 30
# cells, focus at z0 = 100 cells; plasma from a linear ramp over 64 cells
# starting at z = 200 to the plateau n = 1e-3 n_c, 2 particles per cell, cold.
WAKEFIELD = dict(n=(128, 128, 1024), ppc=2, order=2, lambda0=24.0, a0=2.0, w0=24.0, tau=30.0, z0=100.0,
                 ramp_start=200.0, ramp_length=64.0, n_over_nc=1e-3, cfl=0.99, speed=1.0, steps=2000)
# The same recipe shrunk to 16 x 16 x 64 cells (parity tests).
WAKEFIELD_SMALL = dict(n=(16, 16, 64), ppc=2, order=2, lambda0=8.0, a0=2.0, w0=4.0, tau=6.0, z0=16.0,
                       ramp_start=24.0, ramp_length=8.0, n_over_nc=1e-2, cfl=0.99, speed=1.0, steps=60)


def wakefield_plasma_density(cfg) -> float:
    omega0 = 2.0 * np.pi / cfg["lambda0"]
    return cfg["n_over_nc"] * omega0 * omega0


def laser_fields(cfg, d=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Initial fields (9, nx, ny, nz): a linearly polarised Gaussian pulse
    moving along +z, E_x = E0 exp(-r^2/w0^2) exp(-(z-z0)^2/tau^2)
    cos(omega0 (z-z0)) with r measured from the box axis, and B_y equal to the
    same expression at B_y's staggered location; everything else zero."""
    nx, ny, nz = cfg["n"]
    omega0 = 2.0 * np.pi / cfg["lambda0"]
    E0 = cfg["a0"] * omega0
    cx, cy = 0.5 * nx * d[0], 0.5 * ny * d[1]

    def pulse(x, y, z):
        r2 = (x - cx) ** 2 + (y - cy) ** 2
        return (E0 * np.exp(-r2 / cfg["w0"] ** 2) * np.exp(-((z - cfg["z0"]) / cfg["tau"]) ** 2)
                * np.cos(omega0 * (z - cfg["z0"])))

    i = (np.arange(nx) + 0.5)[:, None, None] * d[0]      # E_x and B_y sit at i + 1/2
    j = np.arange(ny)[None, :, None] * d[1]
    F = np.zeros((9, nx, ny, nz))
    F[0] = pulse(i, j, np.arange(nz)[None, None, :] * d[2])
    F[4] = pulse(i, j, (np.arange(nz) + 0.5)[None, None, :] * d[2])
    return F


def lattice_plasma(n, ppc, n0, ramp_start, ramp_length, d=(1.0, 1.0, 1.0), shifts=0):
    """Cold plasma on a lattice: in each cell (i, j, k) particles m = 0..ppc-1
    at in-cell offset (m + 1/2)/ppc on every axis, weight = density(lab z) dV /
    ppc with the density rising linearly from 0 at ramp_start over
    ramp_length to n0 (lab z = window z + shifts dz); particles where the
    density is zero are left out.  Order: i, j, k, m."""
    nx, ny, nz = (int(a) for a in n)
    i, j, k, m = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), np.arange(ppc), indexing="ij")
    off = (m.ravel() + 0.5) / ppc
    x = (i.ravel() + off) * d[0]
    y = (j.ravel() + off) * d[1]
    z = (k.ravel() + off) * d[2]
    zl = z + shifts * d[2]
    if ramp_length > 0:
        dens = n0 * np.clip((zl - ramp_start) / ramp_length, 0.0, 1.0)
    else:
        dens = np.where(zl >= ramp_start, n0, 0.0)
    keep = dens > 0
    zero = np.zeros(int(keep.sum()))
    return {"x": x[keep], "y": y[keep], "z": z[keep], "ux": zero, "uy": zero.copy(), "uz": zero.copy(),
            "w": dens[keep] * d[0] * d[1] * d[2] / ppc}


def wakefield_particles(cfg):
    return lattice_plasma(cfg["n"], cfg["ppc"], wakefield_plasma_density(cfg), cfg["ramp_start"],
                          cfg["ramp_length"])


def drive_amplitude(seed: int) -> float:
    """Amplitude of the external plane-wave drive of the differentiation
    workload: A = 0.05 (1 + U), U uniform in [0, 1) from the seed (draw 15,
    which the particle loader does not use)."""
    return 0.05 * (1.0 + float(uniform(seed, 0, 1, 15)[0]))


def random_fields(seed: int, n, scale: float = 1.0) -> np.ndarray:
    """Nine seeded uniform(-scale, scale) field arrays (Ex..Bz, Jx..Jz)."""
    C = int(n[0]) * int(n[1]) * int(n[2])
    f = np.empty((9, C))
    for c in range(9):
        f[c] = uniform(seed, c * C, C, 9)
    return ((2.0 * f - 1.0) * scale).reshape((9,) + tuple(int(a) for a in n))
