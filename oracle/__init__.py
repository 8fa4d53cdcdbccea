"""FP64 CPU oracle for the electromagnetic PIC hot path (numpy front end).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow definition the CUDA
library is checked against.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the product package never does,
and the two share no code.

Every function forwards to the C implementation in pic_oracle.c, which cites
the method each one restates.  Arrays are numpy float64, C-contiguous.
Fields are held as one array of shape (9, nx, ny, nz):
Ex, Ey, Ez, Bx, By, Bz, Jx, Jy, Jz (k fastest).
"""
import ctypes as ct
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_libs = {}

_dp = ct.POINTER(ct.c_double)


class _Grid(ct.Structure):
    _fields_ = [("n", ct.c_int64 * 3), ("d", ct.c_double * 3), ("zopen", ct.c_int64)]


def _declare(lib):
    P = ct.c_void_p
    D = ct.c_double
    I = ct.c_int
    L = ct.c_int64
    G = ct.POINTER(_Grid)
    sig = {
        "orc_shape": (D, [I, D]),
        "orc_gather_many": (None, [G, I, P, L, P, P, P, P]),
        "orc_gather_ec_many": (None, [G, I, P, L, P, P, P, P]),
        "orc_boris_many": (None, [D, D, D, L, P, P, P, P]),
        "orc_vay_many": (None, [D, D, D, L, P, P, P, P]),
        "orc_deposit_many": (None, [G, I, D, D, L, P, P, P, P, P, P, P, P]),
        "orc_rho_many": (None, [G, I, D, L, P, P, P, P, P]),
        "orc_yee_b": (None, [G, D, P, P]),
        "orc_yee_e": (None, [G, D, P, P, P]),
        "orc_yee_step": (None, [G, D, P, P, P]),
        "orc_pic_step": (None, [G, I, D, D, D, L, P, P, P, P, P, P, P, P, D, D, D]),
        "orc_pic_step_alg": (None, [G, I, D, D, D, L, P, P, P, P, P, P, P, P, D, D, D, I, I]),
        "orc_pic_step_full": (None, [G, I, D, D, D, L, P, P, P, P, P, P, P, P, D, D, D, I, I, I]),
        "orc_yee_b_ckc": (None, [G, D, P, P]),
        "orc_yee_step_ckc": (None, [G, D, P, P, P]),
        "orc_filter_z": (None, [G, I, P, P]),
        "orc_pic_step_filtered": (None, [G, I, D, D, D, L, P, P, P, P, P, P, P, P, D, D, D, I, I, I, I]),
        "orc_div_edge": (None, [G, P, P]),
        "orc_div_face": (None, [G, P, P]),
        "orc_field_energy": (D, [G, P]),
        "orc_kinetic_energy": (D, [D, L, P, P, P, P]),
        "orc_wrap": (D, [D, D]),
        "orc_dshape": (D, [I, D]),
        "orc_gather_adj": (None, [G, I, P, P, P, P, P]),
        "orc_boris_adj": (None, [D, D, D, P, P, P, P, P, P, P]),
        "orc_deposit_adj": (None, [G, I, D, D, P, P, P, P, P]),
        "orc_yee_step_adj": (None, [G, D, P, P, P]),
        "orc_pic_adjoint": (None, [G, I, D, D, D, L, P, P, P, P, P, P, P, P, I, D, D, P, P, P]),
        "orc_curlE": (None, [G, P, P]),
        "orc_curlE_T": (None, [G, P, P]),
        "orc_curlB_T": (None, [G, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(mutant: int = 0):
    """The oracle library (the default build, or a planted-mistake build)."""
    with _lock:
        if mutant not in _libs:
            path = _build.build(mutant)
            _libs[mutant] = _declare(ct.CDLL(os.path.abspath(path)))
        return _libs[mutant]


_mt_lib = None


def load_mt():
    """The multi-threaded CPU baseline library (OpenMP)."""
    global _mt_lib
    with _lock:
        if _mt_lib is None:
            lib = ct.CDLL(os.path.abspath(_build.build_mt()))
            P, D, I, L, G = ct.c_void_p, ct.c_double, ct.c_int, ct.c_int64, ct.POINTER(_Grid)
            lib.orc_mt_pic_step.restype = None
            lib.orc_mt_pic_step.argtypes = [G, I, D, D, D, L, P, P, P, P, P, P, P, P, D, D, D, I, I, I, P]
            lib.orc_mt_threads.restype = I
            lib.orc_mt_threads.argtypes = [I]
            _mt_lib = lib
        return _mt_lib


class OracleMT:
    """The multi-threaded CPU baseline (pic_oracle_mt.c): the oracle's step on
    several threads, each depositing into private current arrays that are
    summed in thread order (the CPU deposition scheme of Sec. 3.4.1)."""

    def __init__(self, nthreads: int = 0):
        self.lib = load_mt()
        self.nthreads = int(self.lib.orc_mt_threads(int(nthreads)))
        self._scratch = np.empty(0)

    def pic_step(self, g, p, dt, q, m, parts, fields, drive_amp=0.0, drive_k=0.0, t=0.0, pusher=0, gather=0):
        keys = ("x", "y", "z", "ux", "uy", "uz", "w")
        for k in keys:
            assert parts[k].dtype == np.float64 and parts[k].flags.c_contiguous
        assert fields.dtype == np.float64 and fields.flags.c_contiguous
        C = int(g.n[0] * g.n[1] * g.n[2])
        if self._scratch.size < 3 * C * self.nthreads:
            self._scratch = np.empty(3 * C * self.nthreads)
        self.lib.orc_mt_pic_step(ct.byref(g), int(p), float(dt), float(q), float(m), parts["x"].size,
                                 *[parts[k].ctypes.data_as(ct.c_void_p) for k in keys],
                                 (ct.c_void_p * 9)(*[fields[c].ctypes.data for c in range(9)]),
                                 float(drive_amp), float(drive_k), float(t), int(pusher), int(gather),
                                 self.nthreads, self._scratch.ctypes.data_as(ct.c_void_p))


class Oracle:
    """Thin numpy wrapper over one oracle build."""

    def __init__(self, mutant: int = 0):
        self.lib = load(mutant)

    # -- helpers -----------------------------------------------------
    @staticmethod
    def grid(n, d=(1.0, 1.0, 1.0), zopen=False):
        g = _Grid()
        for a in range(3):
            g.n[a] = int(n[a])
            g.d[a] = float(d[a])
        g.zopen = 1 if zopen else 0
        return g

    @staticmethod
    def _f64(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a

    @staticmethod
    def _ptr(a):
        return a.ctypes.data_as(ct.c_void_p)

    def _ptr_array(self, arrays):
        arr = (ct.c_void_p * len(arrays))(*[a.ctypes.data for a in arrays])
        return arr

    # -- method steps ------------------------------------------------
    def shape(self, p, xi):
        xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
        f = self.lib.orc_shape
        return np.array([f(int(p), float(v)) for v in xi.ravel()]).reshape(xi.shape)

    def gather(self, g, p, fields, x, y, z, energy=False):
        """E,B at the particle positions; returns (np, 6).  energy=True: the
        energy-conserving gather (order p - 1 along staggered axes)."""
        F = [self._f64(fields[c]) for c in range(6)]
        x, y, z = self._f64(x), self._f64(y), self._f64(z)
        out = np.zeros((x.size, 6))
        f = self.lib.orc_gather_ec_many if energy else self.lib.orc_gather_many
        f(ct.byref(g), int(p), self._ptr_array(F), x.size, self._ptr(x), self._ptr(y), self._ptr(z), self._ptr(out))
        return out

    def vay(self, q, m, dt, EB, ux, uy, uz):
        """Vay's pusher; returns the pushed (ux, uy, uz)."""
        EB = self._f64(EB)
        ux, uy, uz = (self._f64(a).copy() for a in (ux, uy, uz))
        self.lib.orc_vay_many(float(q), float(m), float(dt), ux.size, self._ptr(EB),
                              self._ptr(ux), self._ptr(uy), self._ptr(uz))
        return ux, uy, uz

    def boris(self, q, m, dt, EB, ux, uy, uz):
        """Returns the pushed (ux, uy, uz)."""
        EB = self._f64(EB)
        ux, uy, uz = (self._f64(a).copy() for a in (ux, uy, uz))
        self.lib.orc_boris_many(float(q), float(m), float(dt), ux.size, self._ptr(EB),
                                self._ptr(ux), self._ptr(uy), self._ptr(uz))
        return ux, uy, uz

    def deposit(self, g, p, dt, q, x0, y0, z0, x1, y1, z1, w, J=None):
        """Esirkepov current of all particles; returns J of shape (3, nx, ny, nz)."""
        n = tuple(g.n)
        if J is None:
            J = np.zeros((3,) + n)
        arrs = [self._f64(a) for a in (x0, y0, z0, x1, y1, z1, w)]
        Jl = [J[c] for c in range(3)]
        self.lib.orc_deposit_many(ct.byref(g), int(p), float(dt), float(q), arrs[0].size,
                                  *[self._ptr(a) for a in arrs], self._ptr_array(Jl))
        return J

    def rho(self, g, p, q, x, y, z, w):
        n = tuple(g.n)
        out = np.zeros(n)
        arrs = [self._f64(a) for a in (x, y, z, w)]
        self.lib.orc_rho_many(ct.byref(g), int(p), float(q), arrs[0].size,
                              *[self._ptr(a) for a in arrs], self._ptr(out))
        return out

    def yee_b(self, g, h, E, B):
        self.lib.orc_yee_b(ct.byref(g), float(h), self._ptr_array([E[0], E[1], E[2]]),
                           self._ptr_array([B[0], B[1], B[2]]))

    def yee_e(self, g, dt, E, B, J):
        self.lib.orc_yee_e(ct.byref(g), float(dt), self._ptr_array([E[0], E[1], E[2]]),
                           self._ptr_array([B[0], B[1], B[2]]), self._ptr_array([J[0], J[1], J[2]]))

    def yee_b_ckc(self, g, h, E, B):
        self.lib.orc_yee_b_ckc(ct.byref(g), float(h), self._ptr_array([E[0], E[1], E[2]]),
                               self._ptr_array([B[0], B[1], B[2]]))

    def yee_step(self, g, dt, fields, solver=0):
        """In place on fields (9, nx, ny, nz); solver 0 Yee, 1 CKC."""
        f = self.lib.orc_yee_step_ckc if solver else self.lib.orc_yee_step
        f(ct.byref(g), float(dt),
                              self._ptr_array([fields[0], fields[1], fields[2]]),
                              self._ptr_array([fields[3], fields[4], fields[5]]),
                              self._ptr_array([fields[6], fields[7], fields[8]]))

    def pic_step(self, g, p, dt, q, m, parts, fields, drive_amp=0.0, drive_k=0.0, t=0.0, pusher=0, gather=0,
                 solver=0, filter_passes=0):
        """One PIC step, in place on parts (dict of x,y,z,ux,uy,uz,w float64
        arrays) and fields (9, nx, ny, nz); pusher 0 Boris / 1 Vay, gather 0
        momentum- / 1 energy-conserving; filter_passes > 0: the particles
        gather from E and B filtered along z (orc_filter_z)."""
        keys = ("x", "y", "z", "ux", "uy", "uz", "w")
        for k in keys:
            assert parts[k].dtype == np.float64 and parts[k].flags.c_contiguous
        assert fields.dtype == np.float64 and fields.flags.c_contiguous
        if filter_passes:
            self.lib.orc_pic_step_filtered(ct.byref(g), int(p), float(dt), float(q), float(m), parts["x"].size,
                                           *[self._ptr(parts[k]) for k in keys],
                                           self._ptr_array([fields[c] for c in range(9)]),
                                           float(drive_amp), float(drive_k), float(t), int(pusher), int(gather),
                                           int(solver), int(filter_passes))
            return
        self.lib.orc_pic_step_full(ct.byref(g), int(p), float(dt), float(q), float(m), parts["x"].size,
                                   *[self._ptr(parts[k]) for k in keys],
                                   self._ptr_array([fields[c] for c in range(9)]),
                                   float(drive_amp), float(drive_k), float(t), int(pusher), int(gather), int(solver))

    def filter_z(self, g, npass, F):
        """orc_filter_z on one component (nx, ny, nz)."""
        F = self._f64(F)
        out = np.empty_like(F)
        self.lib.orc_filter_z(ct.byref(g), int(npass), self._ptr(F), self._ptr(out))
        return out

    # -- moving window (z open) -----------------------------------------
    # Readings of the wakefield run: z is open (fields beyond the ends are
    # zero, particles leaving [0, Lz) are removed after their deposit); after
    # the field update of step n the window moves one cell along z whenever
    # speed * t_{n+1} reaches (shifts + 1) dz: fields move down one cell (the
    # new front slab is zero), particles move by -dz and those below z = 0 are
    # removed, and the new front slab of cells is filled with plasma.
    @staticmethod
    def density_profile(z_lab, n0, ramp_start, ramp_length):
        """Plasma density at lab-frame z: 0 below ramp_start, rising linearly
        over ramp_length to the plateau n0."""
        z = np.asarray(z_lab, dtype=np.float64)
        if ramp_length > 0:
            return n0 * np.clip((z - ramp_start) / ramp_length, 0.0, 1.0)
        return np.where(z >= ramp_start, n0, 0.0)

    @staticmethod
    def lattice_slab(g, k, ppc, shifts, n0, ramp_start, ramp_length, first_id):
        """Plasma particles of the cell slab k (window frame): in each cell
        (i, j, k) particles m = 0..ppc-1 at in-cell offset (m + 1/2)/ppc on every
        axis, at rest, weight = density(lab z) dV / ppc; ids first_id +
        (i ny + j) ppc + m; particles where the density is zero are not made."""
        nx, ny = int(g.n[0]), int(g.n[1])
        d = [float(g.d[a]) for a in range(3)]
        i, j, m = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(ppc), indexing="ij")
        off = (m.ravel() + 0.5) / ppc
        x = (i.ravel() + off) * d[0]
        y = (j.ravel() + off) * d[1]
        z = (k + off) * d[2]
        dens = Oracle.density_profile(z + shifts * d[2], n0, ramp_start, ramp_length)
        ids = first_id + (i.ravel() * ny + j.ravel()) * ppc + m.ravel()
        keep = dens > 0
        zero = np.zeros(int(keep.sum()))
        return {"x": x[keep], "y": y[keep], "z": z[keep], "ux": zero.copy(), "uy": zero.copy(), "uz": zero.copy(),
                "w": dens[keep] * d[0] * d[1] * d[2] / ppc, "id": ids[keep].astype(np.int64)}

    def window_step(self, g, p, dt, q, m, parts, fields, win):
        """One step of a moving-window run.  parts: dict of the 7 particle
        arrays plus 'id'; fields (9, nx, ny, nz) in place; win: dict with
        step, shifts, speed, next_id and the injected plasma (ppc, n0,
        ramp_start, ramp_length).  Returns the new particle dict."""
        assert g.zopen
        Lz = g.n[2] * g.d[2]
        self.pic_step(g, p, dt, q, m, parts, fields, 0.0, 0.0, win["step"] * dt, pusher=win.get("pusher", 0),
                      gather=win.get("gather", 0), solver=win.get("solver", 0),
                      filter_passes=win.get("filter_passes", 0))
        keep = (parts["z"] >= 0.0) & (parts["z"] < Lz)
        parts = {k: np.ascontiguousarray(v[keep]) for k, v in parts.items()}
        win["step"] += 1
        while win["speed"] > 0 and win["speed"] * (win["step"] * dt) >= (win["shifts"] + 1) * g.d[2]:
            fields[:, :, :, :-1] = fields[:, :, :, 1:].copy()
            fields[:, :, :, -1] = 0.0
            parts["z"] = parts["z"] - g.d[2]
            keep = parts["z"] >= 0.0
            parts = {k: v[keep] for k, v in parts.items()}
            win["shifts"] += 1
            if win["ppc"] > 0:
                new = self.lattice_slab(g, int(g.n[2]) - 1, win["ppc"], win["shifts"], win["n0"], win["ramp_start"],
                                        win["ramp_length"], win["next_id"])
                win["next_id"] += int(g.n[0]) * int(g.n[1]) * win["ppc"]
                parts = {k: np.concatenate([parts[k], new[k]]) for k in parts}
            parts = {k: np.ascontiguousarray(v) for k, v in parts.items()}
        return parts

    # -- diagnostics -------------------------------------------------
    def div_edge(self, g, F3):
        out = np.zeros(tuple(g.n))
        F3 = [self._f64(F3[c]) for c in range(3)]
        self.lib.orc_div_edge(ct.byref(g), self._ptr_array(F3), self._ptr(out))
        return out

    def div_face(self, g, F3):
        out = np.zeros(tuple(g.n))
        F3 = [self._f64(F3[c]) for c in range(3)]
        self.lib.orc_div_face(ct.byref(g), self._ptr_array(F3), self._ptr(out))
        return out

    def field_energy(self, g, fields):
        F = [self._f64(fields[c]) for c in range(6)]
        return self.lib.orc_field_energy(ct.byref(g), self._ptr_array(F))

    def kinetic_energy(self, m, ux, uy, uz, w):
        arrs = [self._f64(a) for a in (ux, uy, uz, w)]
        return self.lib.orc_kinetic_energy(float(m), arrs[0].size, *[self._ptr(a) for a in arrs])

    def wrap(self, x, L):
        return self.lib.orc_wrap(float(x), float(L))

    # -- adjoint -----------------------------------------------------
    def dshape(self, p, xi):
        xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
        f = self.lib.orc_dshape
        return np.array([f(int(p), float(v)) for v in xi.ravel()]).reshape(xi.shape)

    @staticmethod
    def _v3(a):
        return np.ascontiguousarray(a, dtype=np.float64)

    def gather_adj(self, g, p, fields, x, lamEB):
        """One particle: returns (lamF (6, n...), lam_x (3))."""
        F = [self._f64(fields[c]) for c in range(6)]
        lamF = np.zeros((6,) + tuple(g.n))
        lx = np.zeros(3)
        self.lib.orc_gather_adj(ct.byref(g), int(p), self._ptr_array(F), self._ptr_array([lamF[c] for c in range(6)]),
                                self._ptr(self._v3(x)), self._ptr(self._v3(lamEB)), self._ptr(lx))
        return lamF, lx

    def boris_adj(self, q, m, dt, E, B, u_old, lam_unew):
        """Returns (lam_uold, lam_E, lam_B)."""
        lu, lE, lB = np.zeros(3), np.zeros(3), np.zeros(3)
        self.lib.orc_boris_adj(float(q), float(m), float(dt), self._ptr(self._v3(E)), self._ptr(self._v3(B)),
                               self._ptr(self._v3(u_old)), self._ptr(self._v3(lam_unew)), self._ptr(lu),
                               self._ptr(lE), self._ptr(lB))
        return lu, lE, lB

    def deposit_adj(self, g, p, dt, qw, x0, x1, lamJ):
        """One particle: returns (lam_x0, lam_x1)."""
        l0, l1 = np.zeros(3), np.zeros(3)
        LJ = [self._f64(lamJ[c]) for c in range(3)]
        self.lib.orc_deposit_adj(ct.byref(g), int(p), float(dt), float(qw), self._ptr(self._v3(x0)),
                                 self._ptr(self._v3(x1)), self._ptr_array(LJ), self._ptr(l0), self._ptr(l1))
        return l0, l1

    def yee_step_adj(self, g, dt, lamE, lamB):
        """Returns (lamE^n, lamB^n, lamJ) from the adjoints after the step."""
        lE = np.array(lamE, dtype=np.float64, copy=True)
        lB = np.array(lamB, dtype=np.float64, copy=True)
        lJ = np.zeros_like(lE)
        self.lib.orc_yee_step_adj(ct.byref(g), float(dt), self._ptr_array([lE[c] for c in range(3)]),
                                  self._ptr_array([lB[c] for c in range(3)]), self._ptr_array([lJ[c] for c in range(3)]))
        return lE, lB, lJ

    def _map3(self, fname, g, A):
        A = [self._f64(A[c]) for c in range(3)]
        out = np.zeros((3,) + tuple(g.n))
        getattr(self.lib, fname)(ct.byref(g), self._ptr_array(A), self._ptr_array([out[c] for c in range(3)]))
        return out

    def curlE(self, g, E):
        return self._map3("orc_curlE", g, E)

    def curlE_T(self, g, B):
        return self._map3("orc_curlE_T", g, B)

    def curlB_T(self, g, E):
        return self._map3("orc_curlB_T", g, E)

    def pic_adjoint(self, g, p, dt, q, m, parts, fields, nsteps, A, kd):
        """Forward nsteps then reverse; returns (loss, dL/dA, dL/du (3, np)).
        parts and fields are left at the final forward state."""
        keys = ("x", "y", "z", "ux", "uy", "uz", "w")
        np_ = parts["x"].size
        dA = ct.c_double()
        loss = ct.c_double()
        du = np.zeros((3, np_))
        self.lib.orc_pic_adjoint(ct.byref(g), int(p), float(dt), float(q), float(m), np_,
                                 *[self._ptr(parts[k]) for k in keys], self._ptr_array([fields[c] for c in range(9)]),
                                 int(nsteps), float(A), float(kd), ct.byref(dA), self._ptr(du), ct.byref(loss))
        return loss.value, dA.value, du
