"""Thin ctypes binding of libpic (include/pic.h).  Argument marshalling only:
every step of the PIC path runs in the CUDA library.

Arrays may be numpy arrays (host memory) or torch CUDA tensors (device
memory of the context's GPU); float64 unless stated.  The binding fails
loudly if libpic has not been built: there is no CPU fallback.
"""
import ctypes as ct
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PIC_LIBRARY may name another build of the same library (e.g. the
# self-checking libpic_check.so).
LIB_PATH = os.environ.get("PIC_LIBRARY") or os.path.join(HERE, "_build", "libpic.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pic.h")

PIC_OK, PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_OOM, PIC_ERR_CUDA, PIC_ERR_STATE, PIC_ERR_PARTICLE, PIC_ERR_TIMEOUT = range(8)
STATUS_NAMES = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_CFL", 3: "PIC_ERR_OOM", 4: "PIC_ERR_CUDA",
                5: "PIC_ERR_STATE", 6: "PIC_ERR_PARTICLE", 7: "PIC_ERR_TIMEOUT"}
FP64, FP32_MIXED = 0, 1
ORDER_RANDOM = -1
FIELDS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz")
PARTICLE_KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")

_lock = threading.Lock()
_lib = None


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ct.Structure):
    _fields_ = [("n", ct.c_int32 * 3), ("d", ct.c_double * 3), ("dt", ct.c_double), ("cfl", ct.c_double),
                ("precision", ct.c_int32), ("order", ct.c_int32), ("sort_every", ct.c_int32),
                ("window_axis", ct.c_int32), ("window_speed", ct.c_double), ("seed", ct.c_uint64),
                ("tile", ct.c_int32 * 3), ("solver", ct.c_int32)]


class BatchTuning(ct.Structure):
    _fields_ = [("tile", ct.c_int32 * 3), ("run", ct.c_int32), ("sort_every", ct.c_int32)]


def load_library(path: str = LIB_PATH):
    """Load libpic; raises if it is missing (build it with build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libpic is not built ({path} missing): run paper_2101_12149_gb300.build.build()")
        lib = ct.CDLL(path)
        P, I32, I64, D = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_double
        sigs = {
            "pic_init_grid": [ct.POINTER(GridDesc), P, ct.POINTER(P)],
            "pic_load_particles": [P, D, D, I64, P, P, P, P, P, P, P, ct.c_int],
            "pic_gather_push": [P],
            "pic_deposit": [P],
            "pic_yee_step": [P],
            "pic_sort_particles": [P, I32],
            "pic_step": [P, I32],
            "pic_step_adjoint": [P, I32, I32, P, P, P, ct.c_int],
            "pic_set_window_plasma": [P, I32, D, D, D],
            "pic_set_particle_algorithms": [P, I32, I32],
            "pic_get_window": [P, ct.POINTER(I64), ct.POINTER(D)],
            "pic_get_field": [P, I32, P, ct.c_int],
            "pic_set_field": [P, I32, P, ct.c_int],
            "pic_num_particles": [P, ct.POINTER(I64)],
            "pic_get_particles": [P, P, P, P, P, P, P, P, P, ct.c_int],
            "pic_set_external_drive": [P, D, D],
            "pic_get_time": [P, ct.POINTER(I64), ct.POINTER(D)],
            "pic_diagnostics": [P, P],
            "pic_sync": [P],
            "pic_set_timing": [P, I32],
            "pic_get_timing": [P, I32, P, P, P, ct.POINTER(I32)],
            "pic_launch_count": [P, ct.POINTER(I64)],
            "pic_destroy": [P],
            "pic_sort_keys_noalloc": [P, I64, I32, P, P, P],
            "pic_reserve_adjoint": [P, I32, I32],
            "pic_charge_density": [P, P, ct.c_int],
            "pic_continuity_mark": [P],
            "pic_continuity_residual": [P, P],
            "pic_set_fp64_gamma": [P, D],
            "pic_set_gather_filter": [P, I32],
            "pic_measure_fma_peak": [I32, ct.POINTER(D)],
            "pic_batch_init": [I32, P, P, P, D, D, I32, P, ct.POINTER(P)],
            "pic_batch_load_particles": [P, D, D, P, P, P, P, P, P, P, P, ct.c_int],
            "pic_batch_step": [P, I32],
            "pic_batch_get_field": [P, I32, I32, P, ct.c_int],
            "pic_batch_set_field": [P, I32, I32, P, ct.c_int],
            "pic_batch_get_particles": [P, I32, P, P, P, P, P, P, P, P, ct.c_int],
            "pic_batch_diagnostics": [P, I32, P],
            "pic_batch_info": [P, I32, ct.POINTER(I64), ct.POINTER(I64), ct.POINTER(I64), ct.POINTER(D)],
            "pic_batch_set_tuning": [P, ct.POINTER(BatchTuning)],
            "pic_batch_get_tuning": [P, ct.POINTER(BatchTuning)],
            "pic_batch_autotune": [P, I32, ct.POINTER(BatchTuning), ct.POINTER(D)],
            "pic_batch_launch_count": [P, ct.POINTER(I64)],
            "pic_batch_destroy": [P],
        }
        for name, args in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ct.c_int
        lib.pic_last_error.argtypes = []
        lib.pic_last_error.restype = ct.c_char_p
        _lib = lib
        return lib


def declared_symbols(header: str = HEADER):
    """Names of the functions include/pic.h declares."""
    import re
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:pic_status|const char\*)\s+(pic_\w+)\s*\(", text, re.M)))


def _check(status):
    if status != PIC_OK:
        msg = _lib.pic_last_error().decode() if _lib is not None else ""
        raise PicError(status, msg)


def _ptr(a):
    """(address, on_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


class Context:
    """One PIC simulation: grid, fields and one particle species on one GPU."""

    def __init__(self, n, d=(1.0, 1.0, 1.0), dt=0.0, cfl=0.99, precision=FP64, order=1, sort_every=1,
                 tile=(0, 0, 0), stream=None, window_speed=None, solver=0, seed=0):
        self.lib = load_library()
        desc = GridDesc()
        for a in range(3):
            desc.n[a] = int(n[a])
            desc.d[a] = float(d[a])
            desc.tile[a] = int(tile[a])
        desc.dt = float(dt)
        desc.cfl = float(cfl)
        desc.precision = int(precision)
        desc.order = int(order)
        desc.sort_every = int(sort_every)
        desc.window_axis = -1 if window_speed is None else 2
        desc.window_speed = 0.0 if window_speed is None else float(window_speed)
        desc.seed = int(seed)
        desc.solver = {"yee": 0, "ckc": 1}[solver] if isinstance(solver, str) else int(solver)
        self.n = tuple(int(v) for v in n)
        self.C = self.n[0] * self.n[1] * self.n[2]
        h = ct.c_void_p()
        s = None
        if stream is not None:
            s = ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check(self.lib.pic_init_grid(ct.byref(desc), s, ct.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- particles ---------------------------------------------------
    def load_particles(self, q, m, parts):
        arrs = [parts[k] for k in PARTICLE_KEYS]
        n = int(arrs[0].shape[0]) if hasattr(arrs[0], "shape") else len(arrs[0])
        ptrs = [_ptr(a) for a in arrs]
        on_dev = {p[1] for p in ptrs}
        assert len(on_dev) == 1, "all particle arrays must be on the same side"
        _check(self.lib.pic_load_particles(self.h, float(q), float(m), n, *[p[0] for p in ptrs], on_dev.pop()))

    def num_particles(self):
        v = ct.c_int64()
        _check(self.lib.pic_num_particles(self.h, ct.byref(v)))
        return v.value

    def get_particles(self, out=None):
        """dict of float64 arrays x..w plus int32 id (numpy unless `out` gives device tensors)."""
        n = self.num_particles()
        if out is None:
            out = {k: np.empty(n) for k in PARTICLE_KEYS}
            out["id"] = np.empty(n, dtype=np.int32)
        ptrs = [_ptr(out.get(k)) for k in PARTICLE_KEYS + ("id",)]
        sides = {p[1] for p in ptrs if p[1] is not None}
        assert len(sides) == 1
        _check(self.lib.pic_get_particles(self.h, *[p[0] for p in ptrs], sides.pop()))
        return out

    # -- steps -------------------------------------------------------
    def gather_push(self):
        _check(self.lib.pic_gather_push(self.h))

    def deposit(self):
        _check(self.lib.pic_deposit(self.h))

    def yee_step(self):
        _check(self.lib.pic_yee_step(self.h))

    def sort_particles(self, bin_shift=0):
        """Reorder the particles: by cell (0), by runs of 2**bin_shift cells,
        or in a pseudo-random order (ORDER_RANDOM)."""
        _check(self.lib.pic_sort_particles(self.h, int(bin_shift)))

    def step(self, nsteps=1):
        _check(self.lib.pic_step(self.h, int(nsteps)))

    def set_particle_algorithms(self, pusher="boris", gather="momentum"):
        """pusher "boris" | "vay"; gather "momentum" | "energy" (conserving)."""
        pu = {"boris": 0, "vay": 1}[pusher] if isinstance(pusher, str) else int(pusher)
        ga = {"momentum": 0, "energy": 1}[gather] if isinstance(gather, str) else int(gather)
        _check(self.lib.pic_set_particle_algorithms(self.h, pu, ga))

    def set_window_plasma(self, ppc, n0, ramp_start, ramp_length):
        _check(self.lib.pic_set_window_plasma(self.h, int(ppc), float(n0), float(ramp_start), float(ramp_length)))

    def window(self):
        s, z = ct.c_int64(), ct.c_double()
        _check(self.lib.pic_get_window(self.h, ct.byref(s), ct.byref(z)))
        return {"shifts": s.value, "z_lab": z.value}

    def step_adjoint(self, nsteps, ckpt_every=20, du=None):
        """Run nsteps steps and the discrete adjoint of L = 1/2 sum(|E|^2+|B|^2) dV
        at the end.  Returns (L, dL/dA, dL/du0) with dL/du0 of shape (3, n) in
        load order (numpy, or `du` when given: a (3, n) float64 array or CUDA
        tensor that is written).  The context ends in the state after the
        steps."""
        n = self.num_particles()
        if du is None:
            du = np.empty((3, n))
        p, dev = _ptr(du)
        loss, dA = ct.c_double(), ct.c_double()
        _check(self.lib.pic_step_adjoint(self.h, int(nsteps), int(ckpt_every), ct.byref(loss), ct.byref(dA),
                                         ct.c_void_p(p), dev))
        return loss.value, dA.value, du

    # -- fields ------------------------------------------------------
    def get_field(self, which, out=None):
        w = FIELDS.index(which) if isinstance(which, str) else int(which)
        if out is None:
            out = np.empty(self.n)
        p, dev = _ptr(out)
        _check(self.lib.pic_get_field(self.h, w, p, dev))
        return out

    def get_fields(self):
        return np.stack([self.get_field(i) for i in range(9)])

    def set_field(self, which, arr):
        w = FIELDS.index(which) if isinstance(which, str) else int(which)
        if isinstance(arr, np.ndarray):
            arr = np.ascontiguousarray(arr, dtype=np.float64)
        p, dev = _ptr(arr)
        _check(self.lib.pic_set_field(self.h, w, p, dev))

    def set_fields(self, F):
        for i in range(F.shape[0]):
            self.set_field(i, F[i])

    # -- misc --------------------------------------------------------
    def set_external_drive(self, amp, k):
        _check(self.lib.pic_set_external_drive(self.h, float(amp), float(k)))

    def time(self):
        s, t = ct.c_int64(), ct.c_double()
        _check(self.lib.pic_get_time(self.h, ct.byref(s), ct.byref(t)))
        return s.value, t.value

    def diagnostics(self):
        out = (ct.c_double * 4)()
        _check(self.lib.pic_diagnostics(self.h, out))
        return {"field_energy": out[0], "kinetic_energy": out[1], "charge": out[2], "max_div_b": out[3]}

    def charge_density(self, out=None):
        """Nodal charge density of the current particles (FP64, shape (nx, ny, nz))."""
        if out is None:
            out = np.empty(self.n)
        p, dev = _ptr(out)
        _check(self.lib.pic_charge_density(self.h, p, dev))
        return out

    def continuity_mark(self):
        _check(self.lib.pic_continuity_mark(self.h))

    def continuity_residual(self):
        """max|rho^{n+1} - rho^n + dt div J| over the last step: relative to
        max|rho^n|, absolute, and max|rho^n|; the new density becomes the mark."""
        out = (ct.c_double * 3)()
        _check(self.lib.pic_continuity_residual(self.h, out))
        return {"relative": out[0], "absolute": out[1], "rho_max": out[2]}

    def set_fp64_gamma(self, gamma):
        """FP32-mixed: Lorentz factor above which the push's rotation runs in FP64 (inf: never)."""
        _check(self.lib.pic_set_fp64_gamma(self.h, float(gamma)))

    def set_gather_filter(self, passes):
        """z filter of the gathered E, B: `passes` binomial passes + one compensation pass (0: off)."""
        _check(self.lib.pic_set_gather_filter(self.h, int(passes)))

    def reserve_adjoint(self, nsteps, ckpt_every=20):
        """Keep the work space of step_adjoint(nsteps, ckpt_every) (0 releases it)."""
        _check(self.lib.pic_reserve_adjoint(self.h, int(nsteps), int(ckpt_every)))

    def sync(self):
        _check(self.lib.pic_sync(self.h))

    def set_timing(self, on=True):
        _check(self.lib.pic_set_timing(self.h, 1 if on else 0))

    def get_timing(self):
        cap = 16
        names = (ct.c_char_p * cap)()
        ms = (ct.c_double * cap)()
        cnt = (ct.c_int64 * cap)()
        n = ct.c_int32()
        _check(self.lib.pic_get_timing(self.h, cap, names, ms, cnt, ct.byref(n)))
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(n.value, cap))}

    def launch_count(self):
        v = ct.c_int64()
        _check(self.lib.pic_launch_count(self.h, ct.byref(v)))
        return v.value


class Batch:
    """Many independent periodic boxes stepped together (pic_batch_*): per box
    extents, shape order and cell size; one dt."""

    def __init__(self, ns, orders, d=None, dt=0.0, cfl=0.99, precision=FP32_MIXED, stream=None):
        self.lib = load_library()
        self.nboxes = len(ns)
        n_arr = np.ascontiguousarray(np.asarray(ns, dtype=np.int32).reshape(self.nboxes, 3))
        o_arr = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(self.nboxes))
        d_arr = None if d is None else np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(self.nboxes, 3))
        self.ns = [tuple(int(v) for v in r) for r in n_arr]
        s = None
        if stream is not None:
            s = ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = ct.c_void_p()
        self.h = None
        _check(self.lib.pic_batch_init(self.nboxes, n_arr.ctypes.data, None if d_arr is None else d_arr.ctypes.data,
                                       o_arr.ctypes.data, float(dt), float(cfl), int(precision), s, ct.byref(h)))
        self.h = h

    def close(self):
        if self.h is not None:
            self.lib.pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load_particles(self, q, m, parts, counts):
        """parts: dict of concatenated arrays (box order), counts: per-box sizes."""
        counts = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
        assert counts.size == self.nboxes
        ptrs = [_ptr(parts[k]) for k in PARTICLE_KEYS]
        on_dev = {p[1] for p in ptrs}
        assert len(on_dev) == 1, "all particle arrays must be on the same side"
        _check(self.lib.pic_batch_load_particles(self.h, float(q), float(m), counts.ctypes.data,
                                                 *[p[0] for p in ptrs], on_dev.pop()))

    def step(self, nsteps=1):
        _check(self.lib.pic_batch_step(self.h, int(nsteps)))

    def info(self, box=-1):
        n, c, st, dt = ct.c_int64(), ct.c_int64(), ct.c_int64(), ct.c_double()
        _check(self.lib.pic_batch_info(self.h, int(box), ct.byref(n), ct.byref(c), ct.byref(st), ct.byref(dt)))
        return {"particles": n.value, "cells": c.value, "steps": st.value, "dt": dt.value}

    def get_field(self, box, which, out=None):
        w = FIELDS.index(which) if isinstance(which, str) else int(which)
        if out is None:
            out = np.empty(self.ns[box])
        p, dev = _ptr(out)
        _check(self.lib.pic_batch_get_field(self.h, int(box), w, ct.c_void_p(p), dev))
        return out

    def get_fields(self, box):
        return np.stack([self.get_field(box, i) for i in range(9)])

    def set_field(self, box, which, arr):
        w = FIELDS.index(which) if isinstance(which, str) else int(which)
        a = np.ascontiguousarray(arr, dtype=np.float64) if isinstance(arr, np.ndarray) else arr
        p, dev = _ptr(a)
        _check(self.lib.pic_batch_set_field(self.h, int(box), w, ct.c_void_p(p), dev))

    def set_fields(self, box, F):
        for i in range(F.shape[0]):
            self.set_field(box, i, F[i])

    def get_particles(self, box):
        n = self.info(box)["particles"]
        out = {k: np.empty(n) for k in PARTICLE_KEYS}
        out["id"] = np.empty(n, dtype=np.int32)
        ptrs = [out[k].ctypes.data for k in PARTICLE_KEYS + ("id",)]
        _check(self.lib.pic_batch_get_particles(self.h, int(box), *ptrs, 0))
        return out

    def diagnostics(self, box):
        out = (ct.c_double * 4)()
        _check(self.lib.pic_batch_diagnostics(self.h, int(box), out))
        return {"field_energy": out[0], "kinetic_energy": out[1], "charge": out[2], "max_div_b": out[3]}

    def set_tuning(self, tile=(8, 8, 8), run=0, sort_every=1):
        t = BatchTuning()
        for a in range(3):
            t.tile[a] = int(tile[a])
        t.run, t.sort_every = int(run), int(sort_every)
        _check(self.lib.pic_batch_set_tuning(self.h, ct.byref(t)))

    def get_tuning(self):
        t = BatchTuning()
        _check(self.lib.pic_batch_get_tuning(self.h, ct.byref(t)))
        return {"tile": tuple(t.tile), "run": t.run, "sort_every": t.sort_every}

    def autotune(self, trial_steps=3):
        t, ms = BatchTuning(), ct.c_double()
        _check(self.lib.pic_batch_autotune(self.h, int(trial_steps), ct.byref(t), ct.byref(ms)))
        return {"tile": tuple(t.tile), "run": t.run, "sort_every": t.sort_every}, ms.value

    def launch_count(self):
        v = ct.c_int64()
        _check(self.lib.pic_batch_launch_count(self.h, ct.byref(v)))
        return v.value


def measure_fma_peak(precision):
    """Measured FMA throughput of the current device in TFLOP/s (FP32_MIXED: FP32, FP64: FP64)."""
    lib = load_library()
    out = ct.c_double()
    _check(lib.pic_measure_fma_peak(int(precision), ct.byref(out)))
    return out.value


def sort_keys_noalloc(keys, nbins, offsets, perm, stream=None):
    """pic_sort_keys_noalloc on device int32 tensors: offsets (nbins+1) and
    perm (len(keys)) are written.  The call allocates no device memory."""
    lib = load_library()
    n = int(keys.numel())
    s = None
    if stream is not None:
        s = ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.pic_sort_keys_noalloc(ct.c_void_p(keys.data_ptr()), n, int(nbins), ct.c_void_p(offsets.data_ptr()),
                                     ct.c_void_p(perm.data_ptr()), s))
