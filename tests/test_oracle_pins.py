"""The FP64 CPU oracle against what the mathematics fixes (CPU only)."""
import numpy as np
import pytest
from scipy.optimize import curve_fit

import pins_lib
from oracle import Oracle
from paper_2101_12149_gb300 import inputs


@pytest.fixture(scope="module")
def O():
    return Oracle()


@pytest.mark.parametrize("pin", pins_lib.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(O, pin):
    pin(O)


def _lattice_plasma(n, per_axis, amp, k):
    """Quiet start: per_axis^3 particles per cell on a regular sub-lattice,
    cold, u_x = amp sin(k x); density 1."""
    o = (np.arange(per_axis) + 0.5) / per_axis
    idx = np.indices(n).reshape(3, -1).T
    offs = np.array(np.meshgrid(o, o, o, indexing="ij")).reshape(3, -1).T
    pos = (idx[:, None, :] + offs[None, :, :]).reshape(-1, 3)
    N = pos.shape[0]
    return dict(x=pos[:, 0].copy(), y=pos[:, 1].copy(), z=pos[:, 2].copy(),
                ux=amp * np.sin(k * pos[:, 0]), uy=np.zeros(N), uz=np.zeros(N),
                w=np.full(N, 1.0 / per_axis ** 3))


def _fit_mode_frequency(O, n, p, parts, dt, steps, k):
    g = O.grid(n)
    F = np.zeros((9,) + tuple(n))
    ph = np.sin(k * (np.arange(n[0]) + 0.5))
    series = []
    for _ in range(steps):
        O.pic_step(g, p, dt, -1.0, 1.0, parts, F)
        series.append(2 * np.mean(F[0].mean(axis=(1, 2)) * ph))
    s = np.array(series)
    t = dt * np.arange(1, steps + 1)
    f = lambda t, A, om, phi, B: A * np.cos(om * t + phi) + B  # noqa: E731
    popt, _ = curve_fit(f, t, s, p0=[np.max(np.abs(s)), 1.0, 0.0, 0.0])
    return popt[1]


def _omega_pred(dt, k, p):
    """Cold-plasma Langmuir frequency of the leapfrog scheme with a momentum-
    conserving order-p gather (Fourier transfer sinc^(p+1)) and an Esirkepov
    current of order p-1 along the mode (sinc^p):
    sin(w dt/2) = (dt/2) w_p sinc^((2p+1)/2)(k/2), w_p = 1."""
    sk = np.sin(k / 2) / (k / 2)
    return 2 / dt * np.arcsin(0.5 * dt * sk ** ((2 * p + 1) / 2))


@pytest.mark.parametrize("nx,p,per_axis,tol", [(32, 1, 2, 1e-5), (16, 1, 2, 1e-4), (32, 3, 2, 1e-5),
                                                (32, 2, 4, 1e-4)])
def test_langmuir_quiet_start(O, nx, p, per_axis, tol):
    """Langmuir oscillation of a cold quiet-start plasma at the discrete
    dispersion relation's frequency (32 and 16 cells per wavelength).  The
    even order and the shorter wavelength see a small lattice-aliasing
    shift (a few 1e-5), hence their looser bound."""
    n = (nx, 4, 4)
    k = 2 * np.pi / nx
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    parts = _lattice_plasma(n, per_axis, 1e-3, k)
    om = _fit_mode_frequency(O, n, p, parts, dt, 50, k)
    assert abs(om / _omega_pred(dt, k, p) - 1) < tol


@pytest.mark.slow
def test_langmuir_uniform_32_workload(O):
    """The 32^3, 2-particle-per-cell random thermal workload oscillates near
    w_p; random loading at 2 ppc shifts the measured mode by a few percent."""
    w = inputs.WORKLOADS["uniform_32"]
    dt = inputs.dt_from_cfl((1, 1, 1), w["cfl"])
    parts = inputs.workload_particles("uniform_32")
    om = _fit_mode_frequency(O, w["n"], 1, parts, dt, w["steps"], w["pert_k"])
    assert abs(om - 1.0) < 0.04, om


def test_continuity_full_step(O):
    """Discrete continuity over a full PIC step of a hot plasma (the same rho
    before and after, J from the step), order 3."""
    n = (8, 8, 8)
    g = O.grid(n)
    parts = inputs.uniform_plasma(3, n, 2, sigma_u=0.5)
    F = np.zeros((9,) + n)
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    r0 = O.rho(g, 3, -1.0, parts["x"], parts["y"], parts["z"], parts["w"])
    O.pic_step(g, 3, dt, -1.0, 1.0, parts, F)
    r1 = O.rho(g, 3, -1.0, parts["x"], parts["y"], parts["z"], parts["w"])
    res = r1 - r0 + dt * O.div_edge(g, F[6:9])
    assert np.max(np.abs(res)) < 1e-13 * np.max(np.abs(r0))


def test_wrap_edge_cases(O):
    """x == L maps to 0; values just below 0 wrap into [0, L)."""
    assert O.wrap(8.0, 8.0) == 0.0
    assert O.wrap(-1e-300, 8.0) == 0.0
    assert O.wrap(-0.25, 8.0) == 7.75
    assert O.wrap(8.5, 8.0) == 0.5
    v = O.wrap(-1e-17, 8.0)
    assert 0.0 <= v < 8.0
