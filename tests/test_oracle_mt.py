"""The multi-threaded CPU baseline (OpenMP, private current arrays summed in
thread order: the CPU deposition of Sec. 3.4.1) against the serial oracle
(CPU only).  Gather, push and advance are the oracle's own per-particle
arithmetic, so the particles must match bit for bit; J, E and B differ only
by the order in which the threads' currents are summed."""
import numpy as np
import pytest

from oracle import Oracle, OracleMT
from paper_2101_12149_gb300 import inputs


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("nthreads", [1, 4])
def test_mt_step_matches_serial_oracle(order, nthreads):
    n, d = (12, 8, 16), (1.0, 1.25, 0.75)
    g = Oracle.grid(n, d)
    dt = inputs.dt_from_cfl(d, 0.99)
    parts = inputs.uniform_plasma(70 + order, n, 4, d=d, sigma_u=0.3)
    F = np.zeros((9,) + n)
    F[:6] = inputs.random_fields(71, n, 0.05)[:6]
    ref_p, ref_F = {k: v.copy() for k, v in parts.items()}, F.copy()
    mt_p, mt_F = {k: v.copy() for k, v in parts.items()}, F.copy()
    O, M = Oracle(), OracleMT(nthreads)
    for s in range(3):
        O.pic_step(g, order, dt, -1.0, 1.0, ref_p, ref_F, 0.01, 2 * np.pi / n[0], s * dt)
        M.pic_step(g, order, dt, -1.0, 1.0, mt_p, mt_F, 0.01, 2 * np.pi / n[0], s * dt)
        if s == 0:
            # after one step the particles are bit for bit the oracle's
            for k in ("x", "y", "z", "ux", "uy", "uz"):
                assert np.array_equal(mt_p[k], ref_p[k]), k
            assert _rel(mt_F[6:], ref_F[6:]) < 1e-13
            assert _rel(mt_F[:6], ref_F[:6]) < 1e-13
    if nthreads == 1:  # one thread sums in the oracle's order: identical
        assert np.array_equal(mt_F, ref_F)
    assert _rel(mt_F, ref_F) < 1e-12


def test_mt_vay_energy_gather():
    n = (8, 8, 16)
    g = Oracle.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    parts = inputs.uniform_plasma(75, n, 2, sigma_u=0.5)
    F = np.zeros((9,) + n)
    F[:6] = inputs.random_fields(76, n, 0.1)[:6]
    a, b = {k: v.copy() for k, v in parts.items()}, {k: v.copy() for k, v in parts.items()}
    Fa, Fb = F.copy(), F.copy()
    Oracle().pic_step(g, 2, dt, -1.0, 1.0, a, Fa, pusher=1, gather=1)
    OracleMT(3).pic_step(g, 2, dt, -1.0, 1.0, b, Fb, pusher=1, gather=1)
    for k in ("x", "y", "z", "ux", "uy", "uz"):
        assert np.array_equal(a[k], b[k])
    assert _rel(Fb, Fa) < 1e-13
