"""The oracle's CKC field solver (cubic cells) against what fixes it (CPU):
the vacuum dispersion closed form for oblique modes, stability at Courant
number one where Yee diverges, and identity with Yee for fields that vary
along one axis only (the transverse weights sum to one)."""
import numpy as np
import pytest

import pins_lib
from oracle import Oracle


@pytest.fixture(scope="module")
def O():
    return Oracle()


def test_oblique_mode_dispersion(O):
    pins_lib.pin_ckc_oblique_mode(O)


def test_stable_at_courant_one(O):
    pins_lib.pin_ckc_stable_at_courant_one(O)


def test_yee_modes_match_their_own_closed_form(O):
    """The same machinery with the Yee symbol (no transverse factor) at dt
    below the Yee limit: the check itself discriminates the two solvers."""
    E, E0, c = pins_lib._ckc_mode(O, (8, 6, 10), (1.0, 1.0, 1.0), (2, 1, 3), 17, 0.5, solver=0)
    assert np.max(np.abs(E - c * E0)) < 1e-11
    E1, E01, c1 = pins_lib._ckc_mode(O, (8, 6, 10), (1.0, 1.0, 1.0), (2, 1, 3), 17, 0.5, solver=1)
    assert np.max(np.abs(E1 - c1 * E01)) < 1e-11 and abs(c - c1) > 1e-3


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_one_axis_fields_match_yee(O, axis):
    n = (6, 7, 8)
    g = O.grid(n)
    rng = np.random.default_rng(axis)
    F = np.zeros((9,) + n)
    shape = [1, 1, 1]
    shape[axis] = n[axis]
    for c in range(6):
        F[c] = np.broadcast_to(rng.uniform(-1, 1, n[axis]).reshape(shape), n)
    A, B = F.copy(), F.copy()
    for _ in range(5):
        O.yee_step(g, 0.5, A, solver=1)
        O.yee_step(g, 0.5, B, solver=0)
    assert np.max(np.abs(A - B)) < 1e-14
