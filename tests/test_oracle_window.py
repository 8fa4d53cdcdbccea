"""The oracle's open-z boundary and moving window (wakefield run) against
what fixes them (CPU only):
  - gather / deposit with z open equal the periodic ones on a grid padded
    with zero cells along z (then cropped), for particles at both ends;
  - the Yee update with z open conserves the discrete field energy
    |E|^2 + |B|^2 - (dt/2)^2 |curl E|^2 exactly in vacuum (it does so only if
    the truncated curls stay each other's transposes), and equals the
    periodic update for fields away from the ends;
  - the boundary values of one update, worked out by hand;
  - removal, window shift and injection follow their stated recipe."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2101_12149_gb300 import inputs

PAD = 4


@pytest.fixture(scope="module")
def O():
    return Oracle()


def _rand(seed, shape, scale=1.0, draw=0):
    n = int(np.prod(shape))
    return (2 * inputs.uniform(seed, 0, n, draw) - 1).reshape(shape) * scale


def _padded(F):
    s = F.shape
    P = np.zeros(s[:-1] + (s[-1] + 2 * PAD,))
    P[..., PAD:PAD + s[-1]] = F
    return P


@pytest.mark.parametrize("p", [1, 2, 3])
def test_open_z_gather_equals_zero_padded_periodic(O, p):
    n, d = (6, 5, 9), (1.0, 0.9, 1.2)
    g = O.grid(n, d, zopen=True)
    gp = O.grid((n[0], n[1], n[2] + 2 * PAD), d)
    F = _rand(10 + p, (6,) + n)
    Lz = n[2] * d[2]
    z = np.concatenate([_rand(20, (8,), 0.5) + 0.6, Lz - 0.6 + _rand(21, (8,), 0.55)])
    x = 2.0 + _rand(22, (16,), 1.5)
    y = 2.0 + _rand(23, (16,), 1.5)
    a = O.gather(g, p, F, x, y, z)
    b = O.gather(gp, p, _padded(F), x, y, z + PAD * d[2])
    assert np.max(np.abs(a - b)) < 1e-13
    # and the ends do matter: the periodic gather differs near them
    c = O.gather(O.grid(n, d), p, F, x, y, z)
    assert np.max(np.abs(a - c)) > 1e-3


@pytest.mark.parametrize("p", [1, 2, 3])
def test_open_z_deposit_equals_zero_padded_periodic_cropped(O, p):
    n, d = (6, 5, 9), (1.0, 0.9, 1.2)
    g = O.grid(n, d, zopen=True)
    gp = O.grid((n[0], n[1], n[2] + 2 * PAD), d)
    Lz = n[2] * d[2]
    z0 = np.concatenate([0.3 + 0.25 * _rand(30, (6,)), Lz - 0.3 + 0.25 * _rand(31, (6,))])
    z1 = z0 + np.concatenate([np.full(6, -0.45), np.full(6, 0.45)]) + _rand(32, (12,), 0.04)  # across both ends
    x0, y0 = 2.5 + _rand(33, (12,)), 2.0 + _rand(34, (12,))
    x1, y1 = x0 + _rand(35, (12,), 0.4), y0 + _rand(36, (12,), 0.4)
    w = 0.5 + _rand(37, (12,), 0.3)
    dt = 0.4
    J = O.deposit(g, p, dt, -1.0, x0, y0, z0, x1, y1, z1, w)
    Jp = O.deposit(gp, p, dt, -1.0, x0, y0, z0 + PAD * d[2], x1, y1, z1 + PAD * d[2], w)
    assert np.max(np.abs(J - Jp[..., PAD:PAD + n[2]])) < 1e-13
    # current fell outside the grid and was dropped
    assert np.max(np.abs(Jp[..., :PAD])) > 1e-3 and np.max(np.abs(Jp[..., PAD + n[2]:])) > 1e-3


def _energy_invariant(O, g, dt, F):
    """|E|^2 + |B|^2 - (dt/2)^2 |curl E|^2, with curl E from one B half step."""
    B = F[3:6].copy()
    Bh = B.copy()
    E = np.ascontiguousarray(F[0:3])
    O.yee_b(g, 1.0, E, Bh)                     # Bh = B - curl E
    curlE = B - Bh
    return np.sum(F[0:3] ** 2) + np.sum(B ** 2) - (dt / 2) ** 2 * np.sum(curlE ** 2)


@pytest.mark.parametrize("zopen", [True, False])
def test_yee_conserves_discrete_energy(O, zopen):
    n, d = (5, 6, 8), (1.0, 1.1, 0.9)
    g = O.grid(n, d, zopen=zopen)
    dt = 0.95 * inputs.dt_from_cfl(d, 1.0)
    F = np.zeros((9,) + n)
    F[:6] = _rand(40, (6,) + n)
    W0 = _energy_invariant(O, g, dt, F)
    for _ in range(300):
        O.yee_step(g, dt, F)
    W1 = _energy_invariant(O, g, dt, F)
    assert abs(W1 - W0) < 1e-12 * W0, (W0, W1)


def test_yee_open_z_equals_periodic_away_from_the_ends(O):
    n = (5, 6, 12)
    F = np.zeros((9,) + n)
    F[:6, :, :, 3:9] = _rand(41, (6, 5, 6, 6))
    F[6:, :, :, 3:9] = _rand(42, (3, 5, 6, 6), 0.1)
    a, b = F.copy(), F.copy()
    O.yee_step(O.grid(n, zopen=True), 0.5, a)
    O.yee_step(O.grid(n), 0.5, b)
    assert np.array_equal(a, b)


def test_yee_open_z_boundary_values_by_hand(O):
    """E_y = 1 in the last z layer only; one B half step with h: B_x there gets
    -h * (-(0 - 1)/dz) (E_y beyond the end is zero), B_x one layer down gets
    -h * (-(1 - 0)/dz).  B_x = 1 in the first layer only; one E step with dt:
    E_y there gets dt * (B_x - 0)/dz (B_x below the start is zero)."""
    n, dz, h = (3, 3, 4), 0.8, 0.3
    g = O.grid(n, (1.0, 1.0, dz), zopen=True)
    E = np.zeros((3,) + n)
    B = np.zeros((3,) + n)
    E[1, :, :, 3] = 1.0
    O.yee_b(g, h, E, B)
    assert np.allclose(B[0, :, :, 3], -h * (-(0.0 - 1.0) / dz), rtol=0, atol=1e-15)
    assert np.allclose(B[0, :, :, 2], -h * (-(1.0 - 0.0) / dz), rtol=0, atol=1e-15)
    assert np.all(B[0, :, :, :2] == 0) and np.all(B[1:] == 0)
    E = np.zeros((3,) + n)
    B = np.zeros((3,) + n)
    B[0, :, :, 0] = 1.0
    O.yee_e(g, 0.5, E, B, np.zeros((3,) + n))
    assert np.allclose(E[1, :, :, 0], 0.5 * (1.0 - 0.0) / dz, rtol=0, atol=1e-15)
    assert np.allclose(E[1, :, :, 1], 0.5 * (0.0 - 1.0) / dz, rtol=0, atol=1e-15)
    assert np.all(E[1, :, :, 2:] == 0) and np.all(E[0] == 0) and np.all(E[2] == 0)


def test_particles_leaving_z_are_removed_and_x_y_wrap(O):
    n = (4, 4, 6)
    g = O.grid(n, zopen=True)
    parts = {"x": np.array([3.9, 1.0, 2.0]), "y": np.array([0.05, 2.0, 2.0]), "z": np.array([3.0, 5.9, 0.1]),
             "ux": np.array([0.5, 0.0, 0.0]), "uy": np.array([-0.5, 0.0, 0.0]), "uz": np.array([0.0, 1.0, -1.0]),
             "w": np.ones(3), "id": np.arange(3)}
    F = np.zeros((9,) + n)
    win = dict(step=0, shifts=0, speed=0.0, next_id=3, ppc=0, n0=0.0, ramp_start=0.0, ramp_length=0.0)
    out = O.window_step(g, 1, 0.5, -1.0, 1.0, {k: v.copy() for k, v in parts.items()}, F, win)
    assert out["id"].tolist() == [0]
    assert 0.0 <= out["x"][0] < 4.0 and 0.0 <= out["y"][0] < 4.0
    assert abs(out["x"][0] - (3.9 + 0.5 * 0.5 / np.sqrt(1.5) - 4.0)) < 1e-14


def test_window_shift_and_injection_follow_the_recipe(O):
    n, ppc = (3, 4, 8), 2
    g = O.grid(n, zopen=True)
    dt = 0.6
    F = np.zeros((9,) + n)
    F[:6] = _rand(50, (6,) + n)
    F0 = F.copy()
    parts = {"x": np.array([1.2, 2.5]), "y": np.array([1.0, 3.5]), "z": np.array([0.3, 5.0]),
             "ux": np.zeros(2), "uy": np.zeros(2), "uz": np.zeros(2), "w": np.full(2, 1e-12), "id": np.arange(2)}
    win = dict(step=1, shifts=0, speed=1.0, next_id=2, ppc=ppc, n0=0.5, ramp_start=8.5, ramp_length=2.0)
    # step 1 -> 2: t = 2 dt = 1.2 >= 1 dz: one shift
    Fs = F.copy()
    out = O.window_step(g, 1, dt, -1.0, 1.0, {k: v.copy() for k, v in parts.items()}, Fs, win)
    assert win["shifts"] == 1 and win["step"] == 2
    # the field after the step, moved down one cell, front slab zero
    Fstep = F0.copy()
    O.pic_step(g, 1, dt, -1.0, 1.0, {k: v.copy() for k, v in parts.items() if k != "id"}, Fstep, 0.0, 0.0, dt)
    assert np.array_equal(Fs[:, :, :, :-1], Fstep[:, :, :, 1:]) and np.all(Fs[:, :, :, -1] == 0)
    # the particle at z = 0.3 moved (nearly at rest) to below 0 and was removed; the other moved by -1
    assert 0 not in out["id"].tolist() and 1 in out["id"].tolist()
    # injected: slab k = 7 at lab z = (1 + 7 + (m + 1/2)/2); density 0.5 * clip((z - 8.5)/2, 0, 1)
    new = out["id"] >= 2
    zl = np.array([8.25, 8.75])                   # lab z of m = 0, 1
    dens = 0.5 * np.clip((zl - 8.5) / 2.0, 0, 1)  # 0 and 0.0625
    assert np.sum(new) == n[0] * n[1] * 1          # m = 0 has zero density, m = 1 is made
    assert np.allclose(out["w"][new], dens[1] / ppc, rtol=0, atol=1e-16)
    assert np.allclose(out["z"][new], 7.75, rtol=0, atol=1e-15)
    ids = out["id"][new]
    assert sorted(ids.tolist()) == [2 + (i * n[1] + j) * ppc + 1 for i in range(n[0]) for j in range(n[1])]
    assert win["next_id"] == 2 + n[0] * n[1] * ppc


def test_window_run_counts_shifts(O):
    """The window moves one cell whenever speed * t reaches the next cell:
    after M steps, floor(speed * M dt / dz) shifts."""
    n = (2, 2, 8)
    g = O.grid(n, zopen=True)
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    F = np.zeros((9,) + n)
    parts = {k: np.zeros(0) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
    parts["id"] = np.zeros(0, dtype=np.int64)
    win = dict(step=0, shifts=0, speed=1.0, next_id=0, ppc=1, n0=1.0, ramp_start=1e9, ramp_length=0.0)
    for m in range(1, 40):
        parts = O.window_step(g, 1, dt, -1.0, 1.0, parts, F, win)
        assert win["shifts"] == int(np.floor(m * dt))
    assert parts["x"].size == 0                    # no plasma before the ramp
