"""CKC field solver (pic_grid_desc.solver = 1) through the C-ABI against the
FP64 oracle: particles and fields at dt = 0.95 dx (beyond the Yee limit
dx/sqrt 3) for one step at 1e-12 and twenty steps at 1e-10 for every order,
with Vay and the energy-conserving gather too; the moving window with CKC at
1e-9; FP32-mixed within its single-step bounds."""
import numpy as np
import pytest

from gpu_helpers import compare_particles, rel_l2
from oracle import Oracle
from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu

DT = 0.95


def _run(n, p, ppc, steps, seed, precision=pic.FP64, pusher=0, gather=0, field_scale=0.1):
    parts = inputs.uniform_plasma(seed, n, ppc, sigma_u=0.4)
    F = np.zeros((9,) + n)
    F[:6] = inputs.random_fields(seed + 1000, n, field_scale)[:6]
    with pic.Context(n, dt=DT, order=p, precision=precision, solver="ckc") as c:
        c.set_fields(F)
        c.load_particles(-1.0, 1.0, parts)
        if pusher or gather:
            c.set_particle_algorithms(pusher, gather)
        c.step(steps)
        G, q = c.get_fields(), c.get_particles()
    O = Oracle()
    g = O.grid(n)
    P = {k: v.copy() for k, v in parts.items()}
    for s in range(steps):
        O.pic_step(g, p, DT, -1.0, 1.0, P, F, 0.0, 0.0, s * DT, pusher=pusher, gather=gather, solver=1)
    ep, eu = compare_particles(q, P, [float(v) for v in n])
    return {"EB": rel_l2(G[:6], F[:6]), "J": rel_l2(G[6:], F[6:]), "pos": ep, "mom": eu}


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fp64_one_step(p):
    e = _run((16, 8, 24), p, 3, 1, 110 + p)
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("p", [1, 3])
def test_fp64_twenty_steps(p):
    e = _run((16, 16, 16), p, 2, 20, 120 + p, field_scale=0.02)
    assert max(e.values()) < 1e-10, e


def test_fp64_with_vay_and_energy_gather():
    e = _run((16, 8, 16), 2, 2, 10, 130, pusher=1, gather=1, field_scale=0.02)
    assert max(e.values()) < 1e-11, e


def test_fp32_mixed_one_step():
    e = _run((16, 16, 16), 3, 4, 1, 140, precision=pic.FP32_MIXED, field_scale=0.05)
    assert e["EB"] < 2e-6 and e["J"] < 2e-5 and e["pos"] < 1e-6 and e["mom"] < 2e-6, e


def test_window_run_with_ckc():
    cfg = inputs.WAKEFIELD_SMALL
    n = cfg["n"]
    with pic.Context(n, dt=DT, order=cfg["order"], window_speed=cfg["speed"], solver="ckc") as c:
        c.set_window_plasma(cfg["ppc"], inputs.wakefield_plasma_density(cfg), cfg["ramp_start"], cfg["ramp_length"])
        c.set_fields(inputs.laser_fields(cfg))
        parts = inputs.wakefield_particles(cfg)
        c.load_particles(-1.0, 1.0, parts)
        c.step(30)
        G = c.get_fields()
        q = c.get_particles()
    O = Oracle()
    g = O.grid(n, zopen=True)
    P = {k: v.copy() for k, v in parts.items()}
    P["id"] = np.arange(parts["x"].size, dtype=np.int64)
    F = inputs.laser_fields(cfg)
    win = dict(step=0, shifts=0, speed=cfg["speed"], next_id=parts["x"].size, ppc=cfg["ppc"],
               n0=inputs.wakefield_plasma_density(cfg), ramp_start=cfg["ramp_start"],
               ramp_length=cfg["ramp_length"], solver=1)
    for _ in range(30):
        P = O.window_step(g, cfg["order"], DT, -1.0, 1.0, P, F, win)
    assert win["shifts"] == 28
    assert rel_l2(G[:6], F[:6]) < 1e-9
    o, r = np.argsort(q["id"]), np.argsort(P["id"])
    assert np.array_equal(q["id"][o].astype(np.int64), P["id"][r])
    for k in ("ux", "uz", "z"):
        assert np.linalg.norm(q[k][o] - P[k][r]) < 1e-9 * np.linalg.norm(P[k][r]), k
