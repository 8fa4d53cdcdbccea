"""Vay pusher and energy-conserving gather (pic_set_particle_algorithms)
through the C-ABI against the FP64 oracle with the same options: one step at
1e-12 for every order and combination (fused tile kernel and split API), ten
steps with a sort every third step (outsider path) at 1e-11, the moving-window
run at 1e-9, FP32-mixed within the single-step bounds; a relativistic E x B
drift stays put under Vay on the GPU too."""
import numpy as np
import pytest

from gpu_helpers import Case
from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu

COMBOS = [(1, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("pusher,gather", COMBOS)
@pytest.mark.parametrize("p", [1, 2, 3])
def test_fp64_one_step(p, pusher, gather):
    c = Case((16, 8, 24), p, 3, 0.6, 80 + p, field_scale=0.1, pusher=pusher, gather=gather)
    c.ctx.step(1)
    c.oracle_steps(1)
    e = c.errors()
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("pusher,gather", COMBOS)
def test_fp64_split_api(pusher, gather):
    c = Case((12, 20, 8), 3, 2, 0.5, 90, d=(1.0, 0.9, 1.1), field_scale=0.1, pusher=pusher, gather=gather)
    c.ctx.gather_push()
    c.ctx.deposit()
    c.ctx.yee_step()
    c.oracle_steps(1)
    e = c.errors()
    assert max(e.values()) < 1e-12, e


def test_fp64_ten_steps_with_outsiders():
    c = Case((16, 16, 8), 2, 4, 0.5, 95, field_scale=0.05, sort_every=3, pusher=1, gather=1)
    c.ctx.step(10)
    c.oracle_steps(10)
    e = c.errors()
    assert max(e.values()) < 1e-11, e


@pytest.mark.parametrize("p", [1, 3])
def test_fp32_mixed_one_step(p):
    c = Case((16, 16, 16), p, 4, 0.3, 100 + p, precision=pic.FP32_MIXED, field_scale=0.05, pusher=1, gather=1)
    c.ctx.step(1)
    c.oracle_steps(1)
    e = c.errors()
    assert e["EB"] < 2e-6 and e["J"] < 2e-5 and e["pos"] < 1e-6 and e["mom"] < 2e-6, e


def test_window_run_with_vay_and_energy_gather():
    from oracle import Oracle
    cfg = inputs.WAKEFIELD_SMALL
    n = cfg["n"]
    with pic.Context(n, cfl=cfg["cfl"], order=cfg["order"], window_speed=cfg["speed"]) as c:
        c.set_particle_algorithms("vay", "energy")
        c.set_window_plasma(cfg["ppc"], inputs.wakefield_plasma_density(cfg), cfg["ramp_start"], cfg["ramp_length"])
        c.set_fields(inputs.laser_fields(cfg))
        parts = inputs.wakefield_particles(cfg)
        c.load_particles(-1.0, 1.0, parts)
        c.step(40)
        G = c.get_fields()
        q = c.get_particles()
    O = Oracle()
    g = O.grid(n, zopen=True)
    dt = inputs.dt_from_cfl((1, 1, 1), cfg["cfl"])
    P = {k: v.copy() for k, v in parts.items()}
    P["id"] = np.arange(parts["x"].size, dtype=np.int64)
    F = inputs.laser_fields(cfg)
    win = dict(step=0, shifts=0, speed=cfg["speed"], next_id=parts["x"].size, ppc=cfg["ppc"],
               n0=inputs.wakefield_plasma_density(cfg), ramp_start=cfg["ramp_start"],
               ramp_length=cfg["ramp_length"], pusher=1, gather=1)
    for _ in range(40):
        P = O.window_step(g, cfg["order"], dt, -1.0, 1.0, P, F, win)
    assert np.linalg.norm(G[:6] - F[:6]) < 1e-9 * np.linalg.norm(F[:6])
    o, r = np.argsort(q["id"]), np.argsort(P["id"])
    assert np.array_equal(q["id"][o].astype(np.int64), P["id"][r])
    for k in ("ux", "uy", "uz"):
        assert np.linalg.norm(q[k][o] - P[k][r]) < 1e-9 * np.linalg.norm(P[k][r]), k


def test_vay_keeps_a_relativistic_drift_on_the_gpu():
    """Uniform crossed fields with E = -v x B for gamma = 10: particles loaded
    on the drift keep their momentum under Vay (to rounding) and leave it
    under Boris."""
    n = (8, 8, 8)
    B = np.array([0.0, 0.0, 0.8])
    u = np.array([9.9, 0.0, 0.0])
    v = u / np.sqrt(1 + u @ u)
    E = -np.cross(v, B)
    F = np.zeros((9,) + n)
    for a in range(3):
        F[a] = E[a]
        F[3 + a] = B[a]
    parts = {"x": np.array([1.3, 4.6]), "y": np.array([2.2, 5.1]), "z": np.array([3.7, 0.4]),
             "ux": np.full(2, u[0]), "uy": np.zeros(2), "uz": np.zeros(2), "w": np.full(2, 1e-9)}
    got = {}
    for name, pusher in (("vay", 1), ("boris", 0)):
        with pic.Context(n, order=2) as c:
            c.set_fields(F)
            c.load_particles(-1.0, 1.0, parts)
            c.set_particle_algorithms(pusher, 0)
            c.gather_push()
            q = c.get_particles()
            got[name] = np.stack([q["ux"], q["uy"], q["uz"]], 1)
    assert np.max(np.abs(got["vay"] - u)) < 1e-12 * 10
    assert np.max(np.abs(got["boris"] - u)) > 1e-6


def test_algorithm_choice_checks():
    with pic.Context((8, 8, 8), order=1) as c:
        with pytest.raises(pic.PicError) as e:
            c.set_particle_algorithms(2, 0)
        assert e.value.status == pic.PIC_ERR_ARG
        c.load_particles(-1.0, 1.0, inputs.uniform_plasma(1, (8, 8, 8), 1, sigma_u=0.1))
        c.set_particle_algorithms("vay", "momentum")
        with pytest.raises(pic.PicError) as e:
            c.step_adjoint(2, 1)
        assert e.value.status == pic.PIC_ERR_STATE
        c.set_particle_algorithms("boris", "momentum")
        c.step_adjoint(2, 1)
