"""The z filter of the gathered fields (the Godfrey filter of the paper's
plasma-acceleration run, Sec. 4.2, in its compensated binomial form) on the
GPU against the oracle's filtered step: periodic plasmas with random fields
at every order (FP64 1e-12 after one step, 1e-9 after ten; FP32-mixed
stated), the paper's combination for that run (Vay pusher, energy-conserving
gather, CKC solver), and the moving window (zero beyond the z ends)."""
import numpy as np
import pytest

from gpu_helpers import compare_particles, rel_l2
from oracle import Oracle
from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu


def _run(n, order, npass, steps, precision, pusher=0, gather=0, solver=0, dt=None, seed=80):
    d = (1.0, 1.0, 1.0)
    dt = inputs.dt_from_cfl(d, 0.99) if dt is None else dt
    parts = inputs.uniform_plasma(seed, n, 2, sigma_u=0.2)
    F = np.zeros((9,) + n)
    F[:6] = inputs.random_fields(seed + 1, n, 0.1)[:6]
    with pic.Context(n, dt=dt, order=order, precision=precision, solver="ckc" if solver else "yee") as c:
        c.set_fields(F)
        c.load_particles(-1.0, 1.0, parts)
        if pusher or gather:
            c.set_particle_algorithms(pusher, gather)
        c.set_gather_filter(npass)
        c.step(steps)
        G = c.get_fields()
        q = c.get_particles()
    O = Oracle()
    g = O.grid(n)
    ref = {k: v.copy() for k, v in parts.items()}
    Fr = F.copy()
    for s in range(steps):
        O.pic_step(g, order, dt, -1.0, 1.0, ref, Fr, 0.0, 0.0, s * dt, pusher=pusher, gather=gather,
                   solver=solver, filter_passes=npass)
    ep, eu = compare_particles(q, ref, [float(v) for v in n])
    return {"EB": rel_l2(G[:6], Fr[:6]), "J": rel_l2(G[6:], Fr[6:]), "pos": ep, "mom": eu}


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (10, 1e-9)])
def test_filtered_step_fp64(order, steps, tol):
    e = _run((8, 8, 32), order, 2, steps, pic.FP64)
    assert max(e.values()) < tol, e


def test_filtered_step_fp32_mixed_stated():
    e = _run((8, 8, 32), 3, 2, 10, pic.FP32_MIXED)
    print("FP32-mixed with the z filter after 10 steps:", e)
    assert max(e.values()) < 1e-5, e


@pytest.mark.parametrize("npass", [1, 4])
def test_filtered_step_vay_energy_ckc(npass):
    """The plasma-acceleration run's options together (Sec. 4.2), CKC at dt = 0.95 dx."""
    e = _run((8, 8, 32), 3, npass, 5, pic.FP64, pusher=1, gather=1, solver=1, dt=0.95)
    assert max(e.values()) < 1e-11, e


def test_filter_off_is_the_plain_step():
    a = _run((8, 8, 32), 2, 0, 3, pic.FP64)
    assert max(a.values()) < 1e-12


def test_filtered_window_run():
    """The 16 x 16 x 64 wakefield copy with the window moving and the filter
    on (zero beyond the z ends): FP64 against the oracle's window step."""
    cfg = inputs.WAKEFIELD_SMALL
    n = cfg["n"]
    n0 = inputs.wakefield_plasma_density(cfg)
    parts = inputs.wakefield_particles(cfg)
    steps = 12
    with pic.Context(n, cfl=cfg["cfl"], order=cfg["order"], precision=pic.FP64, window_speed=cfg["speed"]) as c:
        c.set_window_plasma(cfg["ppc"], n0, cfg["ramp_start"], cfg["ramp_length"])
        c.set_fields(inputs.laser_fields(cfg))
        c.load_particles(-1.0, 1.0, parts)
        c.set_gather_filter(3)
        c.step(steps)
        G = c.get_fields()
        q = c.get_particles()
    O = Oracle()
    g = O.grid(n, zopen=True)
    dt = inputs.dt_from_cfl((1.0, 1.0, 1.0), cfg["cfl"])
    P = {k: v.copy() for k, v in parts.items()}
    P["id"] = np.arange(parts["x"].size, dtype=np.int64)
    F = inputs.laser_fields(cfg)
    win = dict(step=0, shifts=0, speed=cfg["speed"], next_id=parts["x"].size, ppc=cfg["ppc"], n0=n0,
               ramp_start=cfg["ramp_start"], ramp_length=cfg["ramp_length"], filter_passes=3)
    for _ in range(steps):
        P = O.window_step(g, cfg["order"], dt, -1.0, 1.0, P, F, win)
    assert rel_l2(G[:6], F[:6]) < 1e-11
    o, r = np.argsort(q["id"]), np.argsort(P["id"])
    assert np.array_equal(q["id"][o].astype(np.int64), P["id"][r])
    assert rel_l2(np.concatenate([q[k][o] for k in ("ux", "uy", "uz")]),
                  np.concatenate([P[k][r] for k in ("ux", "uy", "uz")])) < 1e-11


def test_filter_argument_checks():
    with pic.Context((8, 8, 8), cfl=0.99, order=1) as c:
        with pytest.raises(pic.PicError):
            c.set_gather_filter(-1)
        with pytest.raises(pic.PicError):
            c.set_gather_filter(17)
        c.load_particles(-1.0, 1.0, inputs.uniform_plasma(1, (8, 8, 8), 1, sigma_u=0.1))
        c.set_gather_filter(2)
        with pytest.raises(pic.PicError) as ei:
            c.step_adjoint(2, 1)
        assert ei.value.status == pic.PIC_ERR_STATE
