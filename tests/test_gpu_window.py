"""Moving window (laser-wakefield-shaped run) through the C-ABI against the
FP64 oracle's window step: the 16 x 16 x 64 copy of the recipe (laser with
a0 = 2, ramped lattice plasma, window at c), FP64 1e-12 after one and two
steps (the second shifts the window and injects), 1e-9 after 60 steps (34
shifts, rear removal); particle ids identical; FP32-mixed error stated.  At
the full 128 x 128 x 1024 size: sampled particles after one step against the
oracle, and particle bookkeeping over 20 steps."""
import numpy as np
import pytest

from gpu_helpers import rel_l2
from oracle import Oracle
from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu

CFG = inputs.WAKEFIELD_SMALL


def _gpu(cfg, precision=pic.FP64):
    n = cfg["n"]
    c = pic.Context(n, cfl=cfg["cfl"], order=cfg["order"], precision=precision, window_speed=cfg["speed"])
    c.set_window_plasma(cfg["ppc"], inputs.wakefield_plasma_density(cfg), cfg["ramp_start"], cfg["ramp_length"])
    c.set_fields(inputs.laser_fields(cfg))
    parts = inputs.wakefield_particles(cfg)
    c.load_particles(-1.0, 1.0, parts)
    return c, parts


def _oracle(cfg, parts, steps):
    O = Oracle()
    n = cfg["n"]
    g = O.grid(n, zopen=True)
    dt = inputs.dt_from_cfl((1.0, 1.0, 1.0), cfg["cfl"])
    P = {k: v.copy() for k, v in parts.items()}
    P["id"] = np.arange(parts["x"].size, dtype=np.int64)
    F = inputs.laser_fields(cfg)
    win = dict(step=0, shifts=0, speed=cfg["speed"], next_id=parts["x"].size, ppc=cfg["ppc"],
               n0=inputs.wakefield_plasma_density(cfg), ramp_start=cfg["ramp_start"],
               ramp_length=cfg["ramp_length"])
    for _ in range(steps):
        P = O.window_step(g, cfg["order"], dt, -1.0, 1.0, P, F, win)
    return P, F, win


def _compare(c, P, F, n):
    G = c.get_fields()
    q = c.get_particles()
    o = np.argsort(q["id"])
    q = {k: v[o] for k, v in q.items()}
    r = np.argsort(P["id"])
    P = {k: v[r] for k, v in P.items()}
    assert np.array_equal(q["id"].astype(np.int64), P["id"]), "particle sets differ"
    L = [float(n[0]), float(n[1])]
    pos = np.concatenate([(q[k] - P[k] + 0.5 * L[a]) % L[a] - 0.5 * L[a] for a, k in enumerate(("x", "y"))] +
                         [q["z"] - P["z"]])
    pos_ref = np.concatenate([P[k] for k in ("x", "y", "z")])
    mom = np.concatenate([q[k] - P[k] for k in ("ux", "uy", "uz")])
    mom_ref = np.concatenate([P[k] for k in ("ux", "uy", "uz")])
    return {"EB": rel_l2(G[:6], F[:6]), "J": rel_l2(G[6:], F[6:]),
            "pos": float(np.linalg.norm(pos) / np.linalg.norm(pos_ref)),
            "mom": float(np.linalg.norm(mom) / max(np.linalg.norm(mom_ref), 1e-300))}


@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (2, 1e-12), (60, 1e-9)])
def test_fp64_window_matches_oracle(steps, tol):
    c, parts = _gpu(CFG)
    c.step(steps)
    P, F, win = _oracle(CFG, parts, steps)
    assert c.window()["shifts"] == win["shifts"] == int(np.floor(c.time()[1]))
    assert c.num_particles() == P["x"].size
    e = _compare(c, P, F, CFG["n"])
    assert max(e.values()) < tol, e
    c.close()


def test_window_run_injects_and_removes():
    """After 60 steps the window has moved 34 cells: the plasma that started at
    z = 24 has reached the rear (particles removed), and 34 slabs came in."""
    c, parts = _gpu(CFG)
    c.step(60)
    P, F, win = _oracle(CFG, parts, 60)
    ids = P["id"]
    n0 = parts["x"].size
    assert np.sum(ids >= n0) == 34 * 16 * 16 * CFG["ppc"]         # every injected particle is alive
    assert np.sum(ids < n0) < n0                                    # some loaded ones were removed
    assert c.num_particles() == ids.size
    c.close()


def test_fp32_mixed_window_error_stated():
    c, parts = _gpu(CFG, pic.FP32_MIXED)
    c.step(60)
    P, F, _ = _oracle(CFG, parts, 60)
    e = _compare(c, P, F, CFG["n"])
    print("FP32-mixed window run, 60 steps:", e)
    # measured on GB300: EB 4.8e-7, J 6.0e-7, pos 1.2e-8, mom 5.0e-7
    assert e["EB"] < 5e-6 and e["J"] < 6e-6 and e["pos"] < 1e-7 and e["mom"] < 5e-6, e
    c.close()


def test_window_entry_point_checks():
    n = (8, 8, 16)
    with pic.Context(n, order=1) as c:
        with pytest.raises(pic.PicError) as e:
            c.set_window_plasma(2, 1.0, 0.0, 0.0)
        assert e.value.status == pic.PIC_ERR_STATE
    with pic.Context(n, order=1, window_speed=1.0) as c:
        with pytest.raises(pic.PicError) as e:
            c.set_window_plasma(-1, 1.0, 0.0, 0.0)
        assert e.value.status == pic.PIC_ERR_ARG
        c.set_window_plasma(1, 0.5, 4.0, 0.0)
        parts = inputs.lattice_plasma(n, 1, 0.5, 4.0, 0.0)
        # a particle loaded outside z is dropped by the first sort
        parts = {k: np.concatenate([v, v[:1]]) for k, v in parts.items()}
        parts["z"][-1] = -0.5
        c.load_particles(-1.0, 1.0, parts)
        assert c.num_particles() == parts["x"].size - 1
        with pytest.raises(pic.PicError) as e:
            c.set_window_plasma(1, 0.5, 4.0, 0.0)
        assert e.value.status == pic.PIC_ERR_STATE
        with pytest.raises(pic.PicError) as e:
            c.gather_push()
        assert e.value.status == pic.PIC_ERR_STATE
        with pytest.raises(pic.PicError) as e:
            c.step_adjoint(2, 1)
        assert e.value.status == pic.PIC_ERR_STATE
        c.step(4)
        assert c.window()["shifts"] == 2


def test_wakefield_full_size_sampled():
    """128 x 128 x 1024, FP32-mixed: after one step, 4096 sampled particles
    against the oracle's own step of those particles in the same initial
    fields (gather, push and advance are per particle); over 20 steps the
    particle count follows the window's bookkeeping exactly (11 slabs of
    plateau plasma in, nothing at the rear to remove) and max |div B| stays
    at its initial value."""
    cfg = inputs.WAKEFIELD
    c, parts = _gpu(cfg, pic.FP32_MIXED)
    N0 = parts["x"].size
    divb0 = c.diagnostics()["max_div_b"]  # the paraxial pulse is not divergence-free; Yee keeps div B
    c.step(1)
    q = c.get_particles()
    sel = inputs.uniform(7, 0, 4096, 0)
    ids = np.unique((sel * N0).astype(np.int64))
    o = np.argsort(q["id"])
    got = {k: v[o][ids] for k, v in q.items()}
    O = Oracle()
    g = O.grid(cfg["n"], zopen=True)
    P = {k: np.ascontiguousarray(v[ids]) for k, v in parts.items()}
    F = inputs.laser_fields(cfg)
    O.pic_step(g, cfg["order"], inputs.dt_from_cfl((1, 1, 1), cfg["cfl"]), -1.0, 1.0, P, F)
    for k in ("x", "y", "z"):
        assert np.max(np.abs(got[k] - P[k])) < 2e-5, k
    for k in ("ux", "uy", "uz"):
        scale = max(np.max(np.abs(P[k])), 1e-6)
        assert np.max(np.abs(got[k] - P[k])) < 2e-5 * scale + 1e-7, k
    c.step(19)
    shifts = c.window()["shifts"]
    assert shifts == int(np.floor(c.time()[1]))
    slab = cfg["n"][0] * cfg["n"][1] * cfg["ppc"]
    assert c.num_particles() == N0 + shifts * slab
    d = c.diagnostics()
    assert abs(d["max_div_b"] - divb0) < 1e-3 * divb0
    c.close()


def test_particle_buffers_grow_when_the_box_overfills():
    """Plasma that travels with the window (u_z = 50, v = 0.9998 c) stays in
    the box while every shift injects a new front slab, so the live count
    passes the buffers sized at load (a full box plus two slabs): the step
    grows them, keeps every particle, and still matches the oracle."""
    cfg = CFG
    n = cfg["n"]
    parts = inputs.uniform_plasma(31, n, cfg["ppc"], sigma_u=0.0)
    parts["uz"][:] = 50.0
    c = pic.Context(n, cfl=cfg["cfl"], order=cfg["order"], precision=pic.FP64, window_speed=cfg["speed"])
    c.set_window_plasma(cfg["ppc"], inputs.wakefield_plasma_density(cfg), cfg["ramp_start"], cfg["ramp_length"])
    c.set_fields(inputs.laser_fields(cfg))
    c.load_particles(-1.0, 1.0, parts)
    steps = 14
    c.step(steps)
    P, F, win = _oracle(cfg, parts, steps)
    slab = n[0] * n[1] * cfg["ppc"]
    assert c.num_particles() > n[0] * n[1] * n[2] * cfg["ppc"] + 2 * slab
    e = _compare(c, P, F, n)
    assert max(e.values()) < 1e-12, e
    c.close()
