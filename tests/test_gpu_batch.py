"""Batch of independent boxes (pic_batch_*) against the FP64 CPU oracle run on
each box alone, against single-box contexts, across tunings and through the
autotuner.  Each box must compute what it computes alone: FP64 1e-12 after
one step, 1e-9 after ten; FP32-mixed within the single-box FP32 bounds."""
import numpy as np
import pytest

from gpu_helpers import compare_particles, rel_l2
from oracle import Oracle
from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu

CFL = 0.99
DT = inputs.dt_from_cfl((1.0, 1.0, 1.0), CFL)

# uneven boxes: extents that give tiles of 8, 4, 2 and 1 cells, all three orders,
# 1-3 particles per cell, densities 0.3-3
SMALL = [
    dict(n=(8, 8, 8), order=1, ppc=2, density=1.0, seed=101),
    dict(n=(16, 8, 8), order=3, ppc=1, density=3.0, seed=102),
    dict(n=(8, 12, 8), order=1, ppc=3, density=0.3, seed=103),
    dict(n=(10, 8, 8), order=3, ppc=2, density=1.5, seed=104),
    dict(n=(8, 8, 16), order=2, ppc=2, density=0.7, seed=105),
]


def _batch(boxes, precision=pic.FP64, fields=True, tuning=None, sigma_u=0.3):
    cat, counts, parts = inputs.ensemble_particles(boxes, sigma_u=sigma_u)
    b = pic.Batch([x["n"] for x in boxes], [x["order"] for x in boxes], dt=DT, precision=precision)
    b.load_particles(-1.0, 1.0, cat, counts)
    F0 = []
    for i, x in enumerate(boxes):
        F = np.zeros((9,) + x["n"])
        if fields:
            F[:6] = inputs.random_fields(x["seed"] + 5000, x["n"], 0.05)[:6]
            b.set_fields(i, F)
        F0.append(F)
    if tuning:
        b.set_tuning(**tuning)
    return b, parts, F0


def _oracle(boxes, parts, F0, steps):
    O = Oracle()
    out = []
    for x, p, F in zip(boxes, parts, F0):
        g = O.grid(x["n"])
        P = {k: v.copy() for k, v in p.items()}
        G = F.copy()
        for s in range(steps):
            O.pic_step(g, x["order"], DT, -1.0, 1.0, P, G, 0.0, 0.0, s * DT)
        out.append((P, G))
    return out


def _errors(b, i, x, ref):
    P, G = ref
    F = b.get_fields(i)
    ep, eu = compare_particles(b.get_particles(i), P, [float(v) for v in x["n"]])
    return {"EB": rel_l2(F[:6], G[:6]), "J": rel_l2(F[6:], G[6:]), "pos": ep, "mom": eu}


@pytest.mark.parametrize("steps,tol", [(1, 1e-12), (10, 1e-9)])
def test_fp64_batch_matches_oracle_per_box(steps, tol):
    b, parts, F0 = _batch(SMALL)
    b.step(steps)
    ref = _oracle(SMALL, parts, F0, steps)
    for i, x in enumerate(SMALL):
        e = _errors(b, i, x, ref[i])
        assert max(e.values()) < tol, (i, e)
    assert b.info()["steps"] == steps
    b.close()


def test_fp32_mixed_batch_one_step_within_single_box_bounds():
    b, parts, F0 = _batch(SMALL, precision=pic.FP32_MIXED)
    b.step(1)
    ref = _oracle(SMALL, parts, F0, 1)
    for i, x in enumerate(SMALL):
        e = _errors(b, i, x, ref[i])
        assert e["EB"] < 2e-6 and e["J"] < 2e-5 and e["pos"] < 1e-6 and e["mom"] < 2e-6, (i, e)
    b.close()


@pytest.mark.parametrize("tuning", [
    dict(tile=(4, 4, 4), run=1, sort_every=1),
    dict(tile=(8, 4, 2), run=4, sort_every=3),     # outsiders between sorts
    dict(tile=(1, 1, 1), run=0, sort_every=2),
])
def test_tunings_do_not_change_fp64_results(tuning):
    ref_b, _, _ = _batch(SMALL)
    ref_b.step(8)
    b, _, _ = _batch(SMALL, tuning=tuning)
    assert b.get_tuning() == {"tile": tuning["tile"], "run": tuning["run"], "sort_every": tuning["sort_every"]}
    b.step(8)
    for i, x in enumerate(SMALL):
        F, Fr = b.get_fields(i), ref_b.get_fields(i)
        assert rel_l2(F[:6], Fr[:6]) < 1e-12, (i, tuning)
        ep, eu = compare_particles(b.get_particles(i), _sorted(ref_b.get_particles(i)), [float(v) for v in x["n"]])
        assert ep < 1e-12 and eu < 1e-12, (i, tuning)
    b.close()
    ref_b.close()


def _sorted(parts):
    o = np.argsort(parts["id"])
    return {k: v[o] for k, v in parts.items()}


def test_each_box_equals_its_single_box_context():
    """FP32-mixed: a box in the batch and the same box in its own context take
    the same arithmetic (tiles 8^3 in both); only float atomic order differs."""
    boxes = SMALL[:2] + SMALL[4:]
    b, parts, F0 = _batch(boxes, precision=pic.FP32_MIXED)
    b.step(5)
    for i, x in enumerate(boxes):
        c = pic.Context(x["n"], dt=DT, precision=pic.FP32_MIXED, order=x["order"], tile=(8, 8, 8))
        c.set_fields(F0[i])
        c.load_particles(-1.0, 1.0, parts[i])
        c.step(5)
        Fb, Fc = b.get_fields(i), c.get_fields()
        assert rel_l2(Fb[:6], Fc[:6]) < 1e-5, i
        ep, eu = compare_particles(b.get_particles(i), _sorted(c.get_particles()), [float(v) for v in x["n"]])
        assert ep < 1e-6 and eu < 1e-5, (i, ep, eu)
        c.close()
    b.close()


def test_autotuner_keeps_the_state_and_picks_a_valid_tuning():
    b, parts, F0 = _batch(SMALL)
    b.step(2)
    F_before = [b.get_fields(i) for i in range(len(SMALL))]
    P_before = [_sorted(b.get_particles(i)) for i in range(len(SMALL))]
    launches = b.launch_count()
    best, ms = b.autotune(trial_steps=2)
    assert b.launch_count() > launches
    assert ms > 0 and best["sort_every"] in (1, 2, 4) and best["run"] in (0, 1, 4)
    assert best["tile"] in ((8, 8, 8), (4, 8, 8), (4, 4, 8), (4, 4, 4))
    assert b.get_tuning() == best
    assert b.info()["steps"] == 2
    for i in range(len(SMALL)):
        assert np.array_equal(b.get_fields(i), F_before[i])
        P = _sorted(b.get_particles(i))
        for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
            assert np.array_equal(P[k], P_before[i][k]), (i, k)
    # stepping on matches the oracle
    b.step(3)
    ref = _oracle(SMALL, parts, F0, 5)
    for i, x in enumerate(SMALL):
        e = _errors(b, i, x, ref[i])
        assert max(e.values()) < 1e-10, (i, e)
    b.close()


def test_batch_edge_cases():
    boxes = [dict(n=(8, 8, 8), order=1, ppc=1, density=1.0, seed=201),
             dict(n=(6, 6, 6), order=3, ppc=1, density=1.0, seed=202)]
    cat, counts, parts = inputs.ensemble_particles(boxes[:1])
    counts = np.array([counts[0], 0], dtype=np.int64)       # the second box holds no particles
    with pic.Batch([x["n"] for x in boxes], [x["order"] for x in boxes], dt=DT, precision=pic.FP64) as b:
        with pytest.raises(pic.PicError) as e:
            b.step(1)
        assert e.value.status == pic.PIC_ERR_STATE
        b.load_particles(-1.0, 1.0, cat, counts)
        b.step(3)
        assert b.info(1)["particles"] == 0 and b.info()["particles"] == counts[0]
        assert np.all(b.get_fields(1) == 0.0)          # an empty box stays at rest
        with pytest.raises(pic.PicError) as e:
            b.get_field(2, 0, out=np.empty((8, 8, 8)))
        assert e.value.status == pic.PIC_ERR_ARG
        with pytest.raises(pic.PicError) as e:
            b.set_tuning(tile=(3, 8, 8))
        assert e.value.status == pic.PIC_ERR_ARG
        with pytest.raises(pic.PicError) as e:
            b.step(-1)
        assert e.value.status == pic.PIC_ERR_ARG
        P = b.get_particles(0)
        ref = _oracle(boxes[:1], parts[:1], [np.zeros((9, 8, 8, 8))], 3)[0]
        ep, eu = compare_particles(P, ref[0], [8.0, 8.0, 8.0])
        assert ep < 1e-12 and eu < 1e-12


def test_ensemble_workload_full_size_sampled():
    """The 96-box ensemble, FP32-mixed, default tuning: two steps; the three
    smallest boxes against the oracle, every box's charge conserved and div B
    at rounding level."""
    boxes = inputs.ensemble_boxes()
    cat, counts, parts = inputs.ensemble_particles(boxes)
    with pic.Batch([x["n"] for x in boxes], [x["order"] for x in boxes], dt=DT,
                   precision=pic.FP32_MIXED) as b:
        b.load_particles(-1.0, 1.0, cat, counts)
        q0 = [b.diagnostics(i)["charge"] for i in range(len(boxes))]
        b.step(2)
        for i in range(len(boxes)):
            d = b.diagnostics(i)
            assert abs(d["charge"] - q0[i]) <= 1e-9 * abs(q0[i])
            assert d["max_div_b"] < 1e-6
        small = sorted(range(len(boxes)), key=lambda i: int(np.prod(boxes[i]["n"])) * boxes[i]["ppc"])[:3]
        sel = [boxes[i] for i in small]
        ref = _oracle(sel, [parts[i] for i in small], [np.zeros((9,) + x["n"]) for x in sel], 2)
        for j, i in enumerate(small):
            e = _errors(b, i, boxes[i], ref[j])
            assert e["EB"] < 1e-5 and e["pos"] < 1e-6 and e["mom"] < 1e-5, (i, e)
