"""CUDA path (through the C-ABI) against the FP64 CPU oracle on the same seeded
inputs.  FP64: 1e-12 relative L2 after one step, 1e-9 after the 50-step
32^3 run (atomic summation order is the only allowed difference).
FP32-mixed: error stated against the FP64 oracle."""
import numpy as np
import pytest

from gpu_helpers import Case, rel_l2
from paper_2101_12149_gb300 import inputs, pic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ONE_STEP_CASES = [
    # n, order, ppc, sigma_u, seed, d, tile
    ((16, 8, 24), 1, 3, 0.3, 1, (1.0, 1.0, 1.0), (0, 0, 0)),
    ((16, 8, 24), 2, 3, 0.3, 2, (1.0, 1.0, 1.0), (0, 0, 0)),
    ((16, 8, 24), 3, 3, 0.3, 3, (1.0, 1.0, 1.0), (0, 0, 0)),
    ((12, 20, 8), 3, 2, 0.5, 4, (1.0, 0.9, 1.1), (0, 0, 0)),   # tiles 4x4x8, non-unit cells
    ((5, 6, 7), 3, 2, 0.5, 5, (1.0, 1.0, 1.0), (0, 0, 0)),     # tiles of 1 cell, grid barely > stencil
    ((16, 16, 16), 2, 4, 0.8, 6, (1.0, 1.0, 1.0), (2, 4, 8)),  # non-cubic tiles, relativistic
]


@pytest.mark.parametrize("case", ONE_STEP_CASES, ids=lambda c: f"n{c[0]}-p{c[1]}")
def test_fp64_one_step_fused(case):
    n, p, ppc, sig, seed, d, tile = case
    c = Case(n, p, ppc, sig, seed, d=d, tile=tile, field_scale=0.05)
    c.ctx.step(1)
    c.oracle_steps(1)
    e = c.errors()
    assert e["EB"] < 1e-12 and e["J"] < 1e-12 and e["pos"] < 1e-12 and e["mom"] < 1e-12, e


@pytest.mark.parametrize("case", ONE_STEP_CASES[:4], ids=lambda c: f"n{c[0]}-p{c[1]}")
def test_fp64_one_step_split_api(case):
    """pic_gather_push + pic_deposit + pic_yee_step (global-memory kernels)."""
    n, p, ppc, sig, seed, d, tile = case
    c = Case(n, p, ppc, sig, seed, d=d, tile=tile, field_scale=0.05)
    c.ctx.gather_push()
    c.ctx.deposit()
    c.ctx.yee_step()
    c.oracle_steps(1)
    e = c.errors()
    assert e["EB"] < 1e-12 and e["J"] < 1e-12 and e["pos"] < 1e-12 and e["mom"] < 1e-12, e


@pytest.mark.parametrize("sort_every", [1, 3])
def test_fp64_multi_step(sort_every):
    """Ten steps with and without a sort every step (between sorts particles
    leave their tile and take the global path)."""
    c = Case((16, 16, 8), 3, 4, 0.4, 11, field_scale=0.02, sort_every=sort_every)
    c.ctx.step(10)
    c.oracle_steps(10)
    e = c.errors()
    assert max(e.values()) < 1e-11, e


def test_uniform_32_full_run_fp64():
    """The 32^3, 2 ppc, order-1 workload, 50 steps: 1e-9 relative L2."""
    w = inputs.WORKLOADS["uniform_32"]
    s = torch.cuda.Stream()
    c = Case(w["n"], w["order"], w["ppc"], w["sigma_u"], w["seed"], pert=(w["pert_amp"], w["pert_k"]), stream=s)
    c.ctx.step(w["steps"])
    c.oracle_steps(w["steps"])
    e = c.errors()
    assert max(e.values()) < 1e-9, e


def test_graph_replay_matches_direct():
    """Graph-replayed steps (caller stream) give the direct launches' result."""
    s = torch.cuda.Stream()
    a = Case((16, 8, 8), 2, 4, 0.3, 21, field_scale=0.03, stream=s)
    b = Case((16, 8, 8), 2, 4, 0.3, 21, field_scale=0.03, stream=None)
    a.ctx.step(6)
    b.ctx.step(6)
    Fa, Fb = a.ctx.get_fields(), b.ctx.get_fields()
    assert rel_l2(Fa, Fb) < 1e-13
    assert a.ctx.launch_count() > 0


@pytest.mark.parametrize("use_stream,sort_every", [(False, 1), (True, 1), (False, 3), (True, 3)])
def test_counted_histogram_across_paths(use_stream, sort_every):
    """The step's sort takes its histogram from the previous step's tile
    kernel when that step counted the new keys.  Interleave everything that
    changes keys outside such a step (the split API, a sort by coarse bins,
    graph-replayed pairs and single direct steps, and with sort_every 3 steps
    that do not count) and compare with the oracle after every phase, with
    and without a caller stream (captured pairs, and direct steps with
    sort_every 3)."""
    s = torch.cuda.Stream() if use_stream else None
    c = Case((16, 16, 8), 2, 4, 0.4, 41, field_scale=0.03, stream=s, sort_every=sort_every)

    def check(k):
        c.oracle_steps(k)
        e = c.errors()
        assert max(e.values()) < 1e-11, e

    c.ctx.step(3)            # a replayed pair (with a stream) and one direct step
    check(3)
    c.ctx.gather_push()      # the split API changes the keys without counting
    c.ctx.deposit()
    c.ctx.yee_step()
    check(1)
    c.ctx.step(2)
    check(2)
    c.ctx.sort_particles(3)  # a sort by bins of 8 cells, then the step re-sorts by cell
    c.ctx.step(1)
    check(1)
    c.ctx.step(4)
    check(4)


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_MIXED])
@pytest.mark.parametrize("use_stream", [False, True])
def test_unequal_weights_through_sorted_steps(precision, use_stream):
    """Particles of unequal weights through six steps with a sort every step:
    each sorted-order step moves every particle, weight included, into its
    slot of the other buffer.  With equal weights a weight left behind would
    go unnoticed (the slot's old value would be the same)."""
    from oracle import Oracle
    n, order, steps = (16, 16, 8), 2, 6
    parts = inputs.uniform_plasma(51, n, 4, sigma_u=0.3)
    rng = np.random.default_rng(52)
    parts["w"] = parts["w"] * (0.25 + 1.5 * rng.random(parts["w"].size))
    F = np.zeros((9,) + n)
    F[:6] = inputs.random_fields(53, n, 0.03)[:6]
    dt = inputs.dt_from_cfl((1.0, 1.0, 1.0), 0.99)
    s = torch.cuda.Stream() if use_stream else None
    with pic.Context(n, dt=dt, order=order, precision=precision, stream=s) as c:
        c.set_fields(F)
        c.load_particles(-1.0, 1.0, parts)
        c.step(steps)
        G = c.get_fields()
        q = c.get_particles()
    O = Oracle()
    g = O.grid(n)
    ref = {k: v.copy() for k, v in parts.items()}
    Fr = F.copy()
    for s_ in range(steps):
        O.pic_step(g, order, dt, -1.0, 1.0, ref, Fr, 0.0, 0.0, s_ * dt)
    o = np.argsort(q["id"])
    assert np.array_equal(np.asarray(q["id"])[o], np.arange(parts["w"].size))
    w_err = np.abs(np.asarray(q["w"])[o] - parts["w"]).max() / parts["w"].max()
    if precision == pic.FP64:
        assert w_err == 0.0
        assert rel_l2(G[:6], Fr[:6]) < 1e-11 and rel_l2(G[6:], Fr[6:]) < 1e-11
    else:
        assert w_err < 1e-7
        assert rel_l2(G[:6], Fr[:6]) < 1e-5 and rel_l2(G[6:], Fr[6:]) < 1e-4


def test_external_drive_fp64():
    c = Case((16, 8, 8), 2, 2, 0.05, 31)
    k = 2 * np.pi / 16
    c.ctx.set_external_drive(0.07, k)
    c.ctx.step(4)
    c.oracle_steps(4, drive=(0.07, k))
    e = c.errors()
    assert max(e.values()) < 1e-11, e


@pytest.mark.parametrize("p", [1, 2, 3])
def test_fp32_mixed_one_step_error(p):
    """FP32-mixed after one step: field and particle error against the FP64 oracle."""
    c = Case((16, 16, 16), p, 4, 0.3, 40 + p, precision=pic.FP32_MIXED, field_scale=0.05)
    c.ctx.step(1)
    c.oracle_steps(1)
    e = c.errors()
    assert e["EB"] < 2e-6 and e["J"] < 2e-5 and e["pos"] < 1e-6 and e["mom"] < 2e-6, e


def test_fp32_mixed_split_api():
    c = Case((16, 16, 16), 3, 4, 0.3, 50, precision=pic.FP32_MIXED, field_scale=0.05)
    c.ctx.gather_push()
    c.ctx.deposit()
    c.ctx.yee_step()
    c.oracle_steps(1)
    e = c.errors()
    assert e["EB"] < 2e-6 and e["J"] < 2e-5 and e["pos"] < 1e-6 and e["mom"] < 2e-6, e


def _tile_index(parts, T=8, nt=2):
    ci = np.floor(parts["x"]).astype(int) // T
    cj = np.floor(parts["y"]).astype(int) // T
    ck = np.floor(parts["z"]).astype(int) // T
    return (ci * nt + cj) * nt + ck


def test_particles_sorted_by_tile():
    """Right after a sort the particles are in tile order exactly; after a step
    of a hot plasma only the particles that left their tile are out of order."""
    c = Case((16, 16, 16), 1, 3, 0.5, 60, precision=pic.FP32_MIXED)
    parts = c.ctx.get_particles()
    assert np.all(np.diff(_tile_index(parts)) >= 0)
    assert np.array_equal(np.sort(parts["id"]), np.arange(parts["id"].size))
    c.ctx.step(3)
    parts = c.ctx.get_particles()
    assert np.mean(np.diff(_tile_index(parts)) < 0) < 0.15
    assert np.array_equal(np.sort(parts["id"]), np.arange(parts["id"].size))


def test_diagnostics_match_oracle():
    c = Case((16, 8, 8), 3, 2, 0.2, 70, field_scale=0.05)
    c.ctx.step(2)
    c.oracle_steps(2)
    dg = c.ctx.diagnostics()
    fe = c.O.field_energy(c.g, c.Fref)
    ke = c.O.kinetic_energy(1.0, c.ref["ux"], c.ref["uy"], c.ref["uz"], c.ref["w"])
    assert abs(dg["field_energy"] - fe) < 1e-12 * fe
    assert abs(dg["kinetic_energy"] - ke) < 1e-12 * ke
    assert abs(dg["charge"] - (-c.ref["w"].sum())) < 1e-12 * c.ref["w"].sum()


def test_empty_and_bad_inputs():
    ctx = pic.Context((8, 8, 8), order=1)
    with pytest.raises(pic.PicError) as ei:
        ctx.step(1)
    assert ei.value.status == pic.PIC_ERR_STATE
    parts = inputs.uniform_plasma(1, (8, 8, 8), 1)
    parts["ux"][5] = np.nan
    with pytest.raises(pic.PicError) as ei:
        ctx.load_particles(-1.0, 1.0, parts)
    assert ei.value.status == pic.PIC_ERR_ARG
    with pytest.raises(pic.PicError) as ei:
        ctx.deposit()
    assert ei.value.status == pic.PIC_ERR_STATE
    # zero particles is a valid load; fields still advance
    empty = {k: np.zeros(0) for k in pic.PARTICLE_KEYS}
    ctx.load_particles(-1.0, 1.0, empty)
    assert ctx.num_particles() == 0
    ctx.yee_step()


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_MIXED])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_positions_at_node_boundaries(precision, p):
    """Offsets within an ulp of a node or a half node (where a rounded window
    start would shift the Esirkepov stencil) deposit like the oracle."""
    n = (8, 8, 8)
    eps = 2.0 ** -24 if precision == pic.FP32_MIXED else 2.0 ** -52
    fr = np.array([1 - eps, eps, 0.5 - eps, 0.5, 0.5 + eps, 1 - 2 * eps, 0.0, 0.25])
    m = fr.size
    base = np.arange(m) % 8
    parts = {
        "x": base + fr, "y": (base + 3) % 8 + fr[::-1], "z": (base + 5) % 8 + np.roll(fr, 3),
        "ux": np.tile([0.3, -0.3], m // 2), "uy": np.tile([-0.2, 0.25], m // 2), "uz": np.tile([1e-3, -1e-3], m // 2),
        "w": np.full(m, 0.5),
    }
    parts = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in parts.items()}
    c = Case(n, p, 1, 0.0, 80, precision=precision)
    c.parts = parts
    c.ref = {k: v.copy() for k, v in parts.items()}
    c.ctx.load_particles(c.q, c.m, parts)
    c.ctx.step(1)
    c.oracle_steps(1)
    e = c.errors()
    tol = 1e-12 if precision == pic.FP64 else 1e-5
    assert max(e.values()) < tol, e


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_MIXED])
def test_uneven_particle_spread(precision):
    """Tiles whose particles crowd into one z-row or one cell (the tile kernel
    then cuts the whole tile into runs) beside evenly filled tiles (each warp
    takes its own group of cells) deposit like the oracle."""
    n = (16, 16, 32)
    base = inputs.uniform_plasma(81, n, 2, sigma_u=0.3)
    r = inputs.uniform(82, 0, 3 * 2500, 0).reshape(3, 2500)
    row = {"x": 5 + r[0, :2000], "y": 6 + r[1, :2000], "z": 32 * r[2, :2000]}       # one z-row of cells
    cell = {"x": 9 + r[0, 2000:], "y": 2 + r[1, 2000:], "z": 20 + r[2, 2000:]}      # one cell
    u = 0.3 * (2 * inputs.uniform(83, 0, 3 * 2500, 0).reshape(3, 2500) - 1)
    parts = {}
    for k in ("x", "y", "z"):
        parts[k] = np.concatenate([base[k], row[k], cell[k]])
    for a, k in enumerate(("ux", "uy", "uz")):
        parts[k] = np.concatenate([base[k], u[a]])
    parts["w"] = np.concatenate([base["w"], np.full(2500, base["w"][0])])
    parts = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in parts.items()}
    c = Case(n, 3, 1, 0.0, 84, precision=precision)
    c.parts = parts
    c.ref = {k: v.copy() for k, v in parts.items()}
    c.ctx.load_particles(c.q, c.m, parts)
    c.ctx.step(2)
    c.oracle_steps(2)
    e = c.errors()
    tol = 1e-12 if precision == pic.FP64 else 1e-5
    assert max(e.values()) < tol, e


@pytest.mark.parametrize("n", [(8, 8, 32), (8, 12, 64), (16, 8, 96), (8, 8, 8), (12, 20, 8), (16, 8, 24)])
def test_fp32_mixed_tma_halos(n):
    """FP32-mixed grids in both tile layouts (4x4x32 where nz is a multiple
    of 32, else up to 8x8x8), E/B staged by TMA: tiles touching the grid's
    faces restage their wrapped halo planes; with random fields any wrong
    halo value shows at O(1)."""
    c = Case(n, 3, 2, 0.3, 95, precision=pic.FP32_MIXED, field_scale=0.5)
    c.ctx.step(2)
    c.oracle_steps(2)
    e = c.errors()
    assert e["EB"] < 1e-5 and e["J"] < 1e-4 and e["pos"] < 1e-6 and e["mom"] < 1e-5, e


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_MIXED])
def test_tiles_of_two_z_cells_mix_tma_and_loads(precision):
    """Tiles 4x4x2: tiles whose z origin is a multiple of 4 stage E/B by TMA,
    the others by loads; both kinds in one launch match the oracle."""
    c = Case((8, 8, 16), 3, 2, 0.3, 97, precision=precision, field_scale=0.5, tile=(4, 4, 2))
    c.ctx.step(2)
    c.oracle_steps(2)
    e = c.errors()
    if precision == pic.FP64:
        assert max(e.values()) < 1e-12, e
    else:
        assert e["EB"] < 1e-5 and e["J"] < 1e-4 and e["pos"] < 1e-6 and e["mom"] < 1e-5, e


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_MIXED])
@pytest.mark.parametrize("n", [(70, 19, 61), (33, 9, 30), (4, 3, 5)])
def test_one_pass_field_update_ragged(precision, n):
    """Whole steps (the field half is the one-pass update from one field set
    into the other: y-z tiles of 8 x 29 cells marching along x-chunks of 32)
    on grids whose extents leave ragged x-chunks, y tiles and z tiles, and on
    a grid smaller than one tile's halo in every axis; strong random fields
    so that any wrong halo cell, plane or ring slot shows at O(1); three
    steps, so the field sets swap roles and swap back."""
    c = Case(n, 1, 1, 0.3, 131, precision=precision, field_scale=0.5)
    c.ctx.step(3)
    c.oracle_steps(3)
    e = c.errors()
    if precision == pic.FP64:
        assert max(e.values()) < 1e-12, e
    else:
        assert e["EB"] < 1e-5 and e["J"] < 1e-4 and e["pos"] < 1e-6 and e["mom"] < 1e-5, e


@pytest.mark.parametrize("precision,tol", [(pic.FP64, 1e-14), (pic.FP32_MIXED, 1e-6)])
@pytest.mark.parametrize("n,zopen", [((12, 20, 96), False), ((9, 17, 70), False), ((8, 8, 64), True),
                                     ((128, 128, 128), False)])
def test_field_update_against_oracle(precision, tol, n, zopen):
    """The field update alone (pic_yee_step: B half step, E step with J, B half
    step) on random E, B, J against the oracle's Yee step: odd extents, open z
    ends, and a grid of 2M cells, far more blocks than fit on the GPU at once
    (an update that read neighbours already overwritten by other blocks would
    show there); ten steps."""
    from oracle import Oracle
    F = inputs.random_fields(90 + n[0], n, 0.5)
    kw = {"window_speed": 0.0} if zopen else {}
    with pic.Context(n, cfl=0.99, order=1, precision=precision, **kw) as c:
        c.set_fields(F)
        for _ in range(10):
            c.yee_step()
        G = c.get_fields()
    O = Oracle()
    g = O.grid(n, zopen=zopen)
    dt = inputs.dt_from_cfl((1.0, 1.0, 1.0), 0.99)
    R = F.copy()
    for _ in range(10):
        O.yee_step(g, dt, R)
    err = rel_l2(G[:6], R[:6])
    assert err < tol, err
