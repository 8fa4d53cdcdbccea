"""pic_sort_particles (the sort-interval and bin-size study of Sec. 3.4.2):
the reorders keep every particle, put them in the stated order, and leave
the physics unchanged: steps of the fused path (which sorts by cell first)
and of the split API (which runs in any order) after a random or a coarse
reorder match the FP64 oracle to 1e-12."""
import numpy as np
import pytest

from gpu_helpers import Case, by_id
from paper_2101_12149_gb300 import pic

pytestmark = pytest.mark.gpu

N = (16, 16, 16)
T = (4, 4, 8)


def _keys(parts):
    """Tile-major cell keys of the particles for grid N and tiles T."""
    nt = [N[a] // T[a] for a in range(3)]
    c = [np.floor(parts[k]).astype(np.int64) for k in ("x", "y", "z")]
    t = [c[a] // T[a] for a in range(3)]
    loc = [c[a] % T[a] for a in range(3)]
    tile = (t[0] * nt[1] + t[1]) * nt[2] + t[2]
    return tile * (T[0] * T[1] * T[2]) + (loc[0] * T[1] + loc[1]) * T[2] + loc[2]


def _case(precision=pic.FP64, sort_every=1):
    return Case(N, 3, 4, 0.3, 91, precision=precision, field_scale=0.05, tile=T, sort_every=sort_every)


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_MIXED])
def test_reorders_keep_the_particles_in_the_stated_order(precision):
    c = _case(precision)
    ref = by_id(c.ctx.get_particles())
    for shift in (pic.ORDER_RANDOM, 5, 7, 0, pic.ORDER_RANDOM):
        c.ctx.sort_particles(shift)
        got = c.ctx.get_particles()
        g = by_id(got)
        assert np.array_equal(g["id"], np.arange(g["id"].size))
        for k in pic.PARTICLE_KEYS:
            assert np.array_equal(g[k], ref[k]), (shift, k)
        keys = _keys(got)
        if shift >= 0:
            assert np.all(np.diff(keys >> shift) >= 0), shift
        else:
            # a random order: about half of the neighbours are out of cell order
            assert 0.3 < np.mean(np.diff(keys) < 0) < 0.7
    # two random reorders differ
    c.ctx.sort_particles(pic.ORDER_RANDOM)
    a = c.ctx.get_particles()["id"].copy()
    c.ctx.sort_particles(pic.ORDER_RANDOM)
    assert not np.array_equal(a, c.ctx.get_particles()["id"])


@pytest.mark.parametrize("shift", [pic.ORDER_RANDOM, 6])
@pytest.mark.parametrize("sort_every", [1, 3])
def test_fused_steps_after_a_reorder_match_the_oracle(shift, sort_every):
    c = _case(sort_every=sort_every)
    c.ctx.step(1)
    c.oracle_steps(1)
    c.ctx.sort_particles(shift)
    c.ctx.step(3)
    c.oracle_steps(3)
    e = c.errors()
    assert max(e.values()) < 1e-12, e


@pytest.mark.parametrize("shift", [pic.ORDER_RANDOM, 0, 9])
def test_split_api_in_any_order_matches_the_oracle(shift):
    c = _case()
    for s in range(3):
        c.ctx.sort_particles(shift)
        c.ctx.gather_push()
        c.ctx.deposit()
        c.ctx.yee_step()
    c.oracle_steps(3)
    e = c.errors()
    assert max(e.values()) < 1e-12, e


def test_adjoint_after_a_random_reorder():
    """The adjoint sorts by cell first; its gradients are those of the
    cell-ordered run."""
    from paper_2101_12149_gb300 import inputs
    n = (8, 8, 8)
    parts = inputs.uniform_plasma(5, n, 1, sigma_u=0.05)
    A, kd = inputs.drive_amplitude(5), 2 * np.pi / n[0]
    out = []
    for shuffle in (False, True):
        with pic.Context(n, order=2) as ctx:
            ctx.load_particles(-1.0, 1.0, parts)
            ctx.set_external_drive(A, kd)
            if shuffle:
                ctx.sort_particles(pic.ORDER_RANDOM)
            out.append(ctx.step_adjoint(4, 2))
    assert abs(out[1][0] - out[0][0]) < 1e-12 * abs(out[0][0])
    assert abs(out[1][1] - out[0][1]) < 1e-10 * abs(out[0][1])
    assert np.linalg.norm(out[1][2] - out[0][2]) < 1e-10 * np.linalg.norm(out[0][2])


def test_sort_particles_checks():
    c = _case()
    for bad in (-2, 31):
        with pytest.raises(pic.PicError) as ei:
            c.ctx.sort_particles(bad)
        assert ei.value.status == pic.PIC_ERR_ARG
    # a reorder between pic_gather_push and pic_deposit drops the pending move
    c.ctx.gather_push()
    c.ctx.sort_particles(pic.ORDER_RANDOM)
    with pytest.raises(pic.PicError) as ei:
        c.ctx.deposit()
    assert ei.value.status == pic.PIC_ERR_STATE
    with pic.Context((8, 8, 32), order=1, window_speed=1.0) as w:
        with pytest.raises(pic.PicError) as ei:
            w.sort_particles(0)
        assert ei.value.status == pic.PIC_ERR_STATE
    # no particles: nothing to do
    with pic.Context((8, 8, 8), order=1) as e:
        e.sort_particles(pic.ORDER_RANDOM)
