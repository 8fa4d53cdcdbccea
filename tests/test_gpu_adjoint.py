"""GPU discrete adjoint (pic_step_adjoint) against the FP64 CPU oracle's
adjoint, against central differences of the GPU's own FP64 forward run, and
the FP32-mixed adjoint against the FP64 one.  The workload is a 16^3 copy of
the differentiation workload (4 ppc, order 2, sigma_u 0.05, seed 4, drive
A = 0.05 (1 + U), k_d = 2 pi / 16); loss L = 1/2 sum(|E|^2 + |B|^2) dV."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2101_12149_gb300 import inputs, pic

pytestmark = pytest.mark.gpu

SEED = 4
A0 = inputs.drive_amplitude(SEED)
CFL = 0.99


def _parts(n, ppc, seed=SEED):
    return inputs.uniform_plasma(seed, n, ppc, sigma_u=0.05)


def _gpu_adjoint(n, p, ppc, steps, ckpt, precision=pic.FP64, A=A0, parts=None, sort_every=1):
    parts = _parts(n, ppc) if parts is None else parts
    with pic.Context(n, cfl=CFL, precision=precision, order=p, sort_every=sort_every) as c:
        c.load_particles(-1.0, 1.0, parts)
        c.set_external_drive(A, 2 * np.pi / n[0])
        return c.step_adjoint(steps, ckpt)


def _gpu_loss(n, p, parts, steps, A, precision=pic.FP64):
    with pic.Context(n, cfl=CFL, precision=precision, order=p) as c:
        c.load_particles(-1.0, 1.0, parts)
        c.set_external_drive(A, 2 * np.pi / n[0])
        c.step(steps)
        return c.diagnostics()["field_energy"]


def _oracle_adjoint(n, p, ppc, steps, A=A0):
    O = Oracle()
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1.0, 1.0, 1.0), CFL)
    P = {k: v.copy() for k, v in _parts(n, ppc).items()}
    F = np.zeros((9,) + tuple(n))
    return O.pic_adjoint(g, p, dt, -1.0, 1.0, P, F, steps, A, 2 * np.pi / n[0])


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


CASES = [
    # (n, order, ppc, steps, checkpoint spacing)
    ((16, 16, 16), 2, 4, 20, 7),
    ((8, 8, 8), 1, 2, 12, 5),
    ((8, 8, 16), 3, 2, 10, 4),
]


@pytest.mark.parametrize("n,p,ppc,steps,ckpt", CASES)
def test_fp64_adjoint_matches_oracle_adjoint(n, p, ppc, steps, ckpt):
    loss_o, dA_o, du_o = _oracle_adjoint(n, p, ppc, steps)
    loss, dA, du = _gpu_adjoint(n, p, ppc, steps, ckpt)
    assert abs(loss - loss_o) < 1e-12 * loss_o, (loss, loss_o)
    assert abs(dA - dA_o) < 1e-10 * abs(dA_o), (dA, dA_o)
    assert _rel(du, du_o) < 1e-10, _rel(du, du_o)


def test_fp64_adjoint_with_sort_cadence_matches_oracle():
    n, p, ppc, steps = (8, 8, 8), 2, 2, 12
    loss_o, dA_o, du_o = _oracle_adjoint(n, p, ppc, steps)
    loss, dA, du = _gpu_adjoint(n, p, ppc, steps, 5, sort_every=3)
    assert abs(dA - dA_o) < 1e-10 * abs(dA_o)
    assert _rel(du, du_o) < 1e-10


def test_checkpoint_spacing_does_not_change_the_adjoint():
    n, p, ppc, steps = (8, 8, 8), 2, 2, 12
    ref = _gpu_adjoint(n, p, ppc, steps, steps)
    for k in (1, 5, 64):
        loss, dA, du = _gpu_adjoint(n, p, ppc, steps, k)
        assert abs(loss - ref[0]) < 1e-13 * ref[0]
        assert abs(dA - ref[1]) < 1e-12 * abs(ref[1]), k
        assert _rel(du, ref[2]) < 1e-12, k


def test_fp64_adjoint_matches_central_differences():
    """dL/dA against central differences with h = 1e-4 on A; dL/du0 along a
    seeded unit direction and at 16 single components, h = 1e-4."""
    n, p, ppc, steps = (16, 16, 16), 2, 4, 20
    parts = _parts(n, ppc)
    loss, dA, du = _gpu_adjoint(n, p, ppc, steps, 7, parts=parts)
    h = 1e-4
    fd = (_gpu_loss(n, p, parts, steps, A0 + h) - _gpu_loss(n, p, parts, steps, A0 - h)) / (2 * h)
    assert abs(fd - dA) < 1e-6 * abs(fd), (fd, dA)

    N = parts["x"].size
    v = 2 * inputs.uniform(11, 0, 3 * N, 0).reshape(3, N) - 1
    v /= np.linalg.norm(v)

    def shifted(vec, s):
        Q = {k: a.copy() for k, a in parts.items()}
        for a, key in enumerate(("ux", "uy", "uz")):
            Q[key] = Q[key] + s * vec[a]
        return Q

    fdu = (_gpu_loss(n, p, shifted(v, h), steps, A0) - _gpu_loss(n, p, shifted(v, -h), steps, A0)) / (2 * h)
    assert abs(fdu - np.sum(du * v)) < 1e-6 * abs(fdu), (fdu, np.sum(du * v))
    # 16 single components with the largest sensitivity.  A step of 1e-4 in
    # one particle's momentum is 0.2% of its thermal spread and moves it across
    # shape knots, where the order-2 shape's second derivative jumps; the
    # difference quotient then carries an O(h) error, so these use h = 1e-5
    # (rounding: about 1e-8 relative).
    hs = 1e-5
    order = np.argsort(-np.abs(du).ravel())[:16]
    worst = 0.0
    for flat in order:
        e = np.zeros(3 * N)
        e[flat] = 1.0
        e = e.reshape(3, N)
        fdc = (_gpu_loss(n, p, shifted(e, hs), steps, A0) - _gpu_loss(n, p, shifted(e, -hs), steps, A0)) / (2 * hs)
        err = abs(fdc - du.ravel()[flat]) / abs(fdc)
        worst = max(worst, err)
        assert err < 1e-6, (flat, fdc, du.ravel()[flat])
    print(f"adjoint vs central differences: dA {abs(fd - dA) / abs(fd):.2e}, "
          f"direction {abs(fdu - np.sum(du * v)) / abs(fdu):.2e}, worst component {worst:.2e}")


def test_context_ends_in_the_forward_final_state():
    n, p, ppc, steps = (8, 8, 8), 2, 2, 9
    parts = _parts(n, ppc)
    with pic.Context(n, cfl=CFL, order=p) as a, pic.Context(n, cfl=CFL, order=p) as b:
        for c in (a, b):
            c.load_particles(-1.0, 1.0, parts)
            c.set_external_drive(A0, 2 * np.pi / n[0])
        a.step_adjoint(steps, 4)
        b.step(steps)
        assert a.time()[0] == b.time()[0] == steps
        Fa, Fb = a.get_fields(), b.get_fields()
        assert _rel(Fa[:6], Fb[:6]) < 1e-13
        pa, pb = a.get_particles(), b.get_particles()
        ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
        for k in ("x", "ux", "uz"):
            assert np.max(np.abs(pa[k][ia] - pb[k][ib])) < 1e-12
        # and the context keeps stepping normally
        a.step(2)
        b.step(2)
        assert _rel(a.get_fields()[:6], b.get_fields()[:6]) < 1e-12


def test_fp32_mixed_adjoint_against_fp64():
    """Stated error of the FP32-mixed adjoint on the 16^3, 20-step case."""
    n, p, ppc, steps = (16, 16, 16), 2, 4, 20
    _, dA64, du64 = _gpu_adjoint(n, p, ppc, steps, 7)
    _, dA32, du32 = _gpu_adjoint(n, p, ppc, steps, 7, precision=pic.FP32_MIXED)
    print(f"FP32-mixed adjoint: dA rel err {abs(dA32 - dA64) / abs(dA64):.3e}, du rel L2 {_rel(du32, du64):.3e}")
    # measured on GB300: 9.2e-8 and 3.6e-6
    assert abs(dA32 - dA64) < 1e-6 * abs(dA64)
    assert _rel(du32, du64) < 3e-5


def test_adjoint_edge_cases():
    n = (8, 8, 8)
    parts = _parts(n, 1)
    with pic.Context(n, cfl=CFL, order=2) as c:
        with pytest.raises(pic.PicError) as e:
            c.step_adjoint(3, 1)
        assert e.value.status == pic.PIC_ERR_STATE
        c.load_particles(-1.0, 1.0, parts)
        with pytest.raises(pic.PicError) as e:
            c.step_adjoint(3, 0)
        assert e.value.status == pic.PIC_ERR_ARG
        # zero steps from zero fields: L = 0 and all gradients vanish
        loss, dA, du = c.step_adjoint(0, 4)
        assert loss == 0.0 and dA == 0.0 and not np.any(du)
        # without a drive dL/dA is zero; a single step with a long spacing works
        loss, dA, du = c.step_adjoint(1, 100)
        assert dA == 0.0 and loss > 0.0 and np.all(np.isfinite(du))


def test_autograd_function_returns_the_library_gradients():
    torch = pytest.importorskip("torch")
    from paper_2101_12149_gb300 import adjoint

    n, p, ppc, steps = (8, 8, 8), 2, 2, 10
    parts = _parts(n, ppc)
    spec = adjoint.RunSpec(n=n, parts=parts, nsteps=steps, drive_k=2 * np.pi / n[0], order=p, ckpt_every=4)
    A = torch.tensor(A0, dtype=torch.float64, requires_grad=True)
    u0 = torch.tensor(np.stack([parts["ux"], parts["uy"], parts["uz"]]), dtype=torch.float64,
                      device="cuda", requires_grad=True)
    L = adjoint.field_energy_loss(A, u0, spec)
    (3.0 * L).backward()
    loss, dA, du = _gpu_adjoint(n, p, ppc, steps, 4, parts=parts)
    assert abs(L.item() - loss) < 1e-13 * loss
    assert abs(A.grad.item() - 3.0 * dA) < 1e-12 * abs(3.0 * dA)
    assert u0.grad.is_cuda
    assert _rel(u0.grad.cpu().numpy(), 3.0 * du) < 1e-12


@pytest.mark.slow
def test_fp64_adjoint_200_steps_matches_oracle_adjoint():
    """The differentiation workload's full length on its 16^3 copy: 200 steps,
    checkpoints every 20, the discrete adjoint on the GPU against the oracle's
    (exact for the discrete map up to the order of additions), with the work
    space reserved up front (pic_reserve_adjoint), so the adjoint call itself
    allocates nothing."""
    n, p, ppc, steps, ckpt = (16, 16, 16), 2, 4, 200, 20
    loss_o, dA_o, du_o = _oracle_adjoint(n, p, ppc, steps)
    with pic.Context(n, cfl=CFL, precision=pic.FP64, order=p) as c:
        c.load_particles(-1.0, 1.0, _parts(n, ppc))
        c.set_external_drive(A0, 2 * np.pi / n[0])
        c.reserve_adjoint(steps, ckpt)
        loss, dA, du = c.step_adjoint(steps, ckpt)
    print(f"200-step adjoint: loss {loss:.6e} vs {loss_o:.6e}; dL/dA {dA:.9e} vs {dA_o:.9e}; "
          f"dL/du rel {_rel(du, du_o):.2e}")
    assert abs(loss - loss_o) < 1e-12 * loss_o, (loss, loss_o)
    assert abs(dA - dA_o) < 1e-10 * abs(dA_o), (dA, dA_o)
    assert _rel(du, du_o) < 1e-10, _rel(du, du_o)


def test_reserved_adjoint_space_gives_the_same_gradients():
    """pic_reserve_adjoint only changes where the work space comes from."""
    n, p, ppc, steps, ckpt = (8, 8, 8), 2, 2, 12, 5
    ref = _gpu_adjoint(n, p, ppc, steps, ckpt)
    with pic.Context(n, cfl=CFL, precision=pic.FP64, order=p) as c:
        c.load_particles(-1.0, 1.0, _parts(n, ppc))
        c.set_external_drive(A0, 2 * np.pi / n[0])
        c.reserve_adjoint(steps, ckpt)
        got = c.step_adjoint(steps, ckpt)
        c.reserve_adjoint(0)
    # the two runs differ only in the order of floating-point atomic additions
    assert abs(got[0] - ref[0]) < 1e-13 * ref[0] and abs(got[1] - ref[1]) < 1e-11 * abs(ref[1])
    assert _rel(got[2], ref[2]) < 1e-11
