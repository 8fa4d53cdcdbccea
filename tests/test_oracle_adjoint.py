"""The oracle's discrete adjoint against finite differences and exact
transposes (CPU only).  Each reverse-mode piece is checked by a dot-product
test: <J v, w> from central differences of the forward map equals <v, J^T w>
from the adjoint; the whole run by central differences of the loss."""
import numpy as np
import pytest

from oracle import Oracle
from paper_2101_12149_gb300 import inputs


@pytest.fixture(scope="module")
def O():
    return Oracle()


def _rand(seed, shape, scale=1.0, draw=0):
    n = int(np.prod(shape))
    return (2 * inputs.uniform(seed, 0, n, draw) - 1).reshape(shape) * scale


@pytest.mark.parametrize("p", [1, 2, 3])
def test_dshape_matches_difference_quotient(O, p):
    xs = _rand(1, (400,), 2.4)
    knots = np.arange(-2.0, 2.01, 0.5)
    xs = xs[np.min(np.abs(xs[:, None] - knots[None, :]), axis=1) > 1e-3]
    h = 1e-6
    fd = (O.shape(p, xs + h) - O.shape(p, xs - h)) / (2 * h)
    assert np.max(np.abs(O.dshape(p, xs) - fd)) < 1e-8


def test_curl_transposes(O):
    """<C e, b> = <e, C^T b>, and C^T is the backward-difference curl of the E update."""
    n = (5, 6, 4)
    g = O.grid(n, (1.0, 0.8, 1.3))
    e = _rand(2, (3,) + n)
    b = _rand(3, (3,) + n)
    lhs = np.sum(O.curlE(g, e) * b)
    rhs = np.sum(e * O.curlE_T(g, b))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # backward-difference curl of b: E += dt (curl B - J) with E = J = 0, dt = 1
    E = np.zeros((3,) + n)
    O.yee_e(g, 1.0, E, np.ascontiguousarray(b), np.zeros((3,) + n))
    assert np.max(np.abs(O.curlE_T(g, b) - E)) < 1e-13
    # and the transpose of that curl is the forward curl
    assert np.max(np.abs(O.curlB_T(g, e) - O.curlE(g, e))) < 1e-13


def test_yee_step_adjoint_dot_product(O):
    n = (6, 5, 7)
    g = O.grid(n, (1.0, 0.9, 1.1))
    dt = 0.4
    F = np.zeros((9,) + n)
    F[:] = _rand(4, (9,) + n)
    out = F.copy()
    O.yee_step(g, dt, out)
    wE, wB = _rand(5, (3,) + n), _rand(6, (3,) + n)
    lhs = np.sum(out[0:3] * wE) + np.sum(out[3:6] * wB)
    lE, lB, lJ = O.yee_step_adj(g, dt, wE, wB)
    rhs = np.sum(F[0:3] * lE) + np.sum(F[3:6] * lB) + np.sum(F[6:9] * lJ)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_deposit_adjoint_matches_differences(O, p):
    n = (8, 7, 9)
    g = O.grid(n, (1.0, 0.9, 1.2))
    dt, qw = 0.45, -0.7
    lamJ = _rand(7 + p, (3,) + n)
    for trial in range(6):
        x0 = np.array([3.3, 2.2, 4.4]) + _rand(20 + trial, (3,), 0.3)
        x1 = x0 + _rand(30 + trial, (3,), 0.35)
        v0, v1 = _rand(40 + trial, (3,)), _rand(50 + trial, (3,))
        h = 1e-6

        def J(a, b):
            return O.deposit(g, p, dt, 1.0, [a[0]], [a[1]], [a[2]], [b[0]], [b[1]], [b[2]], [qw])

        fd = np.sum((J(x0 + h * v0, x1 + h * v1) - J(x0 - h * v0, x1 - h * v1)) * lamJ) / (2 * h)
        l0, l1 = O.deposit_adj(g, p, dt, qw, x0, x1, lamJ)
        ad = l0 @ v0 + l1 @ v1
        assert abs(fd - ad) < 1e-6 * max(1.0, abs(ad)), (p, trial, fd, ad)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_gather_adjoint(O, p):
    n = (7, 8, 6)
    g = O.grid(n, (1.0, 1.1, 0.9))
    F = _rand(60 + p, (6,) + n)
    x = np.array([2.37, 3.61, 2.08])
    lamEB = _rand(70 + p, (6,))
    # linear in the fields: exact transpose
    lamF, lx = O.gather_adj(g, p, F, x, lamEB)
    EB = O.gather(g, p, F, [x[0]], [x[1]], [x[2]])[0]
    assert abs(EB @ lamEB - np.sum(F * lamF)) < 1e-12 * max(1.0, abs(EB @ lamEB))
    # position derivative by central differences
    v = _rand(80 + p, (3,))
    h = 1e-6
    Ep = O.gather(g, p, F, [x[0] + h * v[0]], [x[1] + h * v[1]], [x[2] + h * v[2]])[0]
    Em = O.gather(g, p, F, [x[0] - h * v[0]], [x[1] - h * v[1]], [x[2] - h * v[2]])[0]
    fd = (Ep - Em) @ lamEB / (2 * h)
    assert abs(fd - lx @ v) < 1e-6 * max(1.0, abs(fd))


def test_boris_adjoint(O):
    q, m, dt = -1.0, 1.0, 0.5
    for trial in range(5):
        E = _rand(90 + trial, (3,), 0.4)
        B = _rand(100 + trial, (3,), 1.5)
        u = _rand(110 + trial, (3,), 2.0)
        lam = _rand(120 + trial, (3,))
        vu, vE, vB = _rand(130 + trial, (3,)), _rand(140 + trial, (3,)), _rand(150 + trial, (3,))
        h = 1e-6

        def f(s):
            EB = np.concatenate([E + s * vE, B + s * vB])[None, :]
            ux, uy, uz = O.boris(q, m, dt, EB, [u[0] + s * vu[0]], [u[1] + s * vu[1]], [u[2] + s * vu[2]])
            return np.array([ux[0], uy[0], uz[0]])

        fd = (f(h) - f(-h)) @ lam / (2 * h)
        lu, lE, lB = O.boris_adj(q, m, dt, E, B, u, lam)
        assert abs(fd - (lu @ vu + lE @ vE + lB @ vB)) < 1e-7 * max(1.0, abs(fd))


def _adjoint_case(O, seed, n=(8, 8, 8), p=2, ppc=1, steps=12, A=0.05):
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    parts = inputs.uniform_plasma(seed, n, ppc, sigma_u=0.05)
    kd = 2 * np.pi / n[0]
    return g, dt, parts, kd, p, steps, A


def _loss(O, g, p, dt, parts, steps, A, kd):
    P = {k: v.copy() for k, v in parts.items()}
    F = np.zeros((9,) + tuple(g.n))
    for s in range(steps):
        O.pic_step(g, p, dt, -1.0, 1.0, P, F, A, kd, s * dt)
    return 0.5 * np.sum(F[:6] ** 2)


def test_full_adjoint_matches_central_differences(O):
    """dL/dA and a directional dL/du0 against central differences (h = 1e-4 on A,
    1e-5 on u0) of the oracle's own forward run."""
    g, dt, parts, kd, p, steps, A = _adjoint_case(O, 7)
    P = {k: v.copy() for k, v in parts.items()}
    F = np.zeros((9,) + tuple(g.n))
    loss, dA, du = O.pic_adjoint(g, p, dt, -1.0, 1.0, P, F, steps, A, kd)
    assert abs(loss - _loss(O, g, p, dt, parts, steps, A, kd)) < 1e-14 * loss
    h = 1e-4
    fdA = (_loss(O, g, p, dt, parts, steps, A + h, kd) - _loss(O, g, p, dt, parts, steps, A - h, kd)) / (2 * h)
    assert abs(fdA - dA) < 1e-6 * abs(fdA), (fdA, dA)
    v = _rand(200, (3, parts["x"].size))
    v /= np.linalg.norm(v)
    hu = 1e-5

    def shifted(s):
        Q = {k: c.copy() for k, c in parts.items()}
        for a, key in enumerate(("ux", "uy", "uz")):
            Q[key] = Q[key] + s * v[a]
        return Q

    fdu = (_loss(O, g, p, dt, shifted(hu), steps, A, kd) - _loss(O, g, p, dt, shifted(-hu), steps, A, kd)) / (2 * hu)
    assert abs(fdu - np.sum(du * v)) < 1e-6 * abs(fdu), (fdu, np.sum(du * v))
