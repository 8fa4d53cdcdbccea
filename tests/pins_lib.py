"""Pins for the FP64 CPU oracle: checks against what the mathematics fixes.

Every pin is a function of an `oracle.Oracle` instance that raises
AssertionError when the oracle disagrees with an independent statement of the
method: closed forms, invariants, a library routine, or brute force.  The
plain test module runs them on the default oracle; the mutation test runs them
on oracle builds with one planted mistake each and expects at least one pin to
fail for every such build.

Methods pinned (the paper names them; the formulas are the textbook ones):
order-p B-spline shapes (Sec. 4.1.1 uses 3rd order), momentum-conserving
gather on the Yee lattice (Sec. 2.4), relativistic Boris push, Esirkepov
current deposition (Sec. 3.4.1), Yee FDTD (Sec. 2.4, Sec. 4.1.1).
"""
import numpy as np
from scipy.interpolate import BSpline

from paper_2101_12149_gb300 import inputs

STAG = np.array([[0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0, 0.5, 0.5], [0.5, 0, 0.5], [0.5, 0.5, 0]])


def bspline(p):
    """Centred cardinal B-spline of degree p from scipy (zero outside its support)."""
    knots = np.arange(p + 2, dtype=np.float64) - 0.5 * (p + 1)
    b = BSpline.basis_element(knots, extrapolate=False)

    def f(x):
        v = b(np.asarray(x, dtype=np.float64))
        return np.nan_to_num(v, nan=0.0)
    return f


def _rand(seed, n, lo, hi, draw=0):
    return lo + (hi - lo) * inputs.uniform(seed, 0, n, draw)


# --------------------------------------------------------------------- shapes

def pin_shape_library(O):
    """The oracle's s_p equals scipy's cardinal B-spline basis element."""
    xs = _rand(11, 4000, -2.6, 2.6)
    for p in (1, 2, 3):
        ref = bspline(p)(xs)
        got = O.shape(p, xs)
        assert np.max(np.abs(got - ref)) < 1e-15, f"shape p={p} differs from scipy B-spline"


def pin_shape_moments(O):
    """Partition of unity, linear reproduction, and the second moment
    sum_i i^2 s_p(x-i) = x^2 + (p+1)/12 for p >= 2 (variance of p+1 unit boxes)."""
    xs = _rand(12, 3000, -9.0, 9.0)
    for p in (1, 2, 3):
        for x in xs[:1000] if p == 1 else xs:
            i = np.arange(int(np.floor(x)) - 3, int(np.floor(x)) + 5)
            s = O.shape(p, x - i)
            assert abs(s.sum() - 1.0) < 1e-15, f"partition of unity p={p} x={x}"
            assert abs((i * s).sum() - x) < 1e-13, f"linear reproduction p={p} x={x}"
            if p >= 2:
                assert abs((i * i * s).sum() - (x * x + (p + 1) / 12.0)) < 1e-12, f"second moment p={p}"


def pin_shape_convolution(O):
    """s_p(x) = integral of s_{p-1} over [x-1/2, x+1/2], with s_0 the unit box
    (so s_1 is checked against the analytic box integral)."""
    gl_x, gl_w = np.polynomial.legendre.leggauss(6)
    xs = _rand(13, 300, -2.4, 2.4)
    for x in xs:
        box = max(0.0, min(x + 0.5, 0.5) - max(x - 0.5, -0.5))
        assert abs(O.shape(1, x)[0] - box) < 1e-15
        for p in (2, 3):
            lo, hi = x - 0.5, x + 0.5
            cuts = np.unique(np.concatenate([[lo, hi], np.arange(-2.5, 2.6, 0.5)]))
            cuts = cuts[(cuts >= lo) & (cuts <= hi)]
            acc = 0.0
            for a, b in zip(cuts[:-1], cuts[1:]):
                t = 0.5 * (b - a) * gl_x + 0.5 * (a + b)
                acc += 0.5 * (b - a) * np.dot(gl_w, O.shape(p - 1, t))
            assert abs(O.shape(p, x)[0] - acc) < 1e-14, f"convolution identity p={p} x={x}"


def pin_shape_values(O):
    """Textbook node values: s1(0)=1; s2(0)=3/4, s2(1)=1/8; s3(0)=2/3, s3(1)=1/6; zero at +-(p+1)/2."""
    assert O.shape(1, 0.0)[0] == 1.0
    assert O.shape(2, 0.0)[0] == 0.75 and abs(O.shape(2, 1.0)[0] - 0.125) < 1e-16
    assert abs(O.shape(3, 0.0)[0] - 2.0 / 3.0) < 1e-16 and abs(O.shape(3, -1.0)[0] - 1.0 / 6.0) < 1e-16
    for p in (1, 2, 3):
        assert O.shape(p, 0.5 * (p + 1))[0] == 0.0 and O.shape(p, -0.5 * (p + 1))[0] == 0.0


# --------------------------------------------------------------------- gather

def pin_gather_constant(O):
    """Constant fields are reproduced exactly, including next to the periodic seam."""
    n = (8, 6, 10)
    g = O.grid(n, (1.0, 0.9, 1.1))
    L = np.array(n) * np.array([1.0, 0.9, 1.1])
    consts = np.array([0.3, -1.2, 2.5, 0.7, -0.4, 1.9])
    F = np.stack([np.full(n, c) for c in consts])
    m = 400
    pos = [_rand(21, m, 0.0, L[a], draw=a) for a in range(3)]
    pos[0][:20] = np.linspace(0.0, 0.49, 20)
    pos[1][20:40] = L[1] - np.linspace(1e-9, 0.4, 20)
    for p in (1, 2, 3):
        EB = O.gather(g, p, F, *pos)
        assert np.max(np.abs(EB - consts)) < 1e-14, f"constant field p={p}"


def pin_gather_polynomial(O):
    """A field linear along one axis in its own staggered coordinate is gathered
    exactly; a quadratic one returns x^2 + (p+1)/12 for p >= 2.  Checks every
    component's staggering along every axis."""
    n = (16, 16, 16)
    d = (1.0, 1.0, 1.0)
    g = O.grid(n, d)
    m = 60
    pos = [_rand(22, m, 5.0, 11.0, draw=a) for a in range(3)]
    idx = np.indices(n).astype(np.float64)
    for c in range(6):
        for a in range(3):
            coord = idx[a] + STAG[c][a]
            for p in (1, 2, 3):
                F = np.zeros((6,) + n)
                F[c] = 0.25 + 0.5 * coord
                EB = O.gather(g, p, F, *pos)
                assert np.max(np.abs(EB[:, c] - (0.25 + 0.5 * pos[a]))) < 1e-13, f"linear comp={c} axis={a} p={p}"
                others = [o for o in range(6) if o != c]
                assert np.max(np.abs(EB[:, others])) == 0.0
                if p >= 2:
                    F[c] = coord ** 2
                    EB = O.gather(g, p, F, *pos)
                    ref = pos[a] ** 2 + (p + 1) / 12.0
                    assert np.max(np.abs(EB[:, c] - ref)) < 1e-12, f"quadratic comp={c} axis={a} p={p}"


# ---------------------------------------------------------------------- Boris

def pin_boris_pure_b(O):
    """Pure magnetic field: |u| is conserved and u_perp turns by
    2 atan(|q| B dt / (2 m gamma)) per step, in the sense of -q B."""
    q, m, dt = -1.0, 1.0, 0.3
    B = np.array([0.0, 0.0, 1.7])
    u = np.array([0.4, -0.2, 0.3])
    gam = np.sqrt(1 + u @ u)
    theta = 2 * np.arctan(abs(q) * B[2] * dt / (2 * m * gam))
    EB = np.concatenate([np.zeros(3), B])[None, :]
    ux, uy, uz = u[:1].copy(), u[1:2].copy(), u[2:].copy()
    phase0 = np.arctan2(uy[0], ux[0])
    M = 200
    for step in range(1, M + 1):
        ux, uy, uz = O.boris(q, m, dt, EB, ux, uy, uz)
        un = np.array([ux[0], uy[0], uz[0]])
        assert abs(np.linalg.norm(un) - np.linalg.norm(u)) < 1e-14 * np.linalg.norm(u)
        assert abs(uz[0] - u[2]) < 1e-15
    # q < 0 and B along +z: counter-clockwise rotation seen from +z
    expect = phase0 + M * theta
    got = np.arctan2(uy[0], ux[0])
    diff = (got - expect + np.pi) % (2 * np.pi) - np.pi
    assert abs(diff) < 1e-11, f"gyro phase {diff}"


def pin_boris_pure_e(O):
    """Pure electric field: u after M steps is u0 + M q E dt / m."""
    q, m, dt = -1.0, 1.0, 0.4
    E = np.array([0.3, -0.7, 0.11])
    EB = np.concatenate([E, np.zeros(3)])[None, :]
    ux, uy, uz = np.array([0.1]), np.array([0.2]), np.array([-0.05])
    u0 = np.array([0.1, 0.2, -0.05])
    M = 50
    for _ in range(M):
        ux, uy, uz = O.boris(q, m, dt, EB, ux, uy, uz)
    ref = u0 + M * q * E * dt / m
    got = np.array([ux[0], uy[0], uz[0]])
    assert np.max(np.abs(got - ref)) < 1e-13


def pin_boris_exb(O):
    """Crossed fields |E| << |B|: starting on the drift, u stays at E x B / B^2."""
    q, m, dt = -1.0, 1.0, 0.05
    E = np.array([0.0, 1e-3, 0.0])
    B = np.array([0.0, 0.0, 1.0])
    vd = np.cross(E, B) / (B @ B)
    u = vd / np.sqrt(1 - vd @ vd)
    EB = np.concatenate([E, B])[None, :]
    ux, uy, uz = u[:1].copy(), u[1:2].copy(), u[2:].copy()
    acc = np.zeros(3)
    M = 2000
    for _ in range(M):
        ux, uy, uz = O.boris(q, m, dt, EB, ux, uy, uz)
        un = np.array([ux[0], uy[0], uz[0]])
        acc += un / np.sqrt(1 + un @ un)
    v = acc / M
    assert abs(v[0] - vd[0]) < 1e-4 * abs(vd[0]) and abs(v[1]) < 1e-6


# ------------------------------------------------------------------ Esirkepov

def _moves(seed, m, L, maxstep):
    x0 = [_rand(seed, m, 0.0, L[a], draw=a) for a in range(3)]
    dx = [_rand(seed, m, -maxstep, maxstep, draw=3 + a) for a in range(3)]
    return x0, [x0[a] + dx[a] for a in range(3)]


def pin_esirkepov_continuity(O):
    """Discrete continuity (rho1 - rho0)/dt + div J = 0 for single particles
    and for a cloud, all orders, on a non-cubic grid with non-unit spacing."""
    n = (7, 9, 8)
    d = (1.0, 0.8, 1.25)
    g = O.grid(n, d)
    L = np.array(n) * np.array(d)
    dt, q = 0.45, -1.0
    for p in (1, 2, 3):
        x0, x1 = _moves(31 + p, 50, L, 0.95 * min(d))
        w = _rand(40, 50, 0.2, 1.5)
        for s in list(range(5)) + [slice(None)]:
            sl = [a[s] if isinstance(s, slice) else a[s:s + 1] for a in x0]
            sl1 = [a[s] if isinstance(s, slice) else a[s:s + 1] for a in x1]
            ww = w[s] if isinstance(s, slice) else w[s:s + 1]
            J = O.deposit(g, p, dt, q, *sl, *sl1, ww)
            r0 = O.rho(g, p, q, *sl, ww)
            r1 = O.rho(g, p, q, *sl1, ww)
            res = (r1 - r0) / dt + O.div_edge(g, J)
            scale = np.max(np.abs(r1 - r0)) / dt
            assert np.max(np.abs(res)) <= 1e-13 * scale, f"continuity p={p}"


def pin_esirkepov_total_current(O):
    """sum J_c dV = q w (x1_c - x0_c) / dt per particle."""
    n = (8, 8, 8)
    d = (1.0, 1.1, 0.9)
    g = O.grid(n, d)
    L = np.array(n) * np.array(d)
    dt, q = 0.5, -1.0
    dV = np.prod(d)
    for p in (1, 2, 3):
        x0, x1 = _moves(50 + p, 20, L, 0.9)
        for i in range(20):
            J = O.deposit(g, p, dt, q, *[a[i:i + 1] for a in x0], *[a[i:i + 1] for a in x1], np.array([0.7]))
            for c in range(3):
                ref = q * 0.7 * (x1[c][i] - x0[c][i]) / dt
                assert abs(J[c].sum() * dV - ref) < 1e-14 * max(1.0, abs(ref)) + 1e-15, f"total current p={p}"


def pin_esirkepov_pure_x(O):
    """Motion along x only deposits no J_y or J_z."""
    g = O.grid((8, 8, 8))
    for p in (1, 2, 3):
        x0 = [np.array([3.3]), np.array([4.71]), np.array([2.05])]
        x1 = [np.array([3.9]), x0[1].copy(), x0[2].copy()]
        J = O.deposit(g, p, 0.5, -1.0, *x0, *x1, np.array([1.0]))
        assert np.all(J[1] == 0.0) and np.all(J[2] == 0.0)
        assert np.any(J[0] != 0.0)


def _brute_force_J(n, d, p, dt, q, x0, x1, w):
    """Esirkepov current of one particle without any window: shapes on a wide
    unwrapped node range from scipy's B-spline, Esirkepov's S0/S1 form of W
    (1/3 S1S1S1 - ... in his 2001 paper), cumulative sums started far left,
    folded onto the periodic grid."""
    f = bspline(p)
    rng, S0, S1 = [], [], []
    for a in range(3):
        p0, p1 = x0[a] / d[a], x1[a] / d[a]
        r = np.arange(int(np.floor(min(p0, p1))) - 6, int(np.floor(max(p0, p1))) + 8)
        rng.append(r)
        S0.append(f(p0 - r))
        S1.append(f(p1 - r))
    J = np.zeros((3,) + tuple(n))
    dV = np.prod(d)
    for c in range(3):
        a1, a2 = (c + 1) % 3, (c + 2) % 3
        A0, A1 = S0[c], S1[c]
        B0, B1 = S0[a1], S1[a1]
        C0, C1 = S0[a2], S1[a2]
        o = np.einsum
        W = (o("i,j,k->ijk", A1 - A0, B1, C1) / 3 + o("i,j,k->ijk", A1 - A0, B0, C1) / 6 +
             o("i,j,k->ijk", A1 - A0, B1, C0) / 6 + o("i,j,k->ijk", A1 - A0, B0, C0) / 3)
        Jc = -q * w * d[c] / (dt * dV) * np.cumsum(W, axis=0)
        # Jc axes are (c, a1, a2); map to (x, y, z) node indices
        I = np.meshgrid(rng[c], rng[a1], rng[a2], indexing="ij")
        node = [None, None, None]
        node[c], node[a1], node[a2] = I
        flat = ((node[0] % n[0]) * n[1] + (node[1] % n[1])) * n[2] + (node[2] % n[2])
        np.add.at(J[c].reshape(-1), flat.ravel(), Jc.ravel())
    return J


def pin_esirkepov_brute_force(O):
    """Windowed deposit equals the window-free brute force on tiny grids,
    including grids smaller than the stencil (periodic images overlap)."""
    for n, d in (((4, 4, 4), (1.0, 1.0, 1.0)), ((5, 6, 4), (1.0, 0.7, 1.3)), ((8, 8, 8), (1.0, 1.0, 1.0))):
        g = O.grid(n, d)
        L = np.array(n) * np.array(d)
        for p in (1, 2, 3):
            x0, x1 = _moves(60 + p + n[1], 12, L, 0.97 * min(d))
            w = _rand(70, 12, 0.3, 1.2)
            Jo = O.deposit(g, p, 0.5, -1.0, *x0, *x1, w)
            Jb = np.zeros_like(Jo)
            for i in range(12):
                Jb += _brute_force_J(n, d, p, 0.5, -1.0, [a[i] for a in x0], [a[i] for a in x1], w[i])
            err = np.linalg.norm(Jo - Jb) / np.linalg.norm(Jb)
            assert err < 1e-14, f"brute force n={n} p={p} err={err}"


# ------------------------------------------------------------------------ Yee

def _levi(a, b, c):
    return {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1, (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}[(a, b, c)]


def pin_yee_plane_waves(O):
    """Single discrete modes evolve exactly: for k along axis a and E along
    e != a (h the third axis), with B = 0 at t = 0,
      E_e = A cos(n w dt) cos(k x_a),
      B_h = eps(h,a,e) A cos(w dt/2) sin(n w dt) sin(k (x_a + d_a/2)),
    where sin^2(w dt/2)/dt^2 = sin^2(k d_a/2)/d_a^2 (Yee numerical dispersion)."""
    n = (10, 8, 12)
    d = (1.0, 0.8, 1.25)
    g = O.grid(n, d)
    dt = 0.95 / np.sqrt(sum(1 / np.array(d) ** 2))
    M, A = 23, 0.8
    idx = np.indices(n).astype(np.float64)
    for a in range(3):
        m = 2 if n[a] >= 8 else 1
        k = 2 * np.pi * m / (n[a] * d[a])
        kappa = 2 * np.sin(k * d[a] / 2) / d[a]
        w = 2 / dt * np.arcsin(kappa * dt / 2)
        for e in range(3):
            if e == a:
                continue
            h = 3 - a - e
            F = np.zeros((9,) + n)
            F[e] = A * np.cos(k * idx[a] * d[a])
            for _ in range(M):
                O.yee_step(g, dt, F)
            Ee = A * np.cos(M * w * dt) * np.cos(k * idx[a] * d[a])
            Bh = _levi(h, a, e) * A * np.cos(w * dt / 2) * np.sin(M * w * dt) * np.sin(k * (idx[a] + 0.5) * d[a])
            assert np.max(np.abs(F[e] - Ee)) < 1e-12, f"E mode a={a} e={e}"
            assert np.max(np.abs(F[3 + h] - Bh)) < 1e-12, f"B mode a={a} e={e}"
            rest = [c for c in range(6) if c not in (e, 3 + h)]
            assert np.max(np.abs(F[rest])) < 1e-13


def pin_yee_oblique(O):
    """Oblique mode E_z = A cos(kx x + ky y): frequency from
    sin^2(w dt/2)/dt^2 = sum_d sin^2(k_d d_d/2)/d_d^2."""
    n = (12, 10, 4)
    d = (1.0, 1.2, 1.0)
    g = O.grid(n, d)
    dt = 0.9 / np.sqrt(sum(1 / np.array(d) ** 2))
    kx, ky = 2 * np.pi * 2 / (n[0] * d[0]), 2 * np.pi * 3 / (n[1] * d[1])
    s = (np.sin(kx * d[0] / 2) / d[0]) ** 2 + (np.sin(ky * d[1] / 2) / d[1]) ** 2
    w = 2 / dt * np.arcsin(dt * np.sqrt(s))
    idx = np.indices(n).astype(np.float64)
    phase = kx * idx[0] * d[0] + ky * idx[1] * d[1]
    F = np.zeros((9,) + n)
    F[2] = np.cos(phase)
    M = 31
    for _ in range(M):
        O.yee_step(g, dt, F)
    assert np.max(np.abs(F[2] - np.cos(M * w * dt) * np.cos(phase))) < 1e-12


def pin_yee_div_b(O):
    """div B is unchanged by any number of Yee steps with arbitrary E, B, J."""
    n = (6, 7, 5)
    g = O.grid(n, (1.0, 0.9, 1.1))
    F = inputs.random_fields(81, n)
    db0 = O.div_face(g, F[3:6])
    for _ in range(10):
        O.yee_step(g, 0.4, F)
    assert np.max(np.abs(O.div_face(g, F[3:6]) - db0)) < 1e-13


def pin_gauss_with_pic_step(O):
    """div E - rho is constant across full PIC steps (Esirkepov + Yee share one staggering)."""
    n = (8, 8, 8)
    g = O.grid(n)
    for p in (1, 2, 3):
        parts = inputs.uniform_plasma(90 + p, n, 1, sigma_u=0.6, density=1.0)
        F = np.zeros((9,) + n)
        F[:6] = inputs.random_fields(91, n, 0.05)[:6]
        q = -1.0
        r0 = O.rho(g, p, q, parts["x"], parts["y"], parts["z"], parts["w"])
        g0 = O.div_edge(g, F[0:3]) - r0
        for s in range(3):
            O.pic_step(g, p, 0.55, q, 1.0, parts, F)
        r1 = O.rho(g, p, q, parts["x"], parts["y"], parts["z"], parts["w"])
        g1 = O.div_edge(g, F[0:3]) - r1
        assert np.max(np.abs(g1 - g0)) < 1e-13 * np.max(np.abs(r0)), f"Gauss p={p}"


ALL_PINS = [
    pin_shape_library, pin_shape_moments, pin_shape_convolution, pin_shape_values,
    pin_gather_constant, pin_gather_polynomial,
    pin_boris_pure_b, pin_boris_pure_e, pin_boris_exb,
    pin_esirkepov_continuity, pin_esirkepov_total_current, pin_esirkepov_pure_x, pin_esirkepov_brute_force,
    pin_yee_plane_waves, pin_yee_oblique, pin_yee_div_b, pin_gauss_with_pic_step,
]


def pin_free_streaming(O):
    """Zero fields: particles move at v = u/gamma, u is unchanged, positions wrap
    periodically; no current survives a closed orbit of the whole box."""
    n = (6, 5, 7)
    d = (1.0, 1.2, 0.9)
    g = O.grid(n, d)
    L = np.array(n) * np.array(d)
    m = 30
    parts = {
        "x": _rand(100, m, 0.0, L[0], 0), "y": _rand(100, m, 0.0, L[1], 1), "z": _rand(100, m, 0.0, L[2], 2),
        "ux": _rand(100, m, -3.0, 3.0, 3), "uy": _rand(100, m, -3.0, 3.0, 4), "uz": _rand(100, m, -3.0, 3.0, 5),
        "w": np.ones(m),
    }
    x0 = {k: v.copy() for k, v in parts.items()}
    F = np.zeros((9,) + n)
    dt = 0.5
    M = 7
    for _ in range(M):
        O.pic_step(g, 2, dt, 0.0, 1.0, parts, F)  # q = 0: no force, no current
    gam = np.sqrt(1 + x0["ux"] ** 2 + x0["uy"] ** 2 + x0["uz"] ** 2)
    for a, (k, uk) in enumerate((("x", "ux"), ("y", "uy"), ("z", "uz"))):
        ref = np.mod(x0[k] + M * dt * x0[uk] / gam, L[a])
        diff = (parts[k] - ref + L[a] / 2) % L[a] - L[a] / 2
        assert np.max(np.abs(diff)) < 1e-12, f"free streaming axis {a}"
        assert np.all(parts[k] >= 0.0) and np.all(parts[k] < L[a])
        assert np.array_equal(parts[uk], x0[uk])
    assert np.max(np.abs(F)) == 0.0


ALL_PINS.append(pin_free_streaming)


def pin_vay(O):
    """Vay's pusher: the result satisfies its defining equation
    u_new - u = (q dt/m)(E + (v + v_new)/2 x B), and a particle on the E x B
    drift (E = -v x B) keeps its momentum, at gamma ~ 5."""
    q, m, dt = -1.0, 1.0, 0.45
    k = 40
    E = np.stack([_rand(120, k, -0.8, 0.8, a) for a in range(3)], 1)
    B = np.stack([_rand(121, k, -2.0, 2.0, a) for a in range(3)], 1)
    u = np.stack([_rand(122, k, -4.0, 4.0, a) for a in range(3)], 1)
    un = np.stack(O.vay(q, m, dt, np.concatenate([E, B], 1), u[:, 0], u[:, 1], u[:, 2]), 1)
    v = u / np.sqrt(1 + np.sum(u * u, 1))[:, None]
    vn = un / np.sqrt(1 + np.sum(un * un, 1))[:, None]
    assert np.max(np.abs((un - u) - q * dt / m * (E + np.cross(0.5 * (v + vn), B)))) < 1e-13
    Bd = np.array([0.3, -1.1, 0.7])
    d = np.array([1.0, 0.4, 0.2])
    d -= d @ Bd * Bd / (Bd @ Bd)
    ud = 5.0 * d / np.linalg.norm(d)
    Ed = -np.cross(ud / np.sqrt(1 + ud @ ud), Bd)
    got = np.array(O.vay(q, m, dt, np.concatenate([Ed, Bd])[None, :], [ud[0]], [ud[1]], [ud[2]])).ravel()
    assert np.max(np.abs(got - ud)) < 1e-12


ALL_PINS.append(pin_vay)


def pin_energy_gather_work(O):
    """Energy-conserving gather with the Esirkepov current: for a move along
    y, sum J.E dV dt equals q w times the path integral of the gathered E_y
    (order p - 1 along y), computed exactly piece by piece between knots."""
    n = (7, 8, 6)
    g = O.grid(n)
    p = 2
    F = np.zeros((6,) + n)
    F[:3] = (2 * inputs.uniform(130, 0, 3 * int(np.prod(n)), 0) - 1).reshape((3,) + n)
    q, w, dt = -1.0, 0.6, 0.5
    glx, glw = np.polynomial.legendre.leggauss(6)
    for t in range(4):
        x0 = np.array([3.1, 3.6 + 0.2 * t, 2.9])
        x1 = x0 + np.array([0.0, 0.8 - 0.45 * t, 0.0])
        J = O.deposit(g, p, dt, q, [x0[0]], [x0[1]], [x0[2]], [x1[0]], [x1[1]], [x1[2]], [w])
        work = np.sum(J * F[:3]) * dt
        lo, hi = sorted((x0[1], x1[1]))
        knots = np.arange(np.ceil(lo - 0.5), np.floor(hi - 0.5) + 1) + 0.5
        pts = np.concatenate([[lo], knots[(knots > lo) & (knots < hi)], [hi]])
        integral = 0.0
        for a, b in zip(pts[:-1], pts[1:]):
            s = 0.5 * (a + b) + 0.5 * (b - a) * glx
            P = np.repeat(x0[None, :], s.size, 0)
            P[:, 1] = s
            integral += 0.5 * (b - a) * np.sum(glw * O.gather(g, p, F, P[:, 0], P[:, 1], P[:, 2], energy=True)[:, 1])
        integral *= np.sign(x1[1] - x0[1])
        assert abs(work - q * w * integral) < 1e-12 * max(1.0, abs(work))


ALL_PINS.append(pin_energy_gather_work)


def _ckc_mode(O, n, d, m_k, M, dt, solver=1):
    """Evolve the vacuum mode of wave numbers 2 pi m_k / (n d) with E along a
    direction orthogonal to the Yee symbol; return (E^M, E^0, predicted cos)."""
    g = O.grid(n, d)
    k = np.array([2 * np.pi * m_k[a] / (n[a] * d[a]) for a in range(3)])
    kap = np.array([2 / d[a] * np.sin(k[a] * d[a] / 2) for a in range(3)])
    kt = kap.copy()
    if solver:
        for a in range(3):
            for b in range(3):
                if b != a:
                    kt[a] *= np.cos(k[b] * d[b] / 2) ** 2
    e = np.cross(kap, np.array([0.3, -0.7, 0.5]))
    e /= np.linalg.norm(e)
    F = np.zeros((9,) + tuple(n))
    idx = np.meshgrid(*[np.arange(n[a]) for a in range(3)], indexing="ij")
    for c in range(3):
        pos = [(idx[a] + (0.5 if a == c else 0.0)) * d[a] for a in range(3)]
        F[c] = e[c] * np.cos(k[0] * pos[0] + k[1] * pos[1] + k[2] * pos[2])
    E0 = F[:3].copy()
    for _ in range(M):
        O.yee_step(g, dt, F, solver=solver)
    lam = kap @ kt
    w = 2 * np.arcsin(0.5 * dt * np.sqrt(lam)) / dt
    return F[:3], E0, np.cos(M * w * dt)


def pin_ckc_oblique_mode(O):
    """CKC vacuum dispersion: an oblique mode's E evolves as E0 cos(n w dt) with
    sin^2(w dt/2) = dt^2 sum_a sin^2(k_a d/2)/d^2 prod_{b != a} cos^2(k_b d/2),
    at dt = 0.95 dx (beyond the Yee limit dx/sqrt 3)."""
    n, d = (8, 6, 10), (1.0, 1.0, 1.0)
    for m_k in ((1, 1, 2), (3, 2, 1), (2, 3, 4)):
        E, E0, c = _ckc_mode(O, n, d, m_k, 23, 0.95)
        assert np.max(np.abs(E - c * E0)) < 1e-11, m_k


ALL_PINS.append(pin_ckc_oblique_mode)


def pin_ckc_stable_at_courant_one(O):
    """At dt = 0.999 dx a random E (B = 0) stays bounded under CKC for 600
    steps; the Yee update diverges at the same step.  (B is zero at the start:
    where the transverse factor vanishes, e.g. k_x = k_y = pi, the CKC curl of
    E is zero, so B there is frozen and a B seeded there would drive E
    linearly through the Yee curl; runs start from B = 0 or smooth fields.)"""
    n = (6, 6, 6)
    g = O.grid(n)
    rng = np.random.default_rng(5)
    F = np.zeros((9,) + n)
    F[:3] = rng.uniform(-1, 1, size=(3,) + n)
    G = F.copy()
    m0 = np.max(np.abs(F[:6]))
    for _ in range(600):
        O.yee_step(g, 0.999, F, solver=1)
    assert np.max(np.abs(F[:6])) < 30 * m0
    for _ in range(60):
        O.yee_step(g, 0.999, G, solver=0)
    assert np.max(np.abs(G[:6])) > 1e6 * m0


ALL_PINS.append(pin_ckc_stable_at_courant_one)


# ---------------------------------------------------------------- diagnostics

def pin_field_energy_modes(O):
    """Field energy of discrete Fourier modes.  Component c holding
    A_c cos(2 pi m_c.i/n + phi_c) has sum over the grid of squares exactly
    C A_c^2 / 2 whenever 2 m_c is not a multiple of n along some axis (the
    cos(2 theta) part sums to zero), so 1/2 sum (|E|^2 + |B|^2) dV =
    (C dV / 4) sum_c A_c^2; on non-unit cells, with a different amplitude,
    mode and phase per component."""
    n, d = (6, 4, 10), (0.5, 2.0, 1.5)
    g = O.grid(n, d)
    idx = np.indices(n).astype(np.float64)
    modes = [(1, 1, 3), (2, 0, 1), (0, 1, 4), (1, 0, 0), (5, 3, 2), (1, 1, 1)]
    amps = [0.7, 1.3, 0.25, 2.0, 0.9, 1.1]
    F = np.zeros((9,) + n)
    for c, (m, a) in enumerate(zip(modes, amps)):
        ph = 2 * np.pi * sum(m[k] * idx[k] / n[k] for k in range(3)) + 0.37 * (c + 1)
        F[c] = a * np.cos(ph)
    C, dV = np.prod(n), np.prod(d)
    ref = 0.25 * C * dV * sum(a * a for a in amps)
    got = O.field_energy(g, F)
    assert abs(got - ref) < 1e-13 * ref, f"field energy {got} vs mode sum {ref}"
    # a single non-zero value: 1/2 v^2 dV
    G = np.zeros((9,) + n)
    G[4, 2, 1, 7] = 3.0
    assert abs(O.field_energy(g, G) - 0.5 * 9.0 * dV) < 1e-15 * 4.5 * dV


def pin_kinetic_energy_values(O):
    """Kinetic energy sum w m (gamma - 1) at momenta whose gamma is exact:
    |u|^2 = 3 gives gamma = 2, |u|^2 = 9/16 gives 5/4, |u|^2 = 144/25 gives
    13/5; the non-relativistic limit 1/2 w m |u|^2 (1 - |u|^2/4) to O(u^6);
    and the ultra-relativistic |u| = 1e6 (gamma - 1 = 999999.0000005)."""
    m = 3.5
    u = np.array([[1.0, 1.0, 1.0], [0.0, 0.75, 0.0], [0.0, 0.0, -2.4], [1e6, 0.0, 0.0]])
    w = np.array([0.25, 2.0, 1.5, 1e-3])
    gm1 = np.array([1.0, 0.25, 1.6, 999999.0000005])
    ref = float(np.sum(w * m * gm1))
    got = O.kinetic_energy(m, u[:, 0], u[:, 1], u[:, 2], w)
    assert abs(got - ref) < 1e-13 * ref, f"kinetic energy {got} vs {ref}"
    # per particle: each on its own
    for k in range(4):
        one = O.kinetic_energy(m, u[k:k + 1, 0], u[k:k + 1, 1], u[k:k + 1, 2], w[k:k + 1])
        assert abs(one - w[k] * m * gm1[k]) < 1e-13 * w[k] * m * gm1[k], f"particle {k}"
    # non-relativistic limit
    rng = np.random.default_rng(21)
    v = rng.normal(size=(50, 3)) * 1e-3
    ww = rng.uniform(0.5, 2.0, 50)
    u2 = np.sum(v * v, axis=1)
    approx = float(np.sum(0.5 * ww * m * u2 * (1.0 - 0.25 * u2)))
    got = O.kinetic_energy(m, v[:, 0], v[:, 1], v[:, 2], ww)
    assert abs(got - approx) < 1e-9 * approx, "non-relativistic limit"


def pin_rho_values(O):
    """Nodal charge density: a particle on a node spreads q w / dV with the
    shape's node values (p = 1: all on the node; p = 2: 1/8, 3/4, 1/8 per
    axis; p = 3: 1/6, 2/3, 1/6), the total charge sum rho dV is q w, and the
    first moment sum x_node rho dV is q w x (linear reproduction), on
    non-unit cells."""
    n, d = (8, 8, 8), (0.5, 2.0, 1.25)
    g = O.grid(n, d)
    dV = np.prod(d)
    node_w = {1: [1.0], 2: [0.125, 0.75, 0.125], 3: [1 / 6, 2 / 3, 1 / 6]}
    q, wq = -1.0, 0.3
    for p in (1, 2, 3):
        x = np.array([3 * d[0]]), np.array([4 * d[1]]), np.array([2 * d[2]])
        r = O.rho(g, p, q, *x, np.array([wq]))
        s = np.array(node_w[p])
        h = len(s) // 2
        ref = np.zeros(n)
        ref[3 - h:3 + h + 1, 4 - h:4 + h + 1, 2 - h:2 + h + 1] = q * wq / dV * np.einsum("i,j,k->ijk", s, s, s)
        assert np.max(np.abs(r - ref)) < 1e-15, f"rho of a particle on a node, p={p}"
        pos = [np.array([v]) for v in (3.3 * d[0], 4.71 * d[1], 3.05 * d[2])]
        r = O.rho(g, p, q, *pos, np.array([wq]))
        assert abs(r.sum() * dV - q * wq) < 1e-15, f"total charge p={p}"
        for a in range(3):
            coord = np.arange(n[a]) * d[a]
            mom = np.tensordot(r, coord, axes=([a], [0])).sum() * dV
            assert abs(mom - q * wq * pos[a][0]) < 1e-14, f"first moment p={p} axis {a}"


ALL_PINS.extend([pin_field_energy_modes, pin_kinetic_energy_values, pin_rho_values])


# ---------------------------------------------------------------- z filter

def _filter_transfer(npass, theta):
    return np.cos(0.5 * theta) ** (2 * npass) * (1.0 + npass * np.sin(0.5 * theta) ** 2)


def pin_filter_transfer_function(O):
    """The z filter (Godfrey-type, compensated binomial) on periodic Fourier
    modes along z: the output is the input times cos^(2n)(k dz/2) (1 + n
    sin^2(k dz/2)) exactly; a constant passes unchanged, the Nyquist mode is
    removed, variation along x and y is left alone, n = 0 is a copy."""
    n = (4, 3, 16)
    g = O.grid(n, (1.0, 1.0, 0.5))
    kk = np.arange(n[2])
    xy = (1.0 + 0.3 * np.arange(n[0]))[:, None, None] * (2.0 - 0.2 * np.arange(n[1]))[None, :, None]
    for npass in (1, 2, 4):
        for m in (0, 1, 3, 5, 8):
            theta = 2 * np.pi * m / n[2]
            F = xy * np.cos(theta * kk + 0.4)[None, None, :]
            out = O.filter_z(g, npass, F)
            ref = _filter_transfer(npass, theta) * F
            assert np.max(np.abs(out - ref)) < 1e-14 * np.max(np.abs(F)) + 1e-15, (npass, m)
        nyq = xy * np.cos(np.pi * kk)[None, None, :]
        assert np.max(np.abs(O.filter_z(g, npass, nyq))) < 1e-14
    F = np.random.default_rng(3).normal(size=n)
    assert np.array_equal(O.filter_z(g, 0, F), F)


def pin_filter_open_z(O):
    """With z open the filter sees zero beyond the ends: each pass treats the
    outside as zero (checked against the passes applied by hand with zero
    padding on a short open box)."""
    n = (2, 2, 12)
    rng = np.random.default_rng(4)
    F = rng.normal(size=n)
    g = O.grid(n, zopen=True)
    for npass in (1, 3):
        got = O.filter_z(g, npass, F)
        ref = F.copy()
        stencils = [(0.25, 0.5)] * npass + [(-0.25 * npass, 1.0 + 0.5 * npass)]
        for a, b in stencils:
            pad = np.concatenate([np.zeros(n[:2] + (1,)), ref, np.zeros(n[:2] + (1,))], axis=2)
            ref = a * pad[:, :, :-2] + b * pad[:, :, 1:-1] + a * pad[:, :, 2:]
        assert np.max(np.abs(got - ref)) < 1e-13, npass


ALL_PINS.extend([pin_filter_transfer_function, pin_filter_open_z])


def pin_continuity_unequal_weights(O):
    """Discrete continuity over a full PIC step with unequal particle weights
    (orders 1-3): the charge density before and after uses each particle's
    own weight, so a current that took another particle's weight would leave
    a residual of the order of the weights' spread."""
    n = (8, 8, 8)
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    rng = np.random.default_rng(61)
    for p in (1, 2, 3):
        parts = inputs.uniform_plasma(60 + p, n, 2, sigma_u=0.5)
        parts["w"] = parts["w"] * (0.25 + 1.5 * rng.random(parts["w"].size))
        F = np.zeros((9,) + n)
        r0 = O.rho(g, p, -1.0, parts["x"], parts["y"], parts["z"], parts["w"])
        O.pic_step(g, p, dt, -1.0, 1.0, parts, F)
        r1 = O.rho(g, p, -1.0, parts["x"], parts["y"], parts["z"], parts["w"])
        res = r1 - r0 + dt * O.div_edge(g, F[6:9])
        assert np.max(np.abs(res)) < 1e-13 * np.max(np.abs(r0)), p


def pin_current_linear_in_weights(O):
    """With no fields, the step's current is a sum over particles of w times
    a weight-free term: scaling every weight by 3 scales J by 3, and the
    currents of two halves of the particles add up to that of all."""
    n = (8, 8, 8)
    g = O.grid(n)
    dt = inputs.dt_from_cfl((1, 1, 1), 0.99)
    parts = inputs.uniform_plasma(71, n, 2, sigma_u=0.4)
    rng = np.random.default_rng(72)
    parts["w"] = parts["w"] * (0.5 + rng.random(parts["w"].size))

    def current(sel, scale=1.0):
        q = {k: np.ascontiguousarray(v[sel]) for k, v in parts.items()}
        q["w"] = q["w"] * scale
        F = np.zeros((9,) + n)
        O.pic_step(g, 3, dt, -1.0, 1.0, q, F)
        return F[6:9]

    every = np.arange(parts["w"].size)
    J = current(every)
    tol = 1e-13 * np.abs(J).max()
    assert np.max(np.abs(current(every, 3.0) - 3.0 * J)) < tol
    half = parts["w"].size // 2
    assert np.max(np.abs(current(every[:half]) + current(every[half:]) - J)) < tol


ALL_PINS.extend([pin_continuity_unequal_weights, pin_current_linear_in_weights])
