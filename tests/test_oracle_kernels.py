"""Pins for the FP64 oracle's per-particle pieces: shapes, gather, Boris push
and the charge-conserving deposit (Sec. 2, Sec. 5.1, Sec. 5.2).

Every check compares against something fixed independently of the oracle:
the convolution definition of B-splines (numerical quadrature), polynomial
reproduction laws, the Boris rotation angle and orbit radius, the E x B drift,
exact momentum under uniform E, hyperbolic motion, discrete continuity against
an independently written charge deposit, and the Villasenor-Buneman closed
form for linear in-cell moves."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

ORDERS = [1, 2, 3, 4]


# ---------------------------------------------------------------- shapes
def _box(t):
    return 1.0 if abs(t) < 0.5 else (0.5 if abs(t) == 0.5 else 0.0)


@pytest.mark.parametrize("p", ORDERS)
def test_bspline_is_convolution_of_lower_order(p):
    """S_p(t) = int_{t-1/2}^{t+1/2} S_{p-1}(s) ds with S_0 the unit box."""
    lower = _box if p == 1 else (lambda s: oracle.bspline(p - 1, s))
    for t in np.linspace(-3.0, 3.0, 61) + 0.013:
        brk = [b for b in np.arange(-3.0, 3.01, 0.5) if t - 0.5 < b < t + 0.5]
        val, _ = integrate.quad(lower, t - 0.5, t + 0.5, points=brk or None, epsabs=1e-14, epsrel=1e-13)
        assert abs(oracle.bspline(p, t) - val) < 1e-12


@pytest.mark.parametrize("p", ORDERS)
def test_bspline_moments(p):
    """Partition of unity, first moment x; second moment x^2 + (p+1)/12 for
    p >= 2 (the variance of p+1 unit boxes), x^2 + f(1-f) for linear."""
    rng = np.random.default_rng(0)
    for x in rng.uniform(-5, 5, size=50):
        nodes = np.arange(math.floor(x) - 4, math.floor(x) + 5)
        s = np.array([oracle.bspline(p, x - i) for i in nodes])
        assert abs(s.sum() - 1.0) < 1e-14
        assert abs((s * nodes).sum() - x) < 1e-12
        f = x - math.floor(x)
        second = x * x + ((p + 1) / 12.0 if p >= 2 else f * (1 - f))
        assert abs((s * nodes ** 2).sum() - second) < 1e-11


def test_bspline_node_values():
    """Values at a node: quadratic (1/8, 3/4, 1/8), cubic (1/6, 2/3, 1/6)."""
    assert [oracle.bspline(2, t) for t in (-1, 0, 1)] == pytest.approx([1 / 8, 3 / 4, 1 / 8], abs=1e-15)
    assert [oracle.bspline(3, t) for t in (-1, 0, 1)] == pytest.approx([1 / 6, 2 / 3, 1 / 6], abs=1e-15)
    assert oracle.bspline(1, 0.25) == pytest.approx(0.75)


# ---------------------------------------------------------------- gather
YEE = {0: (0.5, 0, 0), 1: (0, 0.5, 0), 2: (0, 0, 0.5), 3: (0, 0.5, 0.5), 4: (0.5, 0, 0.5), 5: (0.5, 0.5, 0)}


def _fill_linear(sim, a, b):
    """Component c at node (i,j,k) := a[c] + b[c] . X_c, X_c = physical Yee location."""
    s = sim.s
    dim = s.dim
    n = [s.n[0], s.n[1], s.n[2]]
    d = [s.d[0], s.d[1], s.d[2]]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = [i, j, k]
    for c in range(6):
        X = [(idx[ax] + YEE[c][ax]) * d[ax] for ax in range(3)]
        val = a[c] + sum(b[c][ax] * X[ax] for ax in range(dim))
        arr = sim.E if c < 3 else sim.B
        cc = c % 3
        arr[cc * sim.ncell:(cc + 1) * sim.ncell] = val.reshape(-1)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("p", ORDERS)
def test_gather_reproduces_constant_and_linear_fields(dim, p):
    """B-splines reproduce degree-1 polynomials, so the gather of a linear
    field is exact at every Yee location; a wrong stagger offset shows up as
    an error of b*d/2."""
    n = (16, 12, 10)[:dim]
    d = (0.3, 0.7, 0.45)[:dim]
    sim = oracle.Sim(dim, n, d, 0.1, p)
    rng = np.random.default_rng(p + 10 * dim)
    a = rng.normal(size=6)
    b = rng.normal(size=(6, 3))
    _fill_linear(sim, a, b)
    for _ in range(20):
        x = [rng.uniform(4, n[ax] - 4) for ax in range(dim)]
        out = sim.gather(x)
        expect = [a[c] + sum(b[c][ax] * x[ax] * d[ax] for ax in range(dim)) for c in range(6)]
        np.testing.assert_allclose(out, expect, rtol=0, atol=1e-12)
    b[:] = 0
    _fill_linear(sim, a, b)
    np.testing.assert_allclose(sim.gather([rng.uniform(0, n[ax]) for ax in range(dim)]), a, atol=1e-13)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_gather_quadratic_field_second_moment(p):
    """f(X) = X^2 along axis 0 gathers to x^2 + (p+1)/12 (cells^2)."""
    sim = oracle.Sim(2, (20, 8), (1.0, 1.0), 0.1, p)
    a = np.zeros(6)
    for c in range(6):
        off = YEE[c][0]
        i = np.arange(20)
        val = np.tile((i + off) ** 2, 8)
        arr = sim.E if c < 3 else sim.B
        arr[(c % 3) * sim.ncell:(c % 3 + 1) * sim.ncell] = val
    for x0 in (7.1, 8.5, 9.93):
        out = sim.gather([x0, 3.3])
        np.testing.assert_allclose(out, x0 * x0 + (p + 1) / 12.0, atol=1e-11)


# ---------------------------------------------------------------- Boris
def test_boris_gyration_angle_radius_and_energy():
    """Uniform B, E = 0: |u| is conserved, the momentum turns by
    theta = 2 atan(|q| B dt / (2 m gamma)) per step, and the orbit vertices lie
    on a circle of radius (|v| dt / 2) / sin(theta / 2)."""
    q, m, B0, dt = -1.0, 1.0, 2.5, 0.2
    u = np.array([3.0, 0.0, 0.7])
    gamma = math.sqrt(1 + u @ u)
    theta = 2 * math.atan(abs(q) * B0 * dt / (2 * m * gamma))
    eb = [0, 0, 0, 0, 0, B0]
    pos = [np.zeros(3)]
    uu = u.copy()
    for n in range(1, 200):
        uu = oracle.boris(q / m, dt, eb, uu)
        pos.append(pos[-1] + dt * uu / gamma)
        assert abs(np.linalg.norm(uu) - np.linalg.norm(u)) < 1e-12
        ang = math.atan2(uu[1], uu[0])
        expect = math.remainder(n * theta, 2 * math.pi)  # q<0, B along +z: counter-clockwise
        assert abs(math.remainder(ang - expect, 2 * math.pi)) < 1e-10
        assert abs(uu[2] - 0.7) < 1e-13
    P = np.array(pos)[:, :2]
    vperp = 3.0 / gamma
    R = (vperp * dt / 2) / math.sin(theta / 2)
    # centre from three vertices
    (x1, y1), (x2, y2), (x3, y3) = P[0], P[37], P[91]
    A = np.array([[x2 - x1, y2 - y1], [x3 - x1, y3 - y1]]) * 2
    rhs = np.array([x2 ** 2 - x1 ** 2 + y2 ** 2 - y1 ** 2, x3 ** 2 - x1 ** 2 + y3 ** 2 - y1 ** 2])
    ctr = np.linalg.solve(A, rhs)
    np.testing.assert_allclose(np.linalg.norm(P - ctr, axis=1), R, rtol=1e-10)


def test_boris_uniform_e_is_exact():
    """B = 0: u^{n+1/2} = u^{n-1/2} + (q/m) E dt exactly, at any gamma."""
    E = np.array([0.3, -1.2, 2.0])
    u = np.array([0.1, 5.0, -2.0])
    uu = u.copy()
    for _ in range(500):
        uu = oracle.boris(-1.0, 0.05, list(E) + [0, 0, 0], uu)
    np.testing.assert_allclose(uu, u - E * 0.05 * 500, rtol=1e-12, atol=1e-12)


def test_boris_hyperbolic_motion():
    """Constant E from rest: x(t) = (m c^2/|qE|)(sqrt(1 + (qEt/m)^2) - 1),
    reproduced by push + leapfrog move to O(dt^2)."""
    E0, dt = 0.8, 0.01
    x = 0.0
    # start the leapfrog at u^{1/2} = -E0 dt/2 (q = -1): u(t) = -E0 t
    uu = np.array([-0.5 * E0 * dt, 0.0, 0.0])
    T = 4.0
    for _ in range(int(round(T / dt))):
        g = math.sqrt(1 + uu @ uu)
        x += dt * uu[0] / g
        uu = oracle.boris(-1.0, dt, [E0, 0, 0, 0, 0, 0], uu)
    exact = -(math.sqrt(1 + (E0 * T) ** 2) - 1) / E0
    assert abs(x - exact) < 5e-4 * abs(exact)


def test_boris_exb_drift():
    """E perpendicular to B, |E| < |B|: the guiding centre drifts at E x B / B^2."""
    E0, B0, dt = 0.02, 1.0, 0.05
    eb = [0, E0, 0, 0, 0, B0]
    uu = np.zeros(3)
    x = np.zeros(3)
    theta = 2 * math.atan(B0 * dt / 2)
    steps = int(round(200 * 2 * math.pi / theta))  # 200 discrete gyro-periods
    for _ in range(steps):
        uu = oracle.boris(-1.0, dt, eb, uu)
        x += dt * uu / math.sqrt(1 + uu @ uu)
    vd = x / (steps * dt)
    assert abs(vd[0] - E0 / B0) < 2e-3 * E0 / B0
    assert abs(vd[1]) < 2e-3 * E0 / B0


# ---------------------------------------------------------------- deposit
def _div_j(sim, J):
    s = sim.s
    nc = sim.ncell
    shp = sim.shape
    out = np.zeros(shp)
    for a in range(s.dim):
        Ja = J[a * nc:(a + 1) * nc].reshape(shp)
        axis = s.dim - 1 - a  # array axes are (z, y, x)
        out += (Ja - np.roll(Ja, 1, axis=axis)) / s.d[a]
    return out.reshape(-1)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("p", ORDERS)
def test_deposit_satisfies_discrete_continuity(dim, p):
    """(rho^{n+1} - rho^n)/dt + div J = 0 to round-off on tiny periodic grids,
    rho from the independent plain charge deposit; moves cross the periodic
    boundary too."""
    n = (7, 6, 6)[:dim]
    d = (0.4, 0.3, 0.5)[:dim]
    dt = 0.11
    sim = oracle.Sim(dim, n, d, dt, p)
    rng = np.random.default_rng(100 * dim + p)
    for trial in range(25):
        xo = np.array([rng.uniform(0, n[a]) for a in range(dim)])
        xn = xo + rng.uniform(-0.95, 0.95, size=dim)
        qw = rng.uniform(-2, 2)
        J = sim.deposit_current(qw, xo, xn, vz=0.3)
        r0 = sim.deposit_rho(qw, xo)
        r1 = sim.deposit_rho(qw, xn)
        resid = (r1 - r0) / dt + _div_j(sim, J)
        assert np.max(np.abs(resid)) < 1e-12 * max(1.0, np.max(np.abs(r0)) / dt)
        # total current identity: sum_nodes J_a = q w (x_new - x_old)_a d_a / dt
        for a in range(dim):
            tot = J[a * sim.ncell:(a + 1) * sim.ncell].sum()
            assert abs(tot - qw * (xn[a] - xo[a]) * d[a] / dt) < 1e-12
        if dim == 2:
            assert abs(J[2 * sim.ncell:].sum() - qw * 0.3) < 1e-12


def test_linear_deposit_equals_villasenor_buneman_in_cell():
    """Linear order, 2D, move inside one cell from (a0,b0) to (a1,b1):
    J_x(i+1/2, j) = q w v_x (1 - bbar), J_x(i+1/2, j+1) = q w v_x bbar,
    J_y(i, j+1/2) = q w v_y (1 - abar), J_y(i+1, j+1/2) = q w v_y abar;
    J_z(i,j) is q w v_z times the path average of S_x S_y."""
    dx, dy, dt = 0.5, 0.25, 0.1
    sim = oracle.Sim(2, (6, 6), (dx, dy), dt, 1)
    rng = np.random.default_rng(7)
    for _ in range(20):
        a0, b0, a1, b1 = rng.uniform(0.01, 0.99, size=4)
        i, j = 2, 3
        qw, vz = -0.7, 0.4
        J = sim.deposit_current(qw, [i + a0, j + b0], [i + a1, j + b1], vz)
        nc = sim.ncell
        Jx = J[:nc].reshape(6, 6)
        Jy = J[nc:2 * nc].reshape(6, 6)
        Jz = J[2 * nc:].reshape(6, 6)
        vx, vy = (a1 - a0) * dx / dt, (b1 - b0) * dy / dt
        ab, bb = 0.5 * (a0 + a1), 0.5 * (b0 + b1)
        assert Jx[j, i] == pytest.approx(qw * vx * (1 - bb), abs=1e-13)
        assert Jx[j + 1, i] == pytest.approx(qw * vx * bb, abs=1e-13)
        assert Jy[j, i] == pytest.approx(qw * vy * (1 - ab), abs=1e-13)
        assert Jy[j, i + 1] == pytest.approx(qw * vy * ab, abs=1e-13)
        assert np.count_nonzero(np.abs(Jx) > 1e-15) <= 2
        # J_z: exact path average of the bilinear weight (Gauss-Legendre, exact for quadratics)
        ts, ws = np.polynomial.legendre.leggauss(4)
        ts, ws = 0.5 * (ts + 1), 0.5 * ws
        for (ii, jj) in [(i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)]:
            xa = a0 + ts * (a1 - a0) + i
            ya = b0 + ts * (b1 - b0) + j
            avg = np.sum(ws * np.maximum(0, 1 - np.abs(xa - ii)) * np.maximum(0, 1 - np.abs(ya - jj)))
            assert Jz[jj, ii] == pytest.approx(qw * vz * avg, abs=1e-13)


def test_deposit_at_rest_gives_only_out_of_plane_current():
    sim = oracle.Sim(2, (6, 6), (0.5, 0.5), 0.1, 2)
    x = [2.3, 3.6]
    J = sim.deposit_current(1.0, x, x, vz=0.5)
    nc = sim.ncell
    assert np.all(J[:2 * nc] == 0)
    np.testing.assert_allclose(J[2 * nc:], 0.5 * sim.deposit_rho(1.0, x), atol=1e-15)
