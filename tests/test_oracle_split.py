"""Pins for the oracle's virtual-trajectory deposit (Sec. 5.2 step iv: the
move is cut into up to four pieces where it crosses a boundary between the
grid points nearest the particle, each piece deposited as a move of its own).

* Discrete continuity (rho^{n+1} - rho^n)/dt + div J = 0 to round-off on tiny
  periodic grids, every order, 2D and 3D, with moves that cross boundaries
  along several axes at once and across the periodic seam; rho from the
  independent charge deposit.
* Total-current identity: sum over nodes of J_a = q w (x_new - x_old)_a d_a/dt.
* A move that crosses no boundary gives exactly the undivided deposit.
* Linear shapes: each piece stays in one cell, and the current is the sum of
  Villasenor and Buneman's in-cell closed form over the pieces, which are cut
  at the cell faces the move crosses.
"""
import numpy as np
import pytest

import oracle

ORDERS = [1, 2, 3, 4]


def _div_j(sim, J):
    s = sim.s
    nc = sim.ncell
    shp = sim.shape
    out = np.zeros(shp)
    for a in range(s.dim):
        Ja = J[a * nc:(a + 1) * nc].reshape(shp)
        out += (Ja - np.roll(Ja, 1, axis=s.dim - 1 - a)) / s.d[a]
    return out.reshape(-1)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("p", ORDERS)
def test_split_deposit_conserves_charge_and_total_current(dim, p):
    n = (7, 6, 6)[:dim]
    d = (0.4, 0.3, 0.5)[:dim]
    dt = 0.11
    sim = oracle.Sim(dim, n, d, dt, p, split=True)
    rng = np.random.default_rng(31 * dim + p)
    crossings = 0
    off = 0.5 if p % 2 == 0 else 0.0
    for _ in range(40):
        xo = np.array([rng.uniform(0, n[a]) for a in range(dim)])
        xn = xo + rng.uniform(-0.95, 0.95, size=dim)
        crossings += sum(int(np.floor(xo[a] - off) != np.floor(xn[a] - off)) for a in range(dim))
        qw = rng.uniform(-2, 2)
        J = sim.deposit_current_split(qw, xo, xn, vz=0.3)
        r0 = sim.deposit_rho(qw, xo)
        r1 = sim.deposit_rho(qw, xn)
        resid = (r1 - r0) / dt + _div_j(sim, J)
        assert np.max(np.abs(resid)) < 1e-12 * max(1.0, np.max(np.abs(r0)) / dt)
        for a in range(dim):
            tot = J[a * sim.ncell:(a + 1) * sim.ncell].sum()
            assert abs(tot - qw * (xn[a] - xo[a]) * d[a] / dt) < 1e-12
        if dim == 2:
            assert abs(J[2 * sim.ncell:].sum() - qw * 0.3) < 1e-12
    assert crossings > 20  # the pieces really were cut


@pytest.mark.parametrize("p", ORDERS)
def test_move_inside_one_node_cell_is_not_split(p):
    sim = oracle.Sim(3, (6, 6, 6), (0.4, 0.3, 0.5), 0.1, p)
    rng = np.random.default_rng(p)
    off = 0.5 if p % 2 == 0 else 0.0
    for _ in range(20):
        base = rng.integers(1, 4, size=3) + off
        xo = base + rng.uniform(0.05, 0.95, size=3)
        xn = base + rng.uniform(0.05, 0.95, size=3)
        a = sim.deposit_current(0.8, xo, xn, 0.0)
        b = sim.deposit_current_split(0.8, xo, xn, 0.0)
        assert np.array_equal(a, b)


def _vb_piece(J, nc, shape, i, j, a0, b0, a1, b1, qw, dx, dy, dt, vzf):
    """Villasenor-Buneman current of a 2D linear move inside cell (i, j)
    from offsets (a0, b0) to (a1, b1): J_x on the cell's two x edges, J_y on
    its two y edges, and q w v_z times the path average of the bilinear
    weight (exact by Gauss-Legendre, the integrand being quadratic)."""
    ny, nx = shape
    Jx = J[:nc].reshape(shape)
    Jy = J[nc:2 * nc].reshape(shape)
    Jz = J[2 * nc:].reshape(shape)
    vx, vy = (a1 - a0) * dx / dt, (b1 - b0) * dy / dt
    ab, bb = 0.5 * (a0 + a1), 0.5 * (b0 + b1)
    Jx[j % ny, i % nx] += qw * vx * (1 - bb)
    Jx[(j + 1) % ny, i % nx] += qw * vx * bb
    Jy[j % ny, i % nx] += qw * vy * (1 - ab)
    Jy[j % ny, (i + 1) % nx] += qw * vy * ab
    ts, ws = np.polynomial.legendre.leggauss(4)
    ts, ws = 0.5 * (ts + 1), 0.5 * ws
    xa, ya = a0 + ts * (a1 - a0), b0 + ts * (b1 - b0)
    for di in (0, 1):
        for dj in (0, 1):
            avg = np.sum(ws * np.maximum(0, 1 - np.abs(xa - di)) * np.maximum(0, 1 - np.abs(ya - dj)))
            Jz[(j + dj) % ny, (i + di) % nx] += qw * vzf * avg


def test_linear_split_equals_villasenor_buneman_pieces_across_faces():
    dx, dy, dt = 0.5, 0.25, 0.1
    shape = (6, 7)
    sim = oracle.Sim(2, (7, 6), (dx, dy), dt, 1)
    nc = sim.ncell
    rng = np.random.default_rng(17)
    both = 0
    for _ in range(40):
        xo = np.array([rng.uniform(1, 5), rng.uniform(1, 4)])
        xn = xo + rng.uniform(-0.95, 0.95, size=2)
        qw, vz = rng.uniform(-2, 2), rng.uniform(-1, 1)
        got = sim.deposit_current_split(qw, xo, xn, vz)
        # pieces cut at the cell faces crossed, in order along the move
        ts = [(np.floor(max(xo[a], xn[a])) - xo[a]) / (xn[a] - xo[a])
              for a in range(2) if np.floor(xo[a]) != np.floor(xn[a])]
        both += len(ts) == 2
        cuts = [0.0] + sorted(ts) + [1.0]
        want = np.zeros(3 * nc)
        for t0, t1 in zip(cuts[:-1], cuts[1:]):
            ps = xo + t0 * (xn - xo)
            pe = xo + t1 * (xn - xo)
            cell = np.floor(0.5 * (ps + pe))  # the piece's cell (its midpoint's)
            _vb_piece(want, nc, shape, int(cell[0]), int(cell[1]), ps[0] - cell[0], ps[1] - cell[1],
                      pe[0] - cell[0], pe[1] - cell[1], qw, dx, dy, dt, vz * (t1 - t0))
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * max(1.0, np.max(np.abs(want))))
    assert both > 3  # moves crossing an x and a y face (three pieces)


def test_split_step_conserves_charge_in_a_thermal_plasma():
    """The whole loop with the split deposit keeps div E - (rho - rho_0) at
    round-off (the pieces conserve charge one by one)."""
    from paper_1310_0930_gb300 import inputs
    w = inputs.thermal_2d(n=(16, 12), steps=15, order=2)
    w.uth = 0.1
    parts = inputs.background(w)
    sim = oracle.Sim(2, w.n, w.d, w.dt, 2, split=True)
    x = np.zeros((3, parts.n))
    x[:2] = parts.positions64()
    sim.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64))
    rho0 = sim.charge()
    for _ in range(w.steps):
        sim.step(1)
        r = sim.div_e() - (sim.charge() - rho0)
        assert np.max(np.abs(r)) < 1e-12 * np.max(np.abs(rho0))
