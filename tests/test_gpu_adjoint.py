"""Adjoint form: the hand-written reverse kernels against (a) the forward
step, through transpose (dot-product) checks of the field update, and
(b) central finite differences of the FP64 oracle for the gradient of the
trailing-window kinetic-energy objective with respect to the density-profile
knots and the laser amplitude a0 (plus the torch.autograd path)."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import FIELD_NAMES, oracle_for
from paper_1310_0930_gb300 import inputs
from paper_1310_0930_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["open_2d", "periodic_2d", "open_3d"])
def test_field_update_transpose(case):
    """<M v, lam> = <v, M^T lam> for one step's field update M (no particles,
    no antenna), including the Mur ends and the frozen entries beyond them."""
    if case == "open_2d":
        w = inputs.lwfa_2d(nx=24, nz=40)
    elif case == "periodic_2d":
        w = inputs.thermal_2d(n=(20, 28))
    else:
        w = inputs.lwfa_3d(n=(8, 12, 24))
    w.laser = None
    w.window = None
    rng = np.random.default_rng(7)
    shape = tuple(reversed(w.n))
    v = rng.normal(size=(6,) + shape).astype(np.float32)
    lam = rng.normal(size=(6,) + shape).astype(np.float32)
    fwd = Simulation(w)
    for c, name in enumerate(FIELD_NAMES):
        fwd.set_field(name, v[c])
    fwd.step(1)
    mv = np.stack([fwd.field(n) for n in FIELD_NAMES]).astype(np.float64)
    fwd.close()
    adj = Simulation(w)
    mtl, _ = adj.adjoint_fields(lam, 0.0)
    adj.close()
    lhs = float(np.sum(mv * lam.astype(np.float64)))
    rhs = float(np.sum(v.astype(np.float64) * mtl.astype(np.float64)))
    scale = float(np.sum(np.abs(mv * lam)))
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs)


def _adjoint_case():
    knots = np.array([0.010, 0.012, 0.008, 0.011])
    w = inputs.lwfa_2d(nx=32, nz=96, ppc=(2, 2), density=0.01, a0=1.2, waist=6.0, steps=48, seed=9)
    w.laser.fwhm = 5.0
    w.window = None
    w.knots = knots
    w.knot_z = (0.0, 96 * 0.3)
    obj = dict(z_lo=5.0, z_hi=35.0, width=2.0)
    return w, obj


def _oracle_L(w, knots, a0, obj):
    """Objective after w.steps oracle steps, FP64 weights from the knots (for
    the loaded plasma and, with a moving window, the plasma it injects)."""
    w = inputs.Workload(**{**w.__dict__})
    w.laser = inputs.Laser(**{**w.laser.__dict__})
    w.laser.a0 = a0
    w.knots = np.asarray(knots, dtype=np.float64)
    parts = inputs.background(w)
    x = np.zeros((3, parts.n))
    x[: w.dim] = parts.positions64()
    zlab = x[w.dim - 1] * w.d[-1]
    wt = np.interp(zlab, np.linspace(w.knot_z[0], w.knot_z[1], len(knots)), knots) / w.ppc_total
    sim = oracle_for(w)
    layer = int(np.prod(w.n[:-1])) * w.ppc_total  # particles one window shift injects
    sim.load(x, parts.u.astype(np.float64), wt, capacity=parts.n + 16 + (w.steps * layer if w.window else 0))
    sim.step(w.steps)
    xx, uu, ww = sim.particles()
    z = xx[w.dim - 1]
    lg = lambda t: 1.0 / (1.0 + np.exp(-t))
    sig = lg((z - obj["z_lo"]) / obj["width"]) * lg((obj["z_hi"] - z) / obj["width"])
    K = np.sqrt(1.0 + np.sum(uu ** 2, axis=0)) - 1.0
    return float(np.sum(ww * K * sig) / np.sum(ww * sig))


@pytest.mark.parametrize("keep", [0, -1, 1])
def test_gradient_matches_fp64_oracle_finite_differences(keep):
    """keep: checkpoint segments recorded by the forward run (0 = all that fit,
    here all three; -1 = every segment recomputed; 1 = the last one kept)."""
    w, obj = _adjoint_case()
    parts = inputs.background(w)
    sim = Simulation(w, track_ids=True, per_particle_weight=True, tuning={"adjoint_keep": keep})
    sim.load(parts)
    sim.adjoint_begin(w.steps, 16)
    sim.step(w.steps)
    res = sim.adjoint_backward(obj["z_lo"], obj["z_hi"], obj["width"], n_knots=len(w.knots), n_ids=parts.n)
    sim.close()
    knots = np.asarray(w.knots, dtype=np.float64)
    a0 = w.laser.a0
    L0 = _oracle_L(w, knots, a0, obj)
    assert abs(res["L"] - L0) <= 1e-4 * abs(L0)
    fd = []
    for k in range(len(knots)):
        h = 1e-3 * knots[k]
        kp, km = knots.copy(), knots.copy()
        kp[k] += h
        km[k] -= h
        fd.append((_oracle_L(w, kp, a0, obj) - _oracle_L(w, km, a0, obj)) / (2 * h))
    h = 1e-3 * a0
    fd_a0 = (_oracle_L(w, knots, a0 + h, obj) - _oracle_L(w, knots, a0 - h, obj)) / (2 * h)
    fd = np.array(fd)
    g = np.asarray(res["dL_dknots"])
    assert np.max(np.abs(g - fd)) <= 1e-3 * np.max(np.abs(fd)), (g, fd)
    assert abs(res["dL_da0"] - fd_a0) <= 1e-3 * abs(fd_a0), (res["dL_da0"], fd_a0)
    # per-particle weights: the knot gradient is their linear image
    assert res["dL_dw"] is not None and np.all(np.isfinite(res["dL_dw"]))


def _window_case():
    """2D LWFA (64 cells along z, pulse of FWHM 3) whose window starts moving
    at t = 12, once the pulse is in the box, and shifts 53 times in the 100
    steps: the layers injected at the front drift back through the pulse
    (cells 0 to 30), and the objective's window (cells 3 to 50) holds loaded
    and injected plasma.  Knots over lab z 0 to 36: the loaded plasma spans
    0 to 19, the injected layers 19 to 34, so the last two knots reach the
    objective only through injected particles (their weights and the fields
    they drive)."""
    knots = np.array([0.010, 0.013, 0.008, 0.012, 0.009])
    w = inputs.lwfa_2d(nx=32, nz=64, ppc=(2, 2), density=0.01, a0=1.2, waist=6.0, steps=100, seed=9)
    w.laser.fwhm = 3.0
    w.window.t0 = 12.0
    w.knots = knots
    w.knot_z = (0.0, 36.0)
    obj = dict(z_lo=3.0, z_hi=50.0, width=2.0)
    return w, obj


@pytest.mark.parametrize("keep", [0, -1])
def test_gradient_through_the_moving_window(keep):
    """keep 0: every segment recorded by the forward run; -1: every segment
    recomputed from its checkpoint (window origin, shifts and the unsorted
    tail restored)."""
    w, obj = _window_case()
    parts = inputs.background(w)
    sim = Simulation(w, track_ids=True, per_particle_weight=True, tuning={"adjoint_keep": keep})
    sim.load(parts)
    sim.adjoint_begin(w.steps, 16)
    sim.step(w.steps)
    d = sim.diagnostics()
    assert d["shifts"] >= 50 and d["status"] == 0
    # ids: the loaded particles keep 0 .. n-1, each shift's layer of m
    # particles gets n + (k - 1) m + j
    p = sim.particles()
    layer = w.n[0] * w.ppc_total
    ids = p["id"]
    assert len(np.unique(ids)) == len(ids) and ids.min() >= 0
    assert ids.max() < parts.n + d["shifts"] * layer
    assert np.count_nonzero(ids >= parts.n + (d["shifts"] - 1) * layer) == layer  # the newest layer
    res = sim.adjoint_backward(obj["z_lo"], obj["z_hi"], obj["width"], n_knots=len(w.knots), n_ids=parts.n)
    sim.close()
    knots = np.asarray(w.knots, dtype=np.float64)
    a0 = w.laser.a0
    L0 = _oracle_L(w, knots, a0, obj)
    assert abs(res["L"] - L0) <= 1e-4 * abs(L0), (res["L"], L0)
    fd = []
    for k in range(len(knots)):
        h = 1e-3 * knots[k]
        kp, km = knots.copy(), knots.copy()
        kp[k] += h
        km[k] -= h
        fd.append((_oracle_L(w, kp, a0, obj) - _oracle_L(w, km, a0, obj)) / (2 * h))
    fd = np.array(fd)
    g = np.asarray(res["dL_dknots"])
    assert np.max(np.abs(g - fd)) <= 1e-3 * np.max(np.abs(fd)), (g, fd)
    # the last two knots lie beyond the loaded plasma: only injected layers carry them
    assert np.min(np.abs(fd[-2:])) > 1e-2 * np.max(np.abs(fd)), fd
    # a0 moves particles across the window's rear margin, where they are
    # dropped: L(a0) has small jumps, and its central differences vary by
    # about 1 % with the step (the knot differences agree to 1e-5); the
    # adjoint, the derivative of the smooth part, must lie within their range
    fa = []
    for rel in (1e-2, 3e-3, 1e-3, 3e-4, 1e-4):
        h = rel * a0
        fa.append((_oracle_L(w, knots, a0 + h, obj) - _oracle_L(w, knots, a0 - h, obj)) / (2 * h))
    lo, hi = min(fa), max(fa)
    tol = 1e-3 * max(abs(lo), abs(hi))
    assert lo - tol <= res["dL_da0"] <= hi + tol, (res["dL_da0"], fa)


def test_torch_autograd_function():
    """The torch.autograd.Function path gives the gradient of
    pic_adjoint_backward on the same run, and that of central differences of
    the FP64 oracle within 1e-3."""
    import torch
    from paper_1310_0930_gb300 import adjoint
    w, obj = _adjoint_case()
    knots = torch.tensor(w.knots, dtype=torch.float64, requires_grad=True)
    a0 = torch.tensor(w.laser.a0, dtype=torch.float64, requires_grad=True)
    L = adjoint.objective(knots, a0, w, adjoint.Objective(**obj), steps=w.steps, checkpoint_every=16)
    L.backward()
    gk = knots.grad.numpy()
    ga = float(a0.grad)
    assert np.all(np.isfinite(gk)) and math.isfinite(ga)
    # the C ABI directly, same run
    parts = inputs.background(w)
    sim = Simulation(w, track_ids=True, per_particle_weight=True)
    sim.load(parts)
    sim.adjoint_begin(w.steps, 16)
    sim.step(w.steps)
    res = sim.adjoint_backward(obj["z_lo"], obj["z_hi"], obj["width"], n_knots=len(w.knots))
    sim.close()
    assert abs(float(L.detach()) - res["L"]) <= 1e-6 * abs(res["L"])
    assert np.max(np.abs(gk - res["dL_dknots"])) <= 1e-4 * np.max(np.abs(res["dL_dknots"]))
    assert abs(ga - res["dL_da0"]) <= 1e-4 * abs(res["dL_da0"])
    # central differences of the FP64 oracle (h = 1e-3 of each value)
    kn = np.asarray(w.knots, dtype=np.float64)
    fd = []
    for k in range(len(kn)):
        h = 1e-3 * kn[k]
        kp, km = kn.copy(), kn.copy()
        kp[k] += h
        km[k] -= h
        fd.append((_oracle_L(w, kp, w.laser.a0, obj) - _oracle_L(w, km, w.laser.a0, obj)) / (2 * h))
    fd = np.array(fd)
    h = 1e-3 * w.laser.a0
    fd_a0 = (_oracle_L(w, kn, w.laser.a0 + h, obj) - _oracle_L(w, kn, w.laser.a0 - h, obj)) / (2 * h)
    assert np.max(np.abs(gk - fd)) <= 1e-3 * np.max(np.abs(fd)), (gk, fd)
    assert abs(ga - fd_a0) <= 1e-3 * abs(fd_a0), (ga, fd_a0)
    assert ga > 0  # a stronger driver heats the window's electrons


def test_gradient_plateau_on_the_configured_fd_copy():
    """The adjoint configuration's finite-difference copy: 2D LWFA 128 x 64
    cells (dz = 0.3, dx = 1, dt = 0.28), 16 ppc, 32 density knots around
    0.005 n_c, a0 = 3 (pulse and waist scaled to the copy).  Central
    differences of the FP64 oracle over h in {1e-2, 1e-3, 1e-4, 1e-5} of
    each value, for a0 and the three knots of largest gradient: the
    differences settle on a plateau (h = 1e-3 and 1e-4 agree to 1e-4), and the
    library's gradient agrees with the plateau value within 1e-3."""
    base = inputs.adjoint_2d(steps=90)
    knots = np.asarray(base.knots, dtype=np.float64)
    w = inputs.lwfa_2d(nx=64, nz=128, ppc=(4, 4), density=0.005, a0=3.0, waist=10.0, steps=90, seed=5,
                       knots=knots)
    w.laser.fwhm = 6.0
    w.window = None
    w.knot_z = (0.0, 128 * 0.3)
    obj = dict(z_lo=8.0, z_hi=60.0, width=2.0)
    parts = inputs.background(w)
    sim = Simulation(w, track_ids=True, per_particle_weight=True)
    sim.load(parts)
    sim.adjoint_begin(w.steps, 30)
    sim.step(w.steps)
    res = sim.adjoint_backward(obj["z_lo"], obj["z_hi"], obj["width"], n_knots=len(knots))
    sim.close()
    L0 = _oracle_L(w, knots, w.laser.a0, obj)
    assert abs(res["L"] - L0) <= 1e-4 * abs(L0)
    g = np.asarray(res["dL_dknots"])
    picks = [("a0", None)] + [("knot", int(k)) for k in np.argsort(-np.abs(g))[:3]]
    got, plateau = [], []
    for kind, k in picks:
        fds = {}
        for rel in (1e-2, 1e-3, 1e-4, 1e-5):
            if kind == "a0":
                h = rel * w.laser.a0
                fds[rel] = (_oracle_L(w, knots, w.laser.a0 + h, obj) - _oracle_L(w, knots, w.laser.a0 - h, obj)) / (2 * h)
            else:
                h = rel * knots[k]
                kp, km = knots.copy(), knots.copy()
                kp[k] += h
                km[k] -= h
                fds[rel] = (_oracle_L(w, kp, w.laser.a0, obj) - _oracle_L(w, km, w.laser.a0, obj)) / (2 * h)
        assert abs(fds[1e-3] - fds[1e-4]) <= 1e-4 * abs(fds[1e-4]), (kind, k, fds)
        plateau.append(fds[1e-4])
        got.append(res["dL_da0"] if kind == "a0" else g[k])
    plateau, got = np.array(plateau), np.array(got)
    assert abs(got[0] - plateau[0]) <= 1e-3 * abs(plateau[0]), (got[0], plateau[0])
    assert np.max(np.abs(got[1:] - plateau[1:])) <= 1e-3 * np.max(np.abs(plateau[1:])), (got, plateau)


def test_profiling_keeps_adjoint_state():
    """Phase profiling of an adjoint-armed forward run leaves the checkpoints
    and records intact: the gradient is the one of an unprofiled run."""
    w, obj = _adjoint_case()
    parts = inputs.background(w)

    def grad(profile):
        sim = Simulation(w, track_ids=True, per_particle_weight=True)
        sim.load(parts)
        sim.adjoint_begin(w.steps, 16)
        if profile:
            sim.profile_begin(w.steps)
        sim.step(w.steps)
        if profile:
            phases, launches = sim.profile_end()
            assert sum(phases.values()) > 0 and launches > 0
        res = sim.adjoint_backward(obj["z_lo"], obj["z_hi"], obj["width"], n_knots=len(w.knots))
        sim.close()
        return res

    a, b = grad(False), grad(True)
    assert abs(a["L"] - b["L"]) <= 1e-6 * abs(a["L"])
    ga, gb = np.asarray(a["dL_dknots"]), np.asarray(b["dL_dknots"])
    assert np.max(np.abs(ga - gb)) <= 1e-4 * np.max(np.abs(ga))
    assert abs(a["dL_da0"] - b["dL_da0"]) <= 1e-4 * abs(a["dL_da0"])


def _particle_map(orc, x, u, w, dim, d, dt, q=-1.0, m=1.0):
    """The particle part of one step in FP64, composed from the oracle's own
    gather, Boris push and current deposit: (E, B held by orc; x, u, w) ->
    (x', u', J); x in cells, J over the grid."""
    n = x.shape[1]
    xn = np.zeros_like(x)
    un = np.zeros_like(u)
    J = np.zeros(3 * orc.ncell)
    for p in range(n):
        eb = orc.gather(x[:, p])
        up = oracle.boris(q / m, dt, eb, u[:, p])
        gam = math.sqrt(1.0 + float(up @ up))
        xp = x[:, p] + dt * up[:dim] / (gam * np.asarray(d[:dim]))
        orc.deposit_current(q * w[p], x[:, p], xp, up[2] / gam, J)
        xn[:, p] = xp
        un[:, p] = up
    return xn, un, J


@pytest.mark.parametrize("dim,order", [(2, 1), (2, 2), (3, 2), (3, 3)])
def test_particle_step_transpose(dim, order):
    """<K v, lam> = <v, K^T lam> for the particle part of one step, K the
    linearisation of (E, B, x, u, w) -> (x', u', J) at a state with smooth
    random fields, random momenta (|u| up to ~2) and weights: K v by central
    differences of the FP64 map composed from the oracle's gather, Boris push
    and deposit (step 1e-6), K^T lam by the library's reverse particle kernel
    (pic_adjoint_particles).  Agreement to FP32 rounding of the reverse sweep."""
    from gpu_helpers import smooth_fields
    if dim == 2:
        w = inputs.thermal_2d(n=(16, 12), order=order)
    else:
        w = inputs.thermal_3d(n=(8, 8, 8), order=order)
    rng = np.random.default_rng(11 + order)
    n = 60
    cell = np.stack([rng.integers(0, m, n) for m in w.n]).astype(np.int32)
    off = rng.uniform(0.05, 0.95, size=(w.dim, n)).astype(np.float32)
    u = (rng.normal(size=(3, n)) * 0.7).astype(np.float32)
    wt = rng.uniform(0.5, 1.5, n).astype(np.float32)
    parts = inputs.Particles(cell, off, u, wt)
    fields = smooth_fields(w, amp=0.3, seed=13)
    gpu = Simulation(w, track_ids=True, per_particle_weight=True)
    gpu.load(parts)
    for name, arr in fields.items():
        gpu.set_field(name, arr)
    shape = tuple(reversed(w.n))
    lam_x = rng.normal(size=(w.dim, n))
    lam_u = rng.normal(size=(3, n))
    lam_j = rng.normal(size=(3,) + shape)
    mx, mu, mw, mf = gpu.adjoint_particles(lam_x, lam_u, lam_j)
    gpu.close()
    # forward map in FP64 at the same state
    orc = oracle_for(w)
    x0 = parts.positions64()
    u0 = u.astype(np.float64)
    w0 = wt.astype(np.float64)
    F0 = {nm: arr.astype(np.float64) for nm, arr in fields.items()}
    vF = {nm: rng.normal(size=shape) * 0.3 for nm in FIELD_NAMES}
    vx = rng.normal(size=x0.shape)
    vu = rng.normal(size=u0.shape)
    vw = rng.normal(size=w0.shape)
    eps = 1e-6

    def F(sign):
        for nm in FIELD_NAMES:
            orc.field(nm)[...] = F0[nm] + sign * eps * vF[nm]
        return _particle_map(orc, x0 + sign * eps * vx, u0 + sign * eps * vu, w0 + sign * eps * vw,
                             w.dim, w.d, w.dt)

    xp, up, Jp = F(+1)
    xm, um, Jm = F(-1)
    lhs = (np.sum(lam_x * (xp - xm)) + np.sum(lam_u * (up - um)) + np.sum(lam_j.reshape(-1) * (Jp - Jm))) / (2 * eps)
    rhs = (np.sum(vx * mx) + np.sum(vu * mu) + np.sum(vw * mw) +
           sum(np.sum(vF[nm] * mf[c].astype(np.float64)) for c, nm in enumerate(FIELD_NAMES)))
    scale = (np.sum(np.abs(vx * mx)) + np.sum(np.abs(vu * mu)) + np.sum(np.abs(vw * mw)) +
             sum(np.sum(np.abs(vF[nm] * mf[c])) for c, nm in enumerate(FIELD_NAMES)))
    assert abs(lhs - rhs) <= 2e-5 * scale, (lhs, rhs, scale)
    # and each input block separately carries weight (the check is not one term's)
    assert np.sum(np.abs(vx * mx)) > 1e-3 * scale and np.sum(np.abs(vu * mu)) > 1e-3 * scale
