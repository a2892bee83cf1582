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
    """Objective after w.steps oracle steps, FP64 weights from the knots."""
    w = inputs.Workload(**{**w.__dict__})
    w.laser = inputs.Laser(**{**w.laser.__dict__})
    w.laser.a0 = a0
    parts = inputs.background(w)
    x = np.zeros((3, parts.n))
    x[: w.dim] = parts.positions64()
    zlab = x[w.dim - 1] * w.d[-1]
    wt = np.interp(zlab, np.linspace(w.knot_z[0], w.knot_z[1], len(knots)), knots) / w.ppc_total
    sim = oracle_for(w)
    sim.load(x, parts.u.astype(np.float64), wt, capacity=parts.n + 16)
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


def test_torch_autograd_function():
    import torch
    from paper_1310_0930_gb300 import adjoint
    w, obj = _adjoint_case()
    knots = torch.tensor(w.knots, dtype=torch.float64, requires_grad=True)
    a0 = torch.tensor(w.laser.a0, dtype=torch.float64, requires_grad=True)
    L = adjoint.objective(knots, a0, w, adjoint.Objective(**obj), steps=w.steps, checkpoint_every=16)
    L.backward()
    assert knots.grad is not None and a0.grad is not None
    assert torch.all(torch.isfinite(knots.grad)) and math.isfinite(float(a0.grad))
    assert float(a0.grad) > 0  # a stronger driver heats the window's electrons


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
