"""Shared helpers for the GPU parity tests: run the same seeded input through
the CUDA library (via the C ABI) and through the FP64 oracle."""
import numpy as np

import oracle
from paper_1310_0930_gb300 import inputs
from paper_1310_0930_gb300.sim import Simulation

FIELD_NAMES = ["Ex", "Ey", "Ez", "Bx", "By", "Bz"]


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_for(w: inputs.Workload, capacity=None, nthreads=None, split=False):
    laser = window = None
    if w.laser is not None:
        L = w.laser
        laser = dict(a0=L.a0, waist=L.waist, fwhm=L.fwhm, plane=L.plane, pol=L.pol, omega0=L.omega0,
                     t_peak=L.peak_time())
    if w.window is not None:
        window = dict(v=w.window.v, t0=w.window.t0, ppc=w.ppc, density=w.density)
        if w.knots is not None:
            window.update(knots=w.knots, z0=w.knot_z[0], z1=w.knot_z[1])
    return oracle.Sim(w.dim, w.n, w.d, w.dt, w.order, open_last=w.open_last, laser=laser, window=window,
                      nthreads=nthreads, split=split)


def load_oracle(sim, w, parts: inputs.Particles, extra=0):
    x = np.zeros((3, parts.n))
    x[: w.dim] = parts.positions64()
    sim.load(x, parts.u.astype(np.float64), parts.w.astype(np.float64), capacity=parts.n + extra + 16)


def smooth_fields(w: inputs.Workload, amp=0.05, seed=11, modes=3):
    """Random smooth periodic fields (sum of a few Fourier modes), float32."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(w.n))
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    out = {}
    for name in FIELD_NAMES:
        f = np.zeros(shape)
        for _ in range(modes):
            k = [rng.integers(-2, 3) for _ in shape]
            ph = rng.uniform(0, 2 * np.pi)
            arg = sum(2 * np.pi * k[i] * grids[i] / shape[i] for i in range(len(shape))) + ph
            f += rng.normal() * np.cos(arg)
        out[name] = (amp * f / modes).astype(np.float32)
    return out


def pair(w, parts, *, fields=None, tuning=None, track_ids=True, extra=0, nthreads=None, per_particle_weight=None):
    """GPU simulation and oracle with identical initial state."""
    gpu = Simulation(w, tuning=tuning, track_ids=track_ids, per_particle_weight=per_particle_weight)
    if parts is not None and parts.n:
        gpu.load(parts)
    orc = oracle_for(w, nthreads=nthreads, split=bool((tuning or {}).get("deposit", 0)))
    if parts is not None:
        load_oracle(orc, w, parts, extra=extra)
    if fields:
        for name, arr in fields.items():
            gpu.set_field(name, arr)
            orc.field(name)[...] = arr.astype(np.float64)
    return gpu, orc
