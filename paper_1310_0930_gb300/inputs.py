"""Seeded synthetic workloads for the EM-PIC timestep.

This module holds the input recipes only (grid, species, laser, window and
the seeded particle loads).  It contains none of the method's arithmetic:
no shapes, gathers, pushes, deposits or field updates.  Both the CUDA path's
tests/bench and the oracle receive the arrays it returns.

Particle positions are produced directly in the split form the paper
recommends for single precision (Sec. 5.1): an integer cell index per axis
plus an FP32 offset in [0, 1) from the cell's lower vertex.  The oracle
receives ``cell + float64(offset)``, i.e. the same FP32-rounded state.

Workloads (lengths in c/omega, omega = omega_p for the thermal plasma and
omega_0 for the laser runs):

* ``thermal_2d``  : 2D periodic 128x128, dx=dy=0.2, dt=0.14, n=1, 4 ppc
                    (2x2 regular + U(-1/8,1/8) jitter), u ~ N(0, 0.01^2),
                    quadratic, 100 steps, seed 1.
* ``lwfa_3d``     : 3D 256x256x1024 (x, y transverse, z = propagation, the
                    slowest axis), dx=dy=1, dz=0.3, dt=0.27 (the 3D Courant
                    limit for these cells is 0.2762, so 0.28 is unstable),
                    n=0.0025 n_c, 8 ppc (2x2x2 regular), cold, a0=4 linearly
                    polarised along x, waist 60, FWHM 30, moving window at c,
                    transverse periodic, open z, quadratic, 500 steps.
* ``bunch_3d``    : 3D 256x256x512 as lwfa_3d plus a Gaussian electron bunch
                    (sigma_z=3, sigma_r=5, 64x peak density, 64 ppc,
                    u_z=100), cubic, 200 steps.
* ``scan_2d``     : 64 independent 2D LWFA runs with seeded parameters.
* ``adjoint_2d``  : 2D 256x1024 LWFA, 16 ppc, 32-knot density profile.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Laser:
    a0: float
    waist: float
    fwhm: float
    omega0: float = 1.0
    t_peak: Optional[float] = None  # default 2*fwhm
    plane: int = 2                 # node index along the propagation (last) axis
    pol: int = 0                   # polarisation axis

    def peak_time(self) -> float:
        return 2.0 * self.fwhm if self.t_peak is None else self.t_peak


@dataclasses.dataclass
class Window:
    v: float = 1.0
    t0: float = 0.0


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    n: tuple            # cells per axis, (nx, ny) or (nx, ny, nz); last axis = propagation
    d: tuple            # cell sizes
    dt: float
    order: int
    ppc: tuple          # particles per cell per axis
    density: float
    uth: float = 0.0
    jitter: float = 0.0  # jitter amplitude as a fraction of the inter-particle spacing
    steps: int = 100
    seed: int = 1
    open_last: bool = False
    laser: Optional[Laser] = None
    window: Optional[Window] = None
    knots: Optional[np.ndarray] = None   # density profile knots (lab frame, last axis)
    knot_z: tuple = (0.0, 0.0)
    bunch: Optional[dict] = None
    mass: float = 1.0    # particle mass in electron masses (charge -1)

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.n))

    @property
    def ppc_total(self) -> int:
        return int(np.prod(self.ppc))

    @property
    def plasma_lo(self) -> int:
        """First cell (last axis) holding plasma when the last axis is open."""
        return self.order + 1 if self.open_last else 0

    @property
    def plasma_hi(self) -> int:
        return self.n[-1] - (self.order + 1) if self.open_last else self.n[-1]

    def n_particles_background(self) -> int:
        ncol = int(np.prod(self.n[:-1]))
        return ncol * (self.plasma_hi - self.plasma_lo) * self.ppc_total


def thermal_2d(n=(128, 128), steps=100, seed=1, order=2) -> Workload:
    return Workload("thermal_2d", 2, tuple(n), (0.2, 0.2), 0.14, order, (2, 2), 1.0,
                    uth=0.01, jitter=0.25, steps=steps, seed=seed)


def thermal_3d(n=(16, 16, 16), steps=20, seed=3, order=2, d=(0.3, 0.3, 0.3), dt=0.15) -> Workload:
    return Workload("thermal_3d", 3, tuple(n), tuple(d), dt, order, (2, 2, 2), 1.0,
                    uth=0.02, jitter=0.25, steps=steps, seed=seed)


def lwfa_3d(n=(256, 256, 1024), steps=500, order=2, with_window=True) -> Workload:
    return Workload("lwfa_3d", 3, tuple(n), (1.0, 1.0, 0.3), 0.27, order, (2, 2, 2), 0.0025,
                    steps=steps, seed=2, open_last=True,
                    laser=Laser(a0=4.0, waist=60.0, fwhm=30.0),
                    window=Window(v=1.0, t0=4.0 * 30.0) if with_window else None)


def bunch_3d(n=(256, 256, 512), steps=200) -> Workload:
    w = lwfa_3d(n=n, steps=steps, order=3)
    w.name = "bunch_3d"
    w.seed = 3
    w.bunch = dict(sigma_z=3.0, sigma_r=5.0, peak=64.0, ppc=(4, 4, 4), uz=100.0)
    return w


def lwfa_2d(nx=128, nz=512, ppc=(2, 2), density=0.005, a0=3.0, waist=40.0, steps=1000,
            seed=4, order=2, knots=None) -> Workload:
    """2D LWFA: axis 0 = transverse x (dx=1), axis 1 = propagation z (dz=0.3)."""
    w = Workload("lwfa_2d", 2, (nx, nz), (1.0, 0.3), 0.28, order, tuple(ppc), density,
                 steps=steps, seed=seed, open_last=True,
                 laser=Laser(a0=a0, waist=waist, fwhm=30.0),
                 window=Window(v=1.0, t0=120.0))
    if knots is not None:
        w.knots = np.asarray(knots, dtype=np.float64)
        w.knot_z = (0.0, nz * 0.3 + steps * 0.28)
    return w


def scan_2d(count=64, seed=4, steps=1000):
    """Parameter scan: uneven independent 2D LWFA runs (seeded)."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(count):
        nz = int(rng.choice([256, 512, 768, 1024, 1280, 1536, 1792, 2048]))
        nx = int(rng.choice([128, 256, 384, 512]))
        dens = float(rng.uniform(0.001, 0.01))
        a0 = float(rng.uniform(1.0, 6.0))
        waist = float(rng.uniform(20.0, 60.0))
        ppc = [(2, 2), (2, 4), (3, 3), (4, 4)][int(rng.integers(0, 4))]
        runs.append(lwfa_2d(nx=nx, nz=nz, ppc=ppc, density=dens, a0=a0, waist=min(waist, nx / 3.0),
                            steps=steps, seed=seed * 1000 + r))
    return runs


def adjoint_2d(nx=256, nz=1024, steps=2000, seed=5, n_knots=32):
    rng = np.random.default_rng(seed)
    knots = 0.005 * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, size=n_knots))
    return lwfa_2d(nx=nx, nz=nz, ppc=(4, 4), density=0.005, a0=3.0, waist=40.0, steps=steps,
                   seed=seed, knots=knots)


# ---------------------------------------------------------------------------
# particle loads
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Particles:
    cell: np.ndarray   # int32 [dim][N], cell index per axis
    off: np.ndarray    # float32 [dim][N], offset in [0, 1) from the lower vertex
    u: np.ndarray      # float32 [3][N], gamma*beta
    w: np.ndarray      # float32 [N], density weight (n / ppc)

    @property
    def n(self) -> int:
        return int(self.cell.shape[1])

    def positions64(self) -> np.ndarray:
        """Global position in cell units, float64 (cell + offset), for the oracle."""
        return self.cell.astype(np.float64) + self.off.astype(np.float64)

    def subset(self, idx) -> "Particles":
        return Particles(self.cell[:, idx].copy(), self.off[:, idx].copy(), self.u[:, idx].copy(),
                         self.w[idx].copy())


def _profile(w: Workload, zlab: np.ndarray) -> np.ndarray:
    if w.knots is None:
        return np.full(zlab.shape, w.density, dtype=np.float64)
    k = np.asarray(w.knots, dtype=np.float64)
    z0, z1 = w.knot_z
    return np.interp(zlab, np.linspace(z0, z1, len(k)), k)


def _clean_offsets(off: np.ndarray) -> np.ndarray:
    off = off.astype(np.float32)
    off = np.where(off >= np.float32(1.0), np.nextafter(np.float32(1.0), np.float32(0.0)), off)
    return np.where(off < 0, np.float32(0.0), off).astype(np.float32)


def background(w: Workload, cells_last: Optional[tuple] = None) -> Particles:
    """Uniform (or profiled) background plasma.

    ppc[a] particles per axis at offsets (m + 1/2)/ppc[a] plus uniform jitter
    of +-jitter/ppc[a]; momenta N(0, uth^2) per component; weight n/ppc.
    ``cells_last`` restricts the load to a range of cells on the last axis.
    """
    rng = np.random.default_rng(w.seed)
    dim = w.dim
    lo, hi = (w.plasma_lo, w.plasma_hi) if cells_last is None else cells_last
    axes = []
    for a in range(dim):
        nlo, nhi = (lo, hi) if a == dim - 1 else (0, w.n[a])
        c = np.arange(nlo, nhi, dtype=np.int32)
        m = (np.arange(w.ppc[a], dtype=np.float64) + 0.5) / w.ppc[a]
        axes.append((c, m))
    # particle ordering: cells x fastest, then sub-positions
    grids_c = np.meshgrid(*[ax[0] for ax in axes], indexing="ij")
    grids_m = np.meshgrid(*[ax[1] for ax in axes], indexing="ij")
    ncell = grids_c[0].size
    nsub = grids_m[0].size
    cell = np.empty((dim, ncell * nsub), dtype=np.int32)
    off = np.empty((dim, ncell * nsub), dtype=np.float32)
    for a in range(dim):
        cell[a] = np.repeat(grids_c[a].reshape(-1), nsub)
        base = np.tile(grids_m[a].reshape(-1), ncell)
        if w.jitter > 0:
            base = base + rng.uniform(-w.jitter, w.jitter, size=base.size) / w.ppc[a]
        off[a] = _clean_offsets(base)
    N = cell.shape[1]
    if w.uth > 0:
        u = rng.normal(0.0, w.uth, size=(3, N)).astype(np.float32)
    else:
        u = np.zeros((3, N), dtype=np.float32)
    zlab = (cell[dim - 1].astype(np.float64) + off[dim - 1]) * w.d[dim - 1]
    wt = (_profile(w, zlab) / w.ppc_total).astype(np.float32)
    return Particles(cell, off, u, wt)


def background_chunks(w: Workload, chunk_cells_last: int = 64):
    """Yield the background load in slabs of the last axis (large 3D runs)."""
    lo, hi = w.plasma_lo, w.plasma_hi
    for z in range(lo, hi, chunk_cells_last):
        yield background(w, (z, min(hi, z + chunk_cells_last)))


def bunch(w: Workload) -> Particles:
    """Gaussian electron bunch at the box centre (on axis, mid last axis):
    ppc per axis regular in every cell within 3 sigma, weight
    n_bg * peak * G(r, z) / ppc, u_z given, other momenta zero."""
    b = w.bunch
    dim = w.dim
    ctr = [0.5 * w.n[a] * w.d[a] for a in range(dim)]
    sig = [b["sigma_r"]] * (dim - 1) + [b["sigma_z"]]
    ranges = []
    for a in range(dim):
        lo = int(math.floor((ctr[a] - 3 * sig[a]) / w.d[a]))
        hi = int(math.ceil((ctr[a] + 3 * sig[a]) / w.d[a]))
        ranges.append(np.arange(max(lo, 0), min(hi, w.n[a]), dtype=np.int32))
    ppc = b["ppc"]
    cells = np.meshgrid(*ranges, indexing="ij")
    subs = np.meshgrid(*[(np.arange(ppc[a]) + 0.5) / ppc[a] for a in range(dim)], indexing="ij")
    nc, ns = cells[0].size, subs[0].size
    cell = np.stack([np.repeat(cells[a].reshape(-1), ns) for a in range(dim)]).astype(np.int32)
    off = np.stack([np.tile(subs[a].reshape(-1), nc) for a in range(dim)]).astype(np.float32)
    pos = (cell + off.astype(np.float64)) * np.asarray(w.d[:dim])[:, None]
    arg = sum(((pos[a] - ctr[a]) / sig[a]) ** 2 for a in range(dim))
    inside = arg <= 9.0
    cell, off, arg = cell[:, inside], off[:, inside], arg[inside]
    wt = (w.density * b["peak"] * np.exp(-0.5 * arg) / np.prod(ppc)).astype(np.float32)
    u = np.zeros((3, cell.shape[1]), dtype=np.float32)
    u[dim - 1] = b["uz"]
    return Particles(cell, off, u, wt)


def concat(parts) -> Particles:
    return Particles(np.concatenate([p.cell for p in parts], axis=1),
                     np.concatenate([p.off for p in parts], axis=1),
                     np.concatenate([p.u for p in parts], axis=1),
                     np.concatenate([p.w for p in parts]))
