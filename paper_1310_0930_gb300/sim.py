"""Convenience wrapper around the C ABI: builds a ``pic_config`` from a
workload description, hands the PyTorch caching allocator and a PyTorch
stream to the library, and moves numpy arrays in and out.  It marshals
arguments only; the timestep itself runs in ``libpic_gb300.so``."""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import abi
from .inputs import Particles, Workload


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.flags.c_contiguous
    return ctypes.c_void_p(a.ctypes.data)


def make_config(w: Workload, *, tuning: Optional[dict] = None, track_ids=False, capacity=0,
                per_particle_weight=None, stream=0, alloc=None, free=None):
    """pic_config for workload `w`; returns (cfg, keepalive)."""
    cfg = abi.pic_config()
    cfg.abi_version = abi.PIC_ABI_VERSION
    cfg.shape_order = w.order
    n = list(w.n) + [1] * (3 - len(w.n))
    d = list(w.d) + [1.0] * (3 - len(w.d))
    cfg.grid.dim = w.dim
    for a in range(3):
        cfg.grid.n[a] = int(n[a])
        cfg.grid.d[a] = float(d[a])
    cfg.grid.dt = float(w.dt)
    cfg.grid.bc_last = abi.PIC_BC_OPEN if w.open_last else abi.PIC_BC_PERIODIC
    sp = abi.pic_species()
    sp.q, sp.m = -1.0, float(getattr(w, "mass", 1.0))
    ppc = list(w.ppc) + [1] * (3 - len(w.ppc))
    for a in range(3):
        sp.ppc[a] = int(ppc[a])
    if per_particle_weight is None:
        per_particle_weight = w.knots is not None or w.bunch is not None
    sp.per_particle_weight = int(bool(per_particle_weight))
    sp.w_const = float(w.density / w.ppc_total)
    sp.density = float(w.density)
    keep = [sp]
    if w.knots is not None:
        k = np.ascontiguousarray(w.knots, dtype=np.float64)
        keep.append(k)
        sp.profile_knots = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        sp.n_knots = len(k)
        sp.profile_z0, sp.profile_z1 = float(w.knot_z[0]), float(w.knot_z[1])
    cfg.n_species = 1
    cfg.track_ids = int(bool(track_ids))
    cfg.species = ctypes.pointer(sp)
    if w.laser is not None:
        L = cfg.laser
        L.enabled = 1
        L.pol_axis = w.laser.pol
        L.plane = w.laser.plane
        L.a0, L.omega0, L.waist, L.fwhm = w.laser.a0, w.laser.omega0, w.laser.waist, w.laser.fwhm
        L.t_peak = w.laser.peak_time()
    if w.window is not None:
        cfg.window.enabled = 1
        cfg.window.velocity = w.window.v
        cfg.window.t_start = w.window.t0
    cfg.seed = int(w.seed)
    cfg.capacity = int(capacity)
    t = dict(tuning or {})
    tile = list(t.get("tile", (0, 0, 0))) + [0] * 3
    for a in range(3):
        cfg.tuning.tile[a] = int(tile[a])
    cfg.tuning.sort_interval = int(t.get("sort_interval", 0))
    cfg.tuning.drift = int(t.get("drift", -1))
    cfg.tuning.block = int(t.get("block", 0))
    cfg.tuning.use_graph = int(t.get("use_graph", 1))
    cfg.tuning.persistent = int(t.get("persistent", 0))
    cfg.tuning.sort_sub = int(t.get("sort_sub", 0))
    cfg.tuning.tma = int(t.get("tma", 0))
    cfg.tuning.adjoint_keep = int(t.get("adjoint_keep", 0))
    cfg.tuning.sort_policy = int(t.get("sort_policy", 0))
    cfg.tuning.stream_zero_tiles = int(t.get("stream_zero_tiles", 0))
    cfg.tuning.deposit = int(t.get("deposit", 0))
    cfg.tuning.j_layout = int(t.get("j_layout", 0))
    cfg.tuning.sort_rows = int(t.get("sort_rows", 0))
    cfg.tuning.quiet_tiles = int(t.get("quiet_tiles", 0))
    if alloc is not None:
        cfg.alloc = alloc
        cfg.free = free
    cfg.stream = stream
    return cfg, keep


class TorchMemory:
    """Allocator hooks and stream from PyTorch (device memory and ordering only)."""

    def __init__(self, device=0, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        dev_index = self.device.index

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev_index, self.stream)
            except Exception:  # out of memory: the library reports PIC_ENOMEM
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = abi.pic_alloc_fn(_alloc)
        self.free = abi.pic_free_fn(_free)

    @property
    def stream_handle(self):
        return self.stream.cuda_stream


class Simulation:
    """One run (or a batch of runs) of the GB300 EM-PIC timestep."""

    def __init__(self, workloads, *, tuning=None, track_ids=False, capacity=0, per_particle_weight=None,
                 memory: Optional[TorchMemory] = None):
        self.batch = isinstance(workloads, (list, tuple))
        self.workloads = list(workloads) if self.batch else [workloads]
        self.w = self.workloads[0]
        self.mem = memory or TorchMemory()
        cfgs, self._keep = [], []
        caps = capacity if isinstance(capacity, (list, tuple)) else [capacity] * len(self.workloads)
        for wl, cap in zip(self.workloads, caps):
            cfg, keep = make_config(wl, tuning=tuning, track_ids=track_ids, capacity=cap,
                                    per_particle_weight=per_particle_weight, stream=self.mem.stream_handle,
                                    alloc=self.mem.alloc, free=self.mem.free)
            cfgs.append(cfg)
            self._keep.append(keep)
        self.h = abi.pic_create_batch(cfgs) if self.batch else abi.pic_create(cfgs[0])
        self.cur = 0

    # -- run selection ------------------------------------------------------
    def select(self, run: int):
        abi.pic_select_run(self.h, run)
        self.cur = run
        self.w = self.workloads[run]

    # -- particles ------------------------------------------------------------
    def load(self, p: Particles):
        cell = np.ascontiguousarray(p.cell, dtype=np.int32)
        off = np.ascontiguousarray(p.off, dtype=np.float32)
        u = np.ascontiguousarray(p.u, dtype=np.float32)
        wt = np.ascontiguousarray(p.w, dtype=np.float32)
        abi.pic_load_particles(self.h, 0, p.n, _ptr(cell), _ptr(off), _ptr(u), _ptr(wt))

    def particles(self, cap=None) -> dict:
        dim = self.w.dim
        if cap is None:
            cap = int(self.diagnostics()["n_particles"]) + 16
        cell = np.zeros((dim, cap), np.int32)
        off = np.zeros((dim, cap), np.float32)
        u = np.zeros((3, cap), np.float32)
        w = np.zeros(cap, np.float32)
        ids = np.zeros(cap, np.int32)
        n = abi.pic_read_particles(self.h, 0, _ptr(cell), _ptr(off), _ptr(u), _ptr(w), _ptr(ids), cap)
        return dict(cell=cell[:, :n], off=off[:, :n], u=u[:, :n], w=w[:n], id=ids[:n], n=n)

    # -- stepping ---------------------------------------------------------------
    def step(self, n: int = 1):
        abi.pic_step(self.h, int(n))

    def sync(self):
        abi.pic_sync(self.h)

    # -- adjoint ------------------------------------------------------------
    def adjoint_begin(self, total_steps: int, checkpoint_every: int) -> int:
        """Arm the reverse mode; returns the number of checkpoint segments the
        forward run records instead of the reverse sweep recomputing them."""
        abi.check(abi.lib().pic_adjoint_begin(self.h, int(total_steps), int(checkpoint_every)), "pic_adjoint_begin")
        kept = abi.lib().pic_adjoint_kept(self.h)
        abi.check(min(kept, 0), "pic_adjoint_kept")
        return kept

    def objective(self, z_lo: float, z_hi: float, width: float) -> float:
        o = abi.pic_objective(z_lo, z_hi, width)
        L = ctypes.c_double()
        abi.check(abi.lib().pic_objective_value(self.h, ctypes.byref(o), ctypes.byref(L)), "pic_objective_value")
        return L.value

    def adjoint_backward(self, z_lo: float, z_hi: float, width: float, n_knots: int = 0, n_ids: int = 0) -> dict:
        o = abi.pic_objective(z_lo, z_hi, width)
        L, da0 = ctypes.c_double(), ctypes.c_double()
        dk = np.zeros(max(n_knots, 1), np.float64)
        dw = np.zeros(n_ids, np.float64) if n_ids else None
        abi.check(abi.lib().pic_adjoint_backward(self.h, ctypes.byref(o), ctypes.byref(L), ctypes.byref(da0),
                                                 _ptr(dk) if n_knots else None, int(n_knots), _ptr(dw)),
                  "pic_adjoint_backward")
        return {"L": L.value, "dL_da0": da0.value, "dL_dknots": dk[:n_knots], "dL_dw": dw}

    def adjoint_fields(self, lam: np.ndarray, t: float):
        """Transpose of one step's field update applied to lam[6][...]."""
        lam = np.ascontiguousarray(lam, dtype=np.float32).copy()
        lj = np.zeros((3,) + lam.shape[1:], np.float32)
        abi.check(abi.lib().pic_adjoint_fields(self.h, _ptr(lam), _ptr(lj), float(t)), "pic_adjoint_fields")
        return lam, lj

    def adjoint_particles(self, lam_x: np.ndarray, lam_u: np.ndarray, lam_j: np.ndarray):
        """Transpose of the next step's particle part at the current state,
        applied to the adjoints of the new positions (cells) and momenta (by
        id) and of the deposited current; returns the adjoints of the old
        positions, momenta, weights and of E, B (six components)."""
        n = lam_u.shape[1]
        lx = np.ascontiguousarray(lam_x, dtype=np.float32).copy()
        lu = np.ascontiguousarray(lam_u, dtype=np.float32).copy()
        lj = np.ascontiguousarray(lam_j, dtype=np.float32)
        lw = np.zeros(n, np.float64)
        lf = np.zeros((6,) + tuple(lj.shape[1:]), np.float32)
        abi.check(abi.lib().pic_adjoint_particles(self.h, _ptr(lx), _ptr(lu), _ptr(lj), _ptr(lw), _ptr(lf), int(n)),
                  "pic_adjoint_particles")
        return lx, lu, lw, lf

    def profile_begin(self, max_steps: int):
        abi.pic_profile_begin(self.h, int(max_steps))

    def profile_end(self):
        return abi.pic_profile_end(self.h)

    # -- fields -------------------------------------------------------------------
    @property
    def shape(self):
        n = self.w.n
        return (n[2], n[1], n[0]) if self.w.dim == 3 else (n[1], n[0])

    def field(self, name: str) -> np.ndarray:
        out = np.zeros(self.shape, np.float32)
        abi.pic_read_fields(self.h, abi.FIELDS[name], _ptr(out), out.size, 0)
        return out

    def set_field(self, name: str, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=np.float32).reshape(self.shape)
        abi.pic_write_fields(self.h, abi.FIELDS[name], _ptr(a), a.size, 0)

    def diagnostics(self) -> dict:
        d = abi.pic_diagnostics(self.h)
        return {k: getattr(d, k) for k, _ in abi.pic_diag._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "h", None):
            abi.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
