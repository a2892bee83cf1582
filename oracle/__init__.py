"""FP64 CPU oracle for the EM-PIC timestep (Fonseca et al., Sec. 2 and Sec. 5.2).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path and never imports ``paper_1310_0930_gb300`` (inputs are
handed to it as plain numpy arrays).

Pinned by tests (``tests/test_oracle_*.py``) against closed forms and brute
force, never against itself:

* ``bspline``            -- convolution identity, partition of unity, first and
                            second moments (Sec. 5.2 step i; Table 3 orders).
* ``gather``             -- exact for constant and linear fields at every Yee
                            location; second-moment law for quadratics.
* ``boris``              -- gyration angle / radius, |u| conservation, E x B
                            drift, exact uniform-E momentum (Sec. 2, Sec. 5.2 iii).
* ``deposit_current``    -- discrete continuity against ``deposit_rho`` to
                            round-off, total-current identity, linear-order
                            Villasenor-Buneman closed form (Sec. 5.2).
* ``yee`` (via ``step``) -- discrete plane-wave solution of the Yee scheme,
                            div B = 0 (Sec. 2).
* ``step``               -- cold-plasma k=0 oscillation obeys the leapfrog
                            relation; Gauss residual at round-off.
* laser antenna          -- vacuum injection reaches a0 with one-way leakage
                            below a bound.
* moving window          -- equals a fixed larger box in the window frame
                            until boundary effects arrive.
* laser-plasma coupling  -- the linear wake of a weak Gaussian pulse: peak
                            field, wavelength at the group velocity, a0^2
                            scaling against the 1D closed form.
* energies               -- kinetic energy of particles accelerated by a
                            uniform field against its closed form, the work
                            q E . dx of a step against the kinetic energy it
                            adds, W_E + W_kin of a cold oscillation within the
                            leapfrog bound (``tests/test_oracle_energy.py``).
* density profile        -- the weights of the plasma a moving window injects
                            follow the piecewise-linear knot profile at each
                            particle's lab position.
* deposit_current_split  -- virtual trajectories (Sec. 5.2 iv): continuity,
                            total current, no split inside one node cell,
                            Villasenor-Buneman pieces across faces.
* energy history         -- one recorded 32x32 warm-plasma history
                            (``tests/golden/``, written from this oracle alone)
                            reproduced to round-off.
LWFA physics beyond these (nonlinear wakes, self-injection): parity unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "libpic_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrSim(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("d", ctypes.c_double * 3),
        ("dt", ctypes.c_double), ("order", ctypes.c_int32), ("open_last", ctypes.c_int32),
        ("q", ctypes.c_double), ("m", ctypes.c_double),
        ("laser_on", ctypes.c_int32), ("laser_plane", ctypes.c_int32), ("laser_pol", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("a0", ctypes.c_double), ("omega0", ctypes.c_double), ("waist", ctypes.c_double),
        ("fwhm", ctypes.c_double), ("t_peak", ctypes.c_double),
        ("window_on", ctypes.c_int32), ("ppc", ctypes.c_int32 * 3),
        ("window_v", ctypes.c_double), ("window_t0", ctypes.c_double),
        ("density", ctypes.c_double),
        ("n_knots", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("knots", ctypes.POINTER(ctypes.c_double)), ("z0", ctypes.c_double), ("z1", ctypes.c_double),
        ("time", ctypes.c_double), ("step", ctypes.c_int64), ("shifts", ctypes.c_int64),
        ("nthreads", ctypes.c_int32), ("pad2", ctypes.c_int32),
        ("split", ctypes.c_int32), ("pad3", ctypes.c_int32),
    ]


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_bspline.restype = ctypes.c_double
            L.or_bspline.argtypes = [ctypes.c_int, ctypes.c_double]
            L.or_gather.argtypes = [ctypes.POINTER(OrSim), _dp, _dp, _dp, _dp]
            L.or_boris.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp]
            L.or_deposit_rho.argtypes = [ctypes.POINTER(OrSim), ctypes.c_double, _dp, _dp]
            L.or_deposit_current.argtypes = [ctypes.POINTER(OrSim), ctypes.c_double, _dp, _dp,
                                             ctypes.c_double, _dp]
            L.or_deposit_current_split.argtypes = [ctypes.POINTER(OrSim), ctypes.c_double, _dp, _dp,
                                                   ctypes.c_double, _dp]
            L.or_yee_b.argtypes = [ctypes.POINTER(OrSim), _dp, _dp, ctypes.c_double]
            L.or_yee_e.argtypes = [ctypes.POINTER(OrSim), _dp, _dp, _dp]
            L.or_step.restype = ctypes.c_int
            L.or_step.argtypes = [ctypes.POINTER(OrSim), _dp, _dp, _dp, _dp, _dp, _dp,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, ctypes.c_int]
            L.or_div_e.argtypes = [ctypes.POINTER(OrSim), _dp, _dp]
            L.or_energies.argtypes = [ctypes.POINTER(OrSim), _dp, _dp, _dp, _dp, ctypes.c_int64,
                                      ctypes.c_int64, _dp]
            L.or_charge.argtypes = [ctypes.POINTER(OrSim), _dp, _dp, ctypes.c_int64, ctypes.c_int64, _dp]
            L.or_abi_size.restype = ctypes.c_int
            assert L.or_abi_size() == ctypes.sizeof(OrSim), "oracle struct layout mismatch"
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def bspline(p: int, t: float) -> float:
    """B-spline shape of order p at distance t (cells) from a node."""
    return lib().or_bspline(int(p), float(t))


def boris(qm: float, dt: float, eb, u) -> np.ndarray:
    """One Boris momentum update; eb = (E0,E1,E2,B0,B1,B2)."""
    eb = np.ascontiguousarray(eb, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    lib().or_boris(float(qm), float(dt), _p(eb), _p(u))
    return u


class Sim:
    """FP64 oracle state: grid, fields and one particle species.

    Positions ``x`` are global coordinates in cell units ([3][cap], unused
    axes zero); ``u`` = gamma*beta ([3][cap]); ``w`` = density weight per
    particle (n/ppc), so that rho(node) = sum q w S.
    """

    def __init__(self, dim, n, d, dt, order, q=-1.0, m=1.0, open_last=False, nthreads=None,
                 laser=None, window=None, split=False):
        self.s = OrSim()
        s = self.s
        s.dim = dim
        nn = list(n) + [1] * (3 - len(n))
        dd = list(d) + [1.0] * (3 - len(d))
        for a in range(3):
            s.n[a] = int(nn[a])
            s.d[a] = float(dd[a])
        s.dt = float(dt)
        s.order = int(order)
        s.open_last = int(bool(open_last))
        s.q, s.m = float(q), float(m)
        s.nthreads = int(nthreads or os.cpu_count() or 1)
        s.split = int(bool(split))
        self._knots = None
        if laser is not None:
            s.laser_on = 1
            s.laser_plane = int(laser.get("plane", 2))
            s.laser_pol = int(laser.get("pol", 0))
            s.a0 = laser["a0"]
            s.omega0 = laser.get("omega0", 1.0)
            s.waist = laser["waist"]
            s.fwhm = laser["fwhm"]
            s.t_peak = laser.get("t_peak", 2.0 * laser["fwhm"])
        if window is not None:
            s.window_on = 1
            s.window_v = window.get("v", 1.0)
            s.window_t0 = window.get("t0", 0.0)
            ppc = list(window["ppc"]) + [1] * (3 - len(window["ppc"]))
            for a in range(3):
                s.ppc[a] = int(ppc[a])
            s.density = float(window.get("density", 0.0))
            knots = window.get("knots")
            if knots is not None:
                self._knots = np.ascontiguousarray(knots, dtype=np.float64)
                s.n_knots = len(self._knots)
                s.knots = self._knots.ctypes.data_as(_dp)
                s.z0, s.z1 = float(window["z0"]), float(window["z1"])
        self.ncell = s.n[0] * s.n[1] * s.n[2]
        self.E = np.zeros(3 * self.ncell)
        self.B = np.zeros(3 * self.ncell)
        self.J = np.zeros(3 * self.ncell)
        self.cap = 0
        self.np = 0
        self.x = np.zeros((3, 0))
        self.u = np.zeros((3, 0))
        self.w = np.zeros(0)

    # -- state -----------------------------------------------------------
    @property
    def shape(self):
        s = self.s
        return (s.n[2], s.n[1], s.n[0]) if s.dim == 3 else (s.n[1], s.n[0])

    def field(self, name: str) -> np.ndarray:
        """View of one field component, shaped (nz, ny, nx) or (ny, nx)."""
        comp = "xyz".index(name[1])
        arr = {"E": self.E, "B": self.B, "J": self.J}[name[0]]
        return arr[comp * self.ncell:(comp + 1) * self.ncell].reshape(self.shape)

    def load(self, x, u, w, capacity=None):
        x = np.asarray(x, dtype=np.float64)
        n = x.shape[1]
        cap = int(capacity or n)
        self.cap = cap
        self.np = n
        self.x = np.zeros((3, cap))
        self.u = np.zeros((3, cap))
        self.w = np.zeros(cap)
        self.x[: x.shape[0], :n] = x
        self.u[:, :n] = np.asarray(u, dtype=np.float64)
        self.w[:n] = np.asarray(w, dtype=np.float64)

    def particles(self):
        n = self.np
        return self.x[:, :n], self.u[:, :n], self.w[:n]

    # -- stepping and diagnostics ----------------------------------------
    def step(self, nsteps: int = 1):
        npv = ctypes.c_int64(self.np)
        rc = lib().or_step(ctypes.byref(self.s), _p(self.E), _p(self.B), _p(self.J),
                           self.x.ctypes.data_as(_dp), self.u.ctypes.data_as(_dp),
                           self.w.ctypes.data_as(_dp), ctypes.byref(npv), self.cap, int(nsteps))
        if rc != 0:
            raise RuntimeError("oracle step failed")
        self.np = int(npv.value)

    def gather(self, x3) -> np.ndarray:
        x = np.zeros(3)
        x[: len(x3)] = x3
        out = np.zeros(6)
        lib().or_gather(ctypes.byref(self.s), _p(self.E), _p(self.B), _p(x), _p(out))
        return out

    def deposit_current(self, qw, x_old, x_new, vz, J=None) -> np.ndarray:
        J = np.zeros(3 * self.ncell) if J is None else J
        xo = np.zeros(3)
        xn = np.zeros(3)
        xo[: len(x_old)] = x_old
        xn[: len(x_new)] = x_new
        lib().or_deposit_current(ctypes.byref(self.s), float(qw), _p(xo), _p(xn), float(vz), _p(J))
        return J

    def deposit_current_split(self, qw, x_old, x_new, vz, J=None) -> np.ndarray:
        """The same move deposited as virtual trajectories (split at the
        boundaries between nearest grid points)."""
        J = np.zeros(3 * self.ncell) if J is None else J
        xo = np.zeros(3)
        xn = np.zeros(3)
        xo[: len(x_old)] = x_old
        xn[: len(x_new)] = x_new
        lib().or_deposit_current_split(ctypes.byref(self.s), float(qw), _p(xo), _p(xn), float(vz), _p(J))
        return J

    def deposit_rho(self, qw, x3, rho=None) -> np.ndarray:
        rho = np.zeros(self.ncell) if rho is None else rho
        x = np.zeros(3)
        x[: len(x3)] = x3
        lib().or_deposit_rho(ctypes.byref(self.s), float(qw), _p(x), _p(rho))
        return rho

    def yee_b(self, h):
        lib().or_yee_b(ctypes.byref(self.s), _p(self.E), _p(self.B), float(h))

    def yee_e(self):
        lib().or_yee_e(ctypes.byref(self.s), _p(self.E), _p(self.B), _p(self.J))

    def div_e(self) -> np.ndarray:
        out = np.zeros(self.ncell)
        lib().or_div_e(ctypes.byref(self.s), _p(self.E), _p(out))
        return out

    def charge(self) -> np.ndarray:
        rho = np.zeros(self.ncell)
        lib().or_charge(ctypes.byref(self.s), self.x.ctypes.data_as(_dp), _p(self.w), self.np, self.cap,
                        _p(rho))
        return rho

    def energies(self):
        out = np.zeros(3)
        lib().or_energies(ctypes.byref(self.s), _p(self.E), _p(self.B), self.u.ctypes.data_as(_dp),
                          _p(self.w), self.np, self.cap, _p(out))
        return {"W_E": out[0], "W_B": out[1], "W_kin": out[2]}

    @property
    def time(self):
        return self.s.time

    @property
    def shifts(self):
        return int(self.s.shifts)
