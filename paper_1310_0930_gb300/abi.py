"""ctypes binding of the C ABI in ``include/pic.h`` (same names, argument
marshalling only).  Every step of the timestep runs in the CUDA library; if
the library is missing this module raises instead of falling back to
anything else."""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

c_int32, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                   ctypes.c_void_p, ctypes.c_size_t)

PIC_ABI_VERSION = 1
PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_EOVERFLOW, PIC_ETIMEOUT, PIC_ESTATE = 0, -1, -2, -3, -4, -5, -6
PIC_BC_PERIODIC, PIC_BC_OPEN = 0, 1
FIELDS = {"Ex": 0, "Ey": 1, "Ez": 2, "Bx": 3, "By": 4, "Bz": 5, "Jx": 6, "Jy": 7, "Jz": 8, "rho": 9}


class pic_grid(ctypes.Structure):
    _fields_ = [("dim", c_int32), ("n", c_int32 * 3), ("d", c_double * 3), ("dt", c_double),
                ("bc_last", c_int32), ("reserved", c_int32)]


class pic_species(ctypes.Structure):
    _fields_ = [("q", c_double), ("m", c_double), ("ppc", c_int32 * 3), ("per_particle_weight", c_int32),
                ("w_const", c_double), ("density", c_double), ("profile_knots", ctypes.POINTER(c_double)),
                ("n_knots", c_int32), ("reserved", c_int32), ("profile_z0", c_double), ("profile_z1", c_double)]


class pic_laser(ctypes.Structure):
    _fields_ = [("enabled", c_int32), ("pol_axis", c_int32), ("plane", c_int32), ("reserved", c_int32),
                ("a0", c_double), ("omega0", c_double), ("waist", c_double), ("fwhm", c_double),
                ("t_peak", c_double)]


class pic_window(ctypes.Structure):
    _fields_ = [("enabled", c_int32), ("reserved", c_int32), ("velocity", c_double), ("t_start", c_double)]


class pic_tuning(ctypes.Structure):
    _fields_ = [("tile", c_int32 * 3), ("sort_interval", c_int32), ("drift", c_int32), ("block", c_int32),
                ("use_graph", c_int32), ("persistent", c_int32), ("sort_sub", c_int32),
                ("tma", c_int32), ("adjoint_keep", c_int32), ("sort_policy", c_int32),
                ("stream_zero_tiles", c_int32), ("deposit", c_int32), ("j_layout", c_int32),
                ("sort_rows", c_int32), ("quiet_tiles", c_int32)]


pic_alloc_fn = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
pic_free_fn = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class pic_config(ctypes.Structure):
    _fields_ = [("abi_version", c_int32), ("shape_order", c_int32), ("grid", pic_grid), ("n_species", c_int32),
                ("track_ids", c_int32), ("species", ctypes.POINTER(pic_species)), ("laser", pic_laser),
                ("window", pic_window), ("seed", ctypes.c_uint64), ("capacity", c_int64),
                ("tuning", pic_tuning), ("alloc", pic_alloc_fn), ("free", pic_free_fn),
                ("alloc_ctx", c_void_p), ("stream", c_void_p)]


class pic_objective(ctypes.Structure):
    _fields_ = [("z_lo", c_double), ("z_hi", c_double), ("width", c_double)]


class pic_diag(ctypes.Structure):
    _fields_ = [("step", c_int64), ("time", c_double), ("shifts", c_int64), ("W_E", c_double), ("W_B", c_double),
                ("W_kin", c_double), ("gauss_resid", c_double), ("n_particles", c_int64),
                ("imbalance", c_double), ("slow_path", c_int64), ("status", c_int32), ("sorts", c_int32),
                ("streamed", c_int64), ("live_tiles", c_int64)]


# name -> (restype, argtypes); the order and types follow include/pic.h
_P = ctypes.POINTER
_handle = c_void_p
SIGNATURES = {
    "pic_create": (c_int32, [_P(pic_config), _P(_handle)]),
    "pic_create_batch": (c_int32, [_P(pic_config), c_int32, _P(_handle)]),
    "pic_select_run": (c_int32, [_handle, c_int32]),
    "pic_num_runs": (c_int32, [_handle]),
    "pic_load_particles": (c_int32, [_handle, c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "pic_step": (c_int32, [_handle, c_int32]),
    "pic_sync": (c_int32, [_handle]),
    "pic_read_fields": (c_int32, [_handle, c_int32, c_void_p, c_size_t, c_int32]),
    "pic_write_fields": (c_int32, [_handle, c_int32, c_void_p, c_size_t, c_int32]),
    "pic_read_particles": (c_int32, [_handle, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                     _P(c_int64)]),
    "pic_diagnostics": (c_int32, [_handle, _P(pic_diag)]),
    "pic_destroy": (None, [_handle]),
    "pic_strerror": (ctypes.c_char_p, [c_int32]),
    "pic_profile_begin": (c_int32, [_handle, c_int32]),
    "pic_profile_end": (c_int32, [_handle, _P(c_double), c_int32, _P(c_int64)]),
    "pic_adjoint_begin": (c_int32, [_handle, c_int32, c_int32]),
    "pic_adjoint_kept": (c_int32, [_handle]),
    "pic_objective_value": (c_int32, [_handle, _P(pic_objective), _P(c_double)]),
    "pic_adjoint_backward": (c_int32, [_handle, _P(pic_objective), _P(c_double), _P(c_double), c_void_p, c_int32,
                                       c_void_p]),
    "pic_adjoint_fields": (c_int32, [_handle, c_void_p, c_void_p, c_double]),
    "pic_adjoint_particles": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64]),
    "pic_charge_density_static": (c_int32, [_P(pic_grid), c_int32, c_double, c_double, c_int64, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p]),
}
PIC_STATIC_MAX_CELLS = 1 << 21

PHASES = ["sort", "zero_j", "push", "yee_b1", "yee_e", "yee_b2", "window", "push_zero"]

_lock = threading.Lock()
_lib = None


class PicError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = lib().pic_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s failed: %s (%d)" % (where, msg, code))


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load the CUDA library (building it if it is absent and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or not _build.up_to_date():
                if not build_if_missing:
                    raise ImportError("libpic_gb300.so is not built")
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code, where=""):
    if code != PIC_OK:
        raise PicError(code, where)
    return code


# -- thin wrappers with the C names ------------------------------------------
def pic_create(cfg: pic_config) -> int:
    h = _handle()
    check(lib().pic_create(ctypes.byref(cfg), ctypes.byref(h)), "pic_create")
    return h.value


def pic_create_batch(cfgs) -> int:
    arr = (pic_config * len(cfgs))(*cfgs)
    h = _handle()
    check(lib().pic_create_batch(arr, len(cfgs), ctypes.byref(h)), "pic_create_batch")
    return h.value


def pic_select_run(h, run):
    return check(lib().pic_select_run(h, run), "pic_select_run")


def pic_num_runs(h):
    return lib().pic_num_runs(h)


def pic_load_particles(h, species, n, cell_ptr, off_ptr, u_ptr, w_ptr):
    return check(lib().pic_load_particles(h, species, n, cell_ptr, off_ptr, u_ptr, w_ptr), "pic_load_particles")


def pic_step(h, nsteps):
    return check(lib().pic_step(h, nsteps), "pic_step")


def pic_sync(h):
    return check(lib().pic_sync(h), "pic_sync")


def pic_read_fields(h, which, dst_ptr, n_elems, on_device):
    return check(lib().pic_read_fields(h, which, dst_ptr, n_elems, on_device), "pic_read_fields")


def pic_write_fields(h, which, src_ptr, n_elems, on_device):
    return check(lib().pic_write_fields(h, which, src_ptr, n_elems, on_device), "pic_write_fields")


def pic_read_particles(h, species, cell, off, u, w, idp, cap):
    n = c_int64()
    check(lib().pic_read_particles(h, species, cell, off, u, w, idp, cap, ctypes.byref(n)), "pic_read_particles")
    return n.value


def pic_diagnostics(h) -> pic_diag:
    d = pic_diag()
    code = lib().pic_diagnostics(h, ctypes.byref(d))
    if code not in (PIC_OK,):
        raise PicError(code, "pic_diagnostics")
    return d


def pic_destroy(h):
    lib().pic_destroy(h)


def pic_profile_begin(h, max_steps):
    return check(lib().pic_profile_begin(h, max_steps), "pic_profile_begin")


def pic_profile_end(h):
    """Summed milliseconds per phase (dict) and the kernels launched meanwhile."""
    ms = (c_double * len(PHASES))()
    steps = c_int64()
    check(lib().pic_profile_end(h, ms, len(PHASES), ctypes.byref(steps)), "pic_profile_end")
    return dict(zip(PHASES, list(ms))), steps.value


def pic_strerror(code) -> str:
    return lib().pic_strerror(code).decode()
