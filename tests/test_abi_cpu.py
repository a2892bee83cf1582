"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function declared in include/pic.h, the ctypes mirrors
match the C struct layout (checked by compiling a probe against the header
with the host C compiler), and configuration validation rejects bad input
before any device call."""
import ctypes
import math
import os
import re
import shutil
import subprocess

import pytest

from paper_1310_0930_gb300 import abi, inputs
from paper_1310_0930_gb300.sim import make_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists(abi.lib_path()),
                                reason="needs nvcc or a prebuilt library")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", text)) - {"pic_alloc_fn", "pic_free_fn"})


def test_library_exports_every_declared_function():
    L = abi.lib()
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
        assert n in abi.SIGNATURES, n


def test_ctypes_layout_matches_c_header(tmp_path):
    structs = {"pic_grid": abi.pic_grid, "pic_species": abi.pic_species, "pic_laser": abi.pic_laser,
               "pic_window": abi.pic_window, "pic_tuning": abi.pic_tuning, "pic_config": abi.pic_config,
               "pic_diag": abi.pic_diag}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[name + "." + fname]) == getattr(cls, fname).offset, (name, fname)


def _create(cfg):
    h = ctypes.c_void_p()
    return abi.lib().pic_create(ctypes.byref(cfg), ctypes.byref(h)), h


def test_validation_rejects_bad_configs_before_touching_the_device():
    w = inputs.thermal_2d(n=(32, 32))
    # Courant: dt * sqrt(sum 1/d^2) >= 1
    cfg, keep = make_config(w)
    cfg.grid.dt = 1.0 / math.sqrt(2 / 0.2 ** 2) * 1.0001
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # unsupported shape order (quartic: the default tiles only)
    cfg, keep = make_config(w)
    cfg.shape_order = 5
    assert _create(cfg)[0] == abi.PIC_EINVAL
    cfg, keep = make_config(w, tuning={"tile": (8, 8)})
    cfg.shape_order = 4
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # more than one species
    cfg, keep = make_config(w)
    cfg.n_species = 2
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # ABI version mismatch
    cfg, keep = make_config(w)
    cfg.abi_version = 99
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # packed cell index would need more than 31 bits
    w3 = inputs.thermal_3d(n=(4096, 4096, 1024), d=(1, 1, 1), dt=0.5)
    cfg, keep = make_config(w3)
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # non power-of-two tile
    cfg, keep = make_config(w, tuning={"tile": (12, 16)})
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # unknown sort policy, negative sort interval
    cfg, keep = make_config(w, tuning={"sort_policy": 2})
    assert _create(cfg)[0] == abi.PIC_EINVAL
    cfg, keep = make_config(w, tuning={"sort_interval": -1})
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # window on a periodic axis
    cfg, keep = make_config(w)
    cfg.window.enabled = 1
    cfg.window.velocity = 1.0
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # laser plane outside the grid
    wl = inputs.lwfa_2d(nx=32, nz=64)
    cfg, keep = make_config(wl)
    cfg.laser.plane = 0
    assert _create(cfg)[0] == abi.PIC_EINVAL
    # the 3D LWFA cells at dt = 0.28 violate Courant (limit 0.2762); 0.27 does not
    w3 = inputs.lwfa_3d(n=(16, 16, 64))
    cfg, keep = make_config(w3)
    cfg.grid.dt = 0.28
    assert _create(cfg)[0] == abi.PIC_EINVAL


def test_null_handles_and_strerror():
    L = abi.lib()
    assert L.pic_step(None, 1) == abi.PIC_EINVAL
    assert L.pic_sync(None) == abi.PIC_EINVAL
    assert L.pic_select_run(None, 0) == abi.PIC_EINVAL
    assert L.pic_num_runs(None) == 0
    L.pic_destroy(None)
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert abi.pic_strerror(code)
    assert abi.pic_strerror(-77) == "unknown status"


def test_static_charge_entry_point_rejects_oversized_grid_without_device_work():
    L = abi.lib()
    g = abi.pic_grid()
    g.dim = 3
    g.n[0], g.n[1], g.n[2] = 256, 128, 65  # 2,129,920 cells > PIC_STATIC_MAX_CELLS
    assert 256 * 128 * 65 > abi.PIC_STATIC_MAX_CELLS
    dummy = ctypes.c_void_p(16)
    rc = L.pic_charge_density_static(ctypes.byref(g), 2, -1.0, 1.0, 10, dummy, dummy, None, dummy, None)
    assert rc == abi.PIC_EINVAL
    g.n[2] = 64  # exactly the limit passes validation (not run here: no device)
    assert 256 * 128 * 64 == abi.PIC_STATIC_MAX_CELLS
    g.dim = 4
    assert L.pic_charge_density_static(ctypes.byref(g), 2, -1.0, 1.0, 10, dummy, dummy, None, dummy, None) == \
        abi.PIC_EINVAL
    # axes whose product wraps a 64-bit count to 0 (2^21 * 2^21 * 2^22 = 2^64)
    # must be refused too, not pass the size check after the wrap
    g.dim = 3
    g.n[0], g.n[1], g.n[2] = 1 << 21, 1 << 21, 1 << 22
    assert L.pic_charge_density_static(ctypes.byref(g), 2, -1.0, 1.0, 10, dummy, dummy, None, dummy, None) == \
        abi.PIC_EINVAL
    g.n[0], g.n[1], g.n[2] = 1 << 30, 1 << 30, 1 << 30
    assert L.pic_charge_density_static(ctypes.byref(g), 2, -1.0, 1.0, 10, dummy, dummy, None, dummy, None) == \
        abi.PIC_EINVAL
