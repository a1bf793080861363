"""The C-ABI library builds, loads and exports every function its header declares;
host-only entry points and argument validation work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"PM_API\s+[\w\s\*]+?\b(pm_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2407_19868_gb300 import build
    build.build()
    from paper_2407_19868_gb300 import api
    return api


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 7
    L = lib.load()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lib.EXPORTED) == names


def test_defaults_and_time_step(lib):
    o = lib.options()
    assert o.Re == 0.01 and o.c2 == 1.5e6 and o.dt_safety == 0.9
    dt = lib.time_step()
    # root of 12 c2 dt^2 + 40 dt / Re - 4 = 0, times 0.9
    a, b = 12 * 1.5e6, 40 / 0.01
    assert dt == pytest.approx(0.9 * (-b + np.sqrt(b * b + 16 * a)) / (2 * a), rel=1e-14)
    assert lib.strerror(lib.PM_ERR_NOT_PERCOLATING).startswith("no fluid path")


def test_invalid_arguments_rejected_before_any_device_work(lib):
    L = lib.load()
    o = lib.options()
    mask = np.zeros((4, 4, 4), dtype=np.uint8)
    dom = lib.Domain(4, 4, 4, mask.ctypes.data, 0, 1.0, 1.0, (C.c_int32 * 3)(0, 0, 0))
    assert L.pm_iterate(C.byref(dom), 3, 1.0, C.byref(o), 1, None, None, None) == lib.PM_ERR_INVALID_ARG
    bad = lib.Domain(0, 4, 4, mask.ctypes.data, 0, 1.0, 1.0, (C.c_int32 * 3)(0, 0, 0))
    k = (C.c_double * 9)()
    assert L.pm_permeability_tensor(C.byref(bad), 1.0, C.byref(o), k, None, None, None) == lib.PM_ERR_INVALID_ARG
    o.precision = 7
    assert L.pm_permeability_tensor(C.byref(dom), 1.0, C.byref(o), k, None, None, None) == lib.PM_ERR_INVALID_ARG
    o = lib.options(tol=-1.0)
    assert L.pm_permeability_tensor(C.byref(dom), 1.0, C.byref(o), k, None, None, None) == lib.PM_ERR_INVALID_ARG
    o = lib.options(schedule=-2)
    assert L.pm_permeability_tensor(C.byref(dom), 1.0, C.byref(o), k, None, None, None) == lib.PM_ERR_INVALID_ARG
    for bad_opt in ({"schedule_split": -1}, {"schedule_split": 65}, {"dc_extrapolate": 2}, {"tile": 4},
                    {"field_memory": 3}, {"sequence": 2}):
        o = lib.options(**bad_opt)
        assert L.pm_permeability_tensor(C.byref(dom), 1.0, C.byref(o), k, None, None, None) == \
            lib.PM_ERR_INVALID_ARG, bad_opt


def test_struct_layout_matches_header(lib, tmp_path):
    """ctypes mirrors of pm_domain / pm_options / pm_stats have the C compiler's layout."""
    import subprocess
    fields = {"pm_domain": (lib.Domain, ["nx", "mask", "voxel_size", "bc"]),
              "pm_options": (lib.Options, ["tol", "max_iter", "precision", "c2", "dc_switch_tol", "kernel",
                                           "autotune", "schedule", "tile", "sequence", "field_memory",
                                           "schedule_split", "dc_extrapolate"]),
              "pm_stats": (lib.Stats, ["iters", "q", "sweep_ms", "status", "percolates", "schedule", "setup_seconds",
                                       "n_fluid", "sweep_ms_src", "kernel_launches", "tile",
                                       "schedule_split"])}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "poremaps_gb.h"', "int main(void){"]
    for st, (_, fs) in fields.items():
        src.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            src.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for st, (cls, fs) in fields.items():
        assert int(out[st]) == C.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_fixed_pressure_axis_rejections_before_any_device_work(lib):
    """A fixed-pressure axis: one at most, at least 3 cells, drive along it; entry points
    that need several drives or the transposed operator refuse it."""
    L = lib.load()
    o = lib.options()
    mask = np.zeros((4, 4, 5), dtype=np.uint8)
    k = (C.c_double * 9)()
    kc = (C.c_double * 3)()

    def dom(bc, m=mask):
        nz, ny, nx = m.shape
        return lib.Domain(nx, ny, nz, m.ctypes.data, 0, 1.0, 1.0, (C.c_int32 * 3)(*bc))

    P = lib.PRESSURE
    two = dom((P, P, 0))
    assert L.pm_solve_direction(C.byref(two), 0, 1.0, C.byref(o), None, None, None, None, kc, None,
                                None) == lib.PM_ERR_INVALID_ARG
    short = dom((0, 0, P), np.zeros((2, 4, 5), dtype=np.uint8))
    assert L.pm_solve_direction(C.byref(short), 2, 1.0, C.byref(o), None, None, None, None, kc, None,
                                None) == lib.PM_ERR_INVALID_ARG
    px = dom((P, 0, 1))
    assert L.pm_solve_direction(C.byref(px), 1, 1.0, C.byref(o), None, None, None, None, kc, None,
                                None) == lib.PM_ERR_INVALID_ARG
    u = (C.c_float * (3 * mask.size))()
    p = (C.c_float * mask.size)()
    assert L.pm_iterate(C.byref(px), 2, 1.0, C.byref(o), 1, u, p, None) == lib.PM_ERR_INVALID_ARG
    assert L.pm_permeability_tensor(C.byref(px), 1.0, C.byref(o), k, None, None, None) == lib.PM_ERR_UNSUPPORTED
    assert L.pm_iterate_noalloc(C.byref(px), 0, 1.0, C.byref(o), 1, u, p, None) == lib.PM_ERR_UNSUPPORTED
    w = (C.c_double * 9)(*([1.0] + [0.0] * 8))
    assert L.pm_sensitivity(C.byref(px), None, w, C.byref(o), None, None, None, None, 0,
                            None) == lib.PM_ERR_UNSUPPORTED
    doms = (lib.Domain * 1)(px)
    assert L.pm_batch_ktensor(1, doms, None, C.byref(o), k, None, None, None) == lib.PM_ERR_UNSUPPORTED
    dc = lib.options(precision="dc64")
    assert L.pm_solve_direction(C.byref(px), 0, 1.0, C.byref(dc), None, None, None, None, kc, None,
                                None) == lib.PM_ERR_UNSUPPORTED
