"""The C-ABI library builds, loads and exports what include/pic.h declares;
host-side validation needs no GPU (CPU only)."""
import ctypes as ct
import os
import subprocess

import pytest

from paper_2101_12149_gb300 import build, pic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return pic.load_library()


def test_exports_every_declared_symbol(lib):
    declared = pic.declared_symbols()
    assert len(declared) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", pic.LIB_PATH], capture_output=True, text=True, check=True)
    exported = {line.split()[-1] for line in out.stdout.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lib, s)


def test_header_struct_layout_matches_binding(tmp_path):
    """sizeof / offsets of pic_grid_desc seen by a C compiler equal the ctypes mirror."""
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "pic.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(pic_grid_desc),"
        " offsetof(pic_grid_desc, order), offsetof(pic_grid_desc, seed), offsetof(pic_grid_desc, tile),"
        " offsetof(pic_grid_desc, solver));return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    G = pic.GridDesc
    assert vals == [ct.sizeof(G), G.order.offset, G.seed.offset, G.tile.offset, G.solver.offset]


def _init(lib, **kw):
    d = pic.GridDesc()
    n = kw.get("n", (8, 8, 8))
    for a in range(3):
        d.n[a] = n[a]
        d.d[a] = kw.get("d", (1.0, 1.0, 1.0))[a]
        d.tile[a] = kw.get("tile", (0, 0, 0))[a]
    d.dt = kw.get("dt", 0.0)
    d.cfl = kw.get("cfl", 0.99)
    d.precision = kw.get("precision", 0)
    d.order = kw.get("order", 1)
    d.sort_every = kw.get("sort_every", 1)
    d.window_axis = kw.get("window_axis", -1)
    d.window_speed = kw.get("window_speed", 0.0)
    d.solver = kw.get("solver", 0)
    h = ct.c_void_p()
    st = lib.pic_init_grid(ct.byref(d), None, ct.byref(h))
    return st, h


@pytest.mark.parametrize("kw,status", [
    (dict(order=0), pic.PIC_ERR_ARG),
    (dict(order=4), pic.PIC_ERR_ARG),
    (dict(precision=7), pic.PIC_ERR_ARG),
    (dict(n=(4, 8, 8), order=3), pic.PIC_ERR_ARG),      # n < order + 2
    (dict(d=(1.0, 0.0, 1.0)), pic.PIC_ERR_ARG),
    (dict(dt=0.6), pic.PIC_ERR_CFL),                     # 1/sqrt(3) = 0.577
    (dict(dt=-0.1), pic.PIC_ERR_ARG),
    (dict(cfl=1.5), pic.PIC_ERR_ARG),
    (dict(sort_every=0), pic.PIC_ERR_ARG),
    (dict(tile=(3, 8, 8)), pic.PIC_ERR_ARG),             # not a power of two
    (dict(tile=(16, 8, 8)), pic.PIC_ERR_ARG),            # larger than the grid
    (dict(window_axis=1), pic.PIC_ERR_ARG),              # only z
    (dict(window_axis=2, sort_every=2), pic.PIC_ERR_ARG),
    (dict(window_axis=2, window_speed=1.5), pic.PIC_ERR_ARG),
    (dict(solver=2), pic.PIC_ERR_ARG),
    (dict(solver=1, d=(1.0, 0.9, 1.0)), pic.PIC_ERR_ARG),   # CKC needs cubic cells
    (dict(solver=1, dt=1.01), pic.PIC_ERR_CFL),              # CKC limit dt = dx
])
def test_invalid_descriptions_rejected_without_gpu(lib, kw, status):
    st, h = _init(lib, **kw)
    assert st == status
    assert h.value is None
    assert lib.pic_last_error()


def test_null_arguments(lib):
    h = ct.c_void_p()
    assert lib.pic_init_grid(None, None, ct.byref(h)) == pic.PIC_ERR_ARG
    assert lib.pic_step(None, 1) == pic.PIC_ERR_ARG
    assert lib.pic_sync(None) == pic.PIC_ERR_ARG
    assert lib.pic_destroy(None) == pic.PIC_OK


def test_batch_tuning_layout_matches_binding(tmp_path):
    src = tmp_path / "tlayout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "pic.h"\n'
        "int main(void){printf(\"%zu %zu %zu\\n\", sizeof(pic_batch_tuning),"
        " offsetof(pic_batch_tuning, run), offsetof(pic_batch_tuning, sort_every));return 0;}\n")
    exe = tmp_path / "tlayout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    T = pic.BatchTuning
    assert vals == [ct.sizeof(T), T.run.offset, T.sort_every.offset]


@pytest.mark.parametrize("ns,orders,dt,cfl,status", [
    ([], [], 0.0, 0.99, pic.PIC_ERR_ARG),                                  # no boxes
    ([(8, 8, 8), (16, 8, 8)], [1, 4], 0.0, 0.99, pic.PIC_ERR_ARG),         # order 4
    ([(8, 8, 8), (4, 8, 8)], [1, 3], 0.0, 0.99, pic.PIC_ERR_ARG),          # n < order + 2
    ([(8, 8, 8)], [1], 0.6, 0.99, pic.PIC_ERR_CFL),                        # above 1/sqrt(3)
    ([(8, 8, 8)], [1], 0.0, 1.5, pic.PIC_ERR_ARG),                         # bad cfl
])
def test_invalid_batches_rejected_without_gpu(lib, ns, orders, dt, cfl, status):
    import numpy as np
    nb = len(ns)
    n_arr = np.ascontiguousarray(np.asarray(ns, dtype=np.int32).reshape(max(nb, 1) if nb else 0, 3)) if nb else \
        np.zeros((1, 3), dtype=np.int32)
    o_arr = np.ascontiguousarray(np.asarray(orders if nb else [1], dtype=np.int32))
    h = ct.c_void_p()
    st = lib.pic_batch_init(nb, n_arr.ctypes.data, None, o_arr.ctypes.data, dt, cfl, 1, None, ct.byref(h))
    assert st == status
    assert h.value is None
