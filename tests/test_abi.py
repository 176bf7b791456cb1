"""C-ABI checks that need no GPU: the library builds, loads, exports every
entry point include/pic.h declares, and rejects invalid configurations on the
host before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1505_04007_gb300 import pic as P
from paper_1505_04007_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(pic_\w+)\s*\(", src, re.M)))


def test_header_matches_binding_list():
    assert declared_functions() == sorted(P.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = P.load()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_struct_layout_matches_header():
    # offsets of the trailing fields pin the ctypes mirror to the C layout
    assert C.sizeof(P.pic_material) == 24
    assert P.pic_config.flags.offset == C.sizeof(P.pic_config) - 8
    assert C.sizeof(P.pic_stats) == 48 and P.pic_stats.field_path.offset == 40
    assert C.sizeof(P.pic_tuning) == 16 and P.pic_tuning.field_path.offset == 12
    # best (16) + n (4) + 20 candidates (320), then 8-byte aligned doubles
    assert P.pic_tune_report.us_per_step.offset == 344 and C.sizeof(P.pic_tune_report) == 600


def _cfg(**kw):
    w = W.c1(nsteps=0)
    for k, v in kw.items():
        setattr(w, k, v)
    cfg, keep = P.make_config(w, P.PIC_FP32)
    return cfg, keep, w


def test_grids_of_2_to_the_32_cells_are_unsupported():
    cfg, keep, w = _cfg()
    cfg.nx, cfg.ny, cfg.nz = 2048, 2048, 1023  # just below 2^32 cells: sized (host only)
    assert P.pic_workspace_size(cfg) > 2048 * 2048 * 1023 * 12 * 4
    cfg.nz = 1024
    with pytest.raises(P.PicError) as e:
        P.pic_workspace_size(cfg)
    assert e.value.code == -7  # PIC_ERR_UNSUPPORTED: cell offsets are 32-bit


def test_workspace_size_is_host_only_and_scales():
    cfg, keep, w = _cfg()
    n32f = P.pic_workspace_size(cfg)  # c1 takes the fused field pass: two copies of the state
    cfg.flags = P.PIC_FLAG_SPLIT_FIELDS
    n32 = P.pic_workspace_size(cfg)
    cfg.flags = 0
    cfg.precision = P.PIC_FP64
    n64 = P.pic_workspace_size(cfg)
    # 12 state arrays per cell in the state precision plus 4 bytes of tables
    assert n32 >= w.ncells * (12 * 4 + 4)
    assert n64 > n32
    # the fused path's second copy: E, H, J_p, J_f again
    assert n32f >= n32 + w.ncells * 12 * 4


@pytest.mark.parametrize("mutate,code", [
    (lambda c: setattr(c, "dt", c.dt * 2.5), -2),                        # CFL
    (lambda c: c.bc.__setitem__(0, W.BC_PERIODIC), -1),                   # unpaired periodic
    (lambda c: setattr(c, "cpml_cells", 40), -1),                         # slabs do not fit
    (lambda c: setattr(c, "precision", 7), -1),
    (lambda c: setattr(c, "flags", 4), -1),  # an unknown flag bit
    (lambda c: setattr(c, "n_materials", 0), -1),
])
def test_create_rejects_invalid_config_on_host(mutate, code):
    cfg, keep, _ = _cfg()
    mutate(cfg)
    h = C.c_void_p()
    rc = P.load().pic_create(C.byref(cfg), C.byref(h))
    assert rc == code
    assert not h.value
    assert P.pic_last_error() != ""


def test_cfl_bound_includes_drude_term():
    # a plasma frequency high enough to break wp^2 dt^2/4 < 1 - c^2 dt^2 sum(1/d^2)
    cfg, keep, w = _cfg()
    tab = (P.pic_material * 2)(P.pic_material(0, 0, 1), P.pic_material(1.8 / cfg.dt, 0, 1))
    cfg.materials = tab
    h = C.c_void_p()
    assert P.load().pic_create(C.byref(cfg), C.byref(h)) == -2


def test_adjoint_header_matches_binding_and_library():
    from paper_1505_04007_gb300 import adjoint as A
    src = open(os.path.join(ROOT, "include", "pic_adjoint.h")).read()
    declared = sorted(set(re.findall(r"^\s*int\s*(pic_\w+)\s*\(", src, re.M)))
    assert declared == sorted(A.ADJ_EXPORTS)
    L = A.load()
    for name in declared:
        assert hasattr(L, name), name


ERR_ARG, ERR_CFL = -1, -2  # PIC_ERR_ARG, PIC_ERR_CFL of include/pic.h


@pytest.mark.parametrize("field, value, code", [
    ("nsteps", 0, ERR_ARG),
    ("design_k1", 5, ERR_ARG),          # slab of no planes
    ("probe_comp", 3, ERR_ARG),
    ("cpml_cells", 30, ERR_ARG),        # two slabs do not fit
    ("dt", 1e-16, ERR_CFL),
])
def test_adjoint_create_rejects_invalid_config_on_host(field, value, code):
    from paper_1505_04007_gb300 import adjoint as A
    cfg = A.film_config(nx=48, ny=24, nz=40, design=(10, 16), nsteps=10)
    if field == "design_k1":
        cfg.design_k0 = 5
    setattr(cfg, field, value)
    out = C.c_void_p()
    assert A.load().pic_adj_create(C.byref(cfg), C.byref(out)) == code
    assert out.value is None



def test_tuning_and_batch_entry_points_reject_null_on_host():
    """The launch-setting and batch entry points answer PIC_ERR_ARG for a NULL
    handle or batch without touching the device."""
    L = P.load()
    t = P.pic_tuning(4096, 16, 256, 1)
    r = P.pic_tune_report()
    assert L.pic_get_tuning(None, C.byref(t)) == ERR_ARG
    assert L.pic_set_tuning(None, C.byref(t)) == ERR_ARG
    assert L.pic_tune(None, 1, C.byref(r)) == ERR_ARG
    assert L.pic_batch_tune(None, 1, C.byref(r)) == ERR_ARG
    assert L.pic_batch_set_lanes(None, 2) == ERR_ARG
    assert L.pic_batch_step(None, 64) == ERR_ARG
    assert L.pic_batch_sync(None) == ERR_ARG
    assert L.pic_batch_destroy(None) == 0


def test_every_entry_point_is_documented_in_its_header():
    """Each declaration in include/*.h has its comment block right above it
    (what it computes, the arguments and their layout, the errors)."""
    for name in ("pic.h", "pic_adjoint.h"):
        lines = open(os.path.join(ROOT, "include", name)).read().split("\n")
        for i, line in enumerate(lines):
            m = re.match(r"^\s*(?:int|const char \*)\s*(pic_\w+)\s*\(", line)
            if m:
                assert "*/" in "\n".join(lines[max(0, i - 3):i]), (name, m.group(1))
