"""The fused FP32 field pass (E of step n+1 and H of step n+3/2 in one sweep
over the grid, two copies of the state, the free current added afterwards)
against the FP64 oracle and against the split FP32 updates.

- Grids of every shape the pass tiles unevenly (x not a multiple of the
  32-cell tile, y not a multiple of the 15-row tile, z not a multiple of the
  plane chunk), CPML on all six faces or PEC on some, metal planes, three
  prescribed sources (two inside the x and y slabs): fields and J_p within
  2e-5 of the oracle; the split updates (PIC_FLAG_SPLIT_FIELDS) agree with
  the fused pass to 1e-5.  All four tile kinds run (inner, y slab, x slab,
  corner).
- A grid too narrow for the pass's tiles (a tile would meet the slabs of
  both faces) takes the split updates and keeps parity.
- Electrons (dense C1 slice): fields, spectra within 2e-5 of the oracle.
- Reading the state at odd and even step counts (the pass keeps H half a
  step ahead) gives the oracle's E^n, H^{n-1/2}, J_p and the last step's
  J_f; overwriting E in the middle of a run leaves the fused state and the
  run continues like the oracle's.
- A checkpoint taken at an odd step on the fused path resumes bit for bit
  (fields only: no atomic sums).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04007_gb300 import workloads as W

from _helpers import box_workload

pytestmark = pytest.mark.gpu

ETA0 = (W.MU0 / W.EPS0) ** 0.5


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


def rel(a, b):
    num = sum(float(((x - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((y ** 2).sum()) for y in b)
    return (num / den) ** 0.5 if den > 0 else num ** 0.5


def fields(get):
    return [get(c) for c in range(3)] + [ETA0 * get(3 + c) for c in range(3)]


def film_box(nx, ny, nz, bc=(W.BC_CPML,) * 6, k0=8, k1=13):
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[k0:k1] = 1
    return box_workload(nx, ny, nz, bc=bc, material=mat, table=W.drude_table())


def sources_for(w):
    c = (w.nx // 2, w.ny // 2)
    return [(2, (c[0], c[0] + 1, c[1], c[1] + 1, 16, 17), 1e18, 30 * w.dt, 8 * w.dt, 0.0),
            (0, (c[0] - 3, c[0] + 2, c[1] - 1, c[1] + 1, 15, 16), 5e17, 40 * w.dt, 10 * w.dt, 1.5e15),
            (1, (3, 7, 2, 5, 18, 19), 4e17, 36 * w.dt, 9 * w.dt, 1.2e15)]  # inside the x and y slabs


SHAPES = [(64, 24, 40), (44, 24, 45), (100, 25, 70)]
BCS = [(W.BC_CPML,) * 6, (W.BC_PEC, W.BC_CPML, W.BC_CPML, W.BC_PEC, W.BC_CPML, W.BC_CPML)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", BCS)
def test_fused_pass_against_oracle_and_split(P, shape, bc):
    w = film_box(*shape, bc=bc)
    srcs = sources_for(w)
    nsteps = 150
    o = O.from_workload(w, with_particles=False, with_probes=False)
    s = P.Simulation(w, P.PIC_FP32, particles=False, probes=False)
    t = P.Simulation(w, P.PIC_FP32, particles=False, probes=False, flags=P.PIC_FLAG_SPLIT_FIELDS)
    assert s.stats().field_path == 1 and t.stats().field_path == 0
    for src in srcs:
        o.add_source(*src)
        P.pic_add_source(s.h, *src)
        P.pic_add_source(t.h, *src)
    o.step(nsteps)
    s.step(nsteps)
    t.step(nsteps)
    s.sync()
    ref = fields(o.get_field)
    got = fields(s.field)
    assert rel(got, ref) <= 2e-5
    assert rel(got, fields(t.field)) <= 1e-5
    for c in range(3):
        jo, jg = o.get_field(6 + c), s.field(P.PIC_JPX + c)
        assert np.linalg.norm(jg - jo) <= 2e-5 * max(np.linalg.norm(jo), 1e-300)
    assert s.stats().device_error == 0


@pytest.mark.parametrize("shape", [(64, 24, 40), (100, 25, 70)])
def test_fused_pass_metal_inside_z_slabs(P, shape):
    """Metal planes inside both z absorbing slabs: planes that hold per-edge
    classes (Eq. 6) and z-slab CPML memory at once, for the group and its halo
    cell, against the oracle and the split updates."""
    nx, ny, nz = shape
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[4:11] = 1
    mat[nz - 6:nz - 2] = 1
    w = box_workload(nx, ny, nz, bc=(W.BC_CPML,) * 6, material=mat, table=W.drude_table())
    o = O.from_workload(w, with_particles=False, with_probes=False)
    s = P.Simulation(w, P.PIC_FP32, particles=False, probes=False)
    t = P.Simulation(w, P.PIC_FP32, particles=False, probes=False, flags=P.PIC_FLAG_SPLIT_FIELDS)
    assert s.stats().field_path == 1
    for src in sources_for(w):
        o.add_source(*src)
        P.pic_add_source(s.h, *src)
        P.pic_add_source(t.h, *src)
    o.step(120)
    s.step(120)
    t.step(120)
    ref = fields(o.get_field)
    got = fields(s.field)
    assert rel(got, ref) <= 2e-5
    assert rel(got, fields(t.field)) <= 1e-5
    for c in range(3):
        jo, jg = o.get_field(6 + c), s.field(P.PIC_JPX + c)
        assert np.linalg.norm(jg - jo) <= 2e-5 * max(np.linalg.norm(jo), 1e-300)
    assert s.stats().device_error == 0


@pytest.mark.parametrize("shape", [(36, 30, 40), (64, 21, 40)])
def test_narrow_grid_takes_the_split_updates(P, shape):
    w = film_box(*shape)
    o = O.from_workload(w, with_particles=False, with_probes=False)
    s = P.Simulation(w, P.PIC_FP32, particles=False, probes=False)
    assert s.stats().field_path == 0 and s.tuning[3] == 0
    src = sources_for(w)[0]
    o.add_source(*src)
    P.pic_add_source(s.h, *src)
    o.step(90)
    s.step(90)
    assert rel(fields(s.field), fields(o.get_field)) <= 2e-5


def test_fused_pass_with_electrons(P):
    w = W.scaled(W.c1(), 64, 24, 40, 4096, 0)
    nsteps = 200
    o = O.from_workload(w)
    s = P.Simulation(w, P.PIC_FP32)
    assert s.stats().field_path == 1
    o.step(nsteps)
    s.step(nsteps)
    assert rel(fields(s.field), fields(o.get_field)) <= 2e-5
    Fo, Fg = o.probe_read(), s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= 2e-5 * np.linalg.norm(Fo)
    assert s.stats().device_error == 0


@pytest.mark.parametrize("first", [36, 37])  # the state read at an even and at an odd step count
def test_state_readout_and_set_field(P, first):
    w = film_box(40, 24, 30)
    srcs = sources_for(w)[:2]
    o = O.from_workload(w, with_particles=False, with_probes=False)
    s = P.Simulation(w, P.PIC_FP32, particles=False, probes=False)
    for src in srcs:
        o.add_source(*src)
        P.pic_add_source(s.h, *src)
    o.step(first)
    s.step(first)
    assert rel(fields(s.field), fields(o.get_field)) <= 2e-5
    jp_o = [o.get_field(6 + c) for c in range(3)]
    jf_o = [o.get_field(9 + c) for c in range(3)]
    assert rel([s.field(P.PIC_JPX + c) for c in range(3)], jp_o) <= 2e-5
    assert rel([s.field(P.PIC_JFX + c) for c in range(3)], jf_o) <= 1e-6  # the last step's source current
    # overwrite E (scaled) in both, then continue
    for c in range(3):
        e = o.get_field(c) * 0.5
        o.set_field(c, e)
        s.set_field(P.PIC_EX + c, e)
    o.step(41)
    s.step(41)
    assert rel(fields(s.field), fields(o.get_field)) <= 2e-5
    assert s.stats().step == first + 41


def test_checkpoint_on_fused_path_bitwise(P, tmp_path):
    w = film_box(64, 24, 40)
    rng = np.random.default_rng(7)
    a = P.Simulation(w, P.PIC_FP32, particles=False, probes=False)
    # a smooth random initial field (no sources: no atomic sums anywhere)
    z, y, x = np.meshgrid(np.arange(w.nz), np.arange(w.ny), np.arange(w.nx), indexing="ij")
    for c in range(3):
        k = rng.uniform(0.05, 0.3, 3)
        a.set_field(P.PIC_EX + c, 1e6 * np.sin(k[0] * x + k[1] * y + k[2] * z))
    a.step(45)  # odd: the state lives in the second copy
    path = os.path.join(tmp_path, "fused.bin")
    a.save(path)
    a.step(70)
    b = P.Simulation(w, P.PIC_FP32, particles=False, probes=False)
    b.load(path)
    b.step(70)
    for c in range(9):
        assert np.array_equal(a.field(c), b.field(c)), c
    assert b.stats().step == 115
