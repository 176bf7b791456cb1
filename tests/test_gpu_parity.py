"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (relative L2 over all cells, E and eta0*H taken together):
  FP64 state: <= 1e-10 (only rounding order differs: atomics, FMA contraction).
  FP32 state: <= 2e-5 against the FP64 oracle.
Probe spectra are compared the same way over all probes and frequencies.
Particle states: FP64 positions within 1e-12 of the cell size, identical
freeze decisions.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04007_gb300 import workloads as W

from _helpers import box_workload, cic_charge, interior_node_mask, node_divergence

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


def rel_l2(a, b):
    nb = np.sqrt(sum((x ** 2).sum() for x in b))
    na = np.sqrt(sum(((x - y) ** 2).sum() for x, y in zip(a, b)))
    return na / nb if nb > 0 else na


def fields_of(getter):
    E = [getter(c) for c in range(3)]
    H = [ETA0 * getter(3 + c) for c in range(3)]
    return E, H


def run_pair(P, w, nsteps, precision, particles=True, probes=True, sources=(), deposit=True):
    o = O.from_workload(w, with_particles=particles, with_probes=probes)
    s = P.Simulation(w, precision, particles=particles, probes=probes)
    for src in sources:
        o.add_source(*src)
        P.pic_add_source(s.h, *src)
    if not deposit:
        o.set_deposit(False)
        P.pic_set_deposit(s.h, False)
    o.step(nsteps)
    s.step(nsteps)
    s.sync()
    return o, s


def compare_fields(o, s, tol):
    Eo, Ho = fields_of(o.get_field)
    Eg, Hg = fields_of(s.field)
    e = rel_l2(Eg, Eo)
    h = rel_l2(Hg, Ho)
    assert e <= tol and h <= tol, (e, h)
    return e, h


# ------------------------------------------------------------ fields only --
def film_box(nx, ny, nz, bc=(W.BC_CPML,) * 6, dx=2e-9):
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[8:13] = 1
    w = box_workload(nx, ny, nz, bc=bc, material=mat, table=W.drude_table(), dx=dx)
    return w


@pytest.mark.parametrize("shape", [(40, 24, 30), (37, 21, 29)])  # several tiles, ragged tails
def test_fields_with_source_fp64(P, shape):
    w = film_box(*shape)
    c = [n // 2 for n in shape]
    srcs = [(2, (c[0], c[0] + 1, c[1], c[1] + 1, 16, 17), 1e18, 30 * w.dt, 8 * w.dt, 0.0),
            (0, (c[0] - 3, c[0] + 2, c[1] - 1, c[1] + 1, 15, 16), 5e17, 40 * w.dt, 10 * w.dt, 1.5e15)]
    o, s = run_pair(P, w, 150, P.PIC_FP64, particles=False, probes=False, sources=srcs)
    compare_fields(o, s, 1e-10)
    for c3 in range(3):
        jo, jg = o.get_field(6 + c3), s.field(P.PIC_JPX + c3)
        assert np.sqrt(((jo - jg) ** 2).sum()) <= 1e-10 * max(np.sqrt((jo ** 2).sum()), 1e-300)


def test_fields_periodic_and_pec_fp64(P):
    bc = (W.BC_PEC, W.BC_CPML, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_CPML, W.BC_PEC)
    w = film_box(36, 20, 28, bc=bc)
    srcs = [(1, (10, 12, 0, 20, 16, 17), 1e18, 30 * w.dt, 8 * w.dt, 0.0)]
    o, s = run_pair(P, w, 120, P.PIC_FP64, particles=False, probes=False, sources=srcs)
    compare_fields(o, s, 1e-10)


# nx % 4 == 0 takes the four-cells-per-thread FP32 kernels, 37 the scalar ones
@pytest.mark.parametrize("shape", [(40, 24, 30), (37, 21, 29)])
def test_fields_with_source_fp32(P, shape):
    w = film_box(*shape)
    srcs = [(2, (20, 21, 12, 13, 16, 17), 1e18, 30 * w.dt, 8 * w.dt, 0.0),
            (1, (14, 18, 3, 15, 14, 15), 4e17, 36 * w.dt, 9 * w.dt, 1.2e15)]
    o, s = run_pair(P, w, 150, P.PIC_FP32, particles=False, probes=False, sources=srcs)
    compare_fields(o, s, 2e-5)


@pytest.mark.parametrize("bc", [
    (W.BC_PEC, W.BC_CPML, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_CPML, W.BC_PEC),
    (W.BC_PERIODIC, W.BC_PERIODIC, W.BC_CPML, W.BC_PEC, W.BC_PEC, W.BC_CPML)])
def test_fields_mixed_boundaries_fp32(P, bc):
    w = film_box(36, 20, 28, bc=bc)
    srcs = [(1, (10, 12, 5, 15, 16, 17), 1e18, 30 * w.dt, 8 * w.dt, 0.0),
            (2, (3, 6, 9, 11, 15, 16), 6e17, 40 * w.dt, 8 * w.dt, 1.4e15)]
    o, s = run_pair(P, w, 140, P.PIC_FP32, particles=False, probes=False, sources=srcs)
    compare_fields(o, s, 2e-5)


# -------------------------------------------------------- full hot path C1 --
@pytest.fixture(scope="module")
def c1_oracle():
    w = W.c1()
    o = O.from_workload(w)
    o.step(w.nsteps)
    Eo, Ho = fields_of(o.get_field)
    xo, uo, so = o.particles()
    return w, Eo, Ho, (xo, uo, so), o.probe_read()


def test_c1_fp64_parity(P, c1_oracle):
    w, Eo, Ho, (xo, uo, so), Fo = c1_oracle
    s = P.Simulation(w, P.PIC_FP64)
    s.step(w.nsteps)
    s.sync()
    Eg, Hg = fields_of(s.field)
    assert rel_l2(Eg, Eo) <= 1e-10
    assert rel_l2(Hg, Ho) <= 1e-10
    xg, ug, sg = s.particles()
    assert np.array_equal(sg, so)
    assert np.abs(xg - xo).max() <= 1e-12 * w.dx
    assert np.abs(ug - uo).max() <= 1e-10 * np.abs(uo).max()
    Fg = s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= 1e-10 * np.linalg.norm(Fo)
    st = s.stats()
    assert st.step == w.nsteps and st.device_error == 0 and st.n_frozen == int(so.sum())


def test_c1_fp32_parity(P, c1_oracle):
    w, Eo, Ho, (xo, uo, so), Fo = c1_oracle
    s = P.Simulation(w, P.PIC_FP32)
    s.step(w.nsteps)
    s.sync()
    Eg, Hg = fields_of(s.field)
    e, h = rel_l2(Eg, Eo), rel_l2(Hg, Ho)
    assert e <= 2e-5 and h <= 2e-5, (e, h)
    Fg = s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= 2e-5 * np.linalg.norm(Fo)
    # freeze decisions may differ only for particles within rounding of a boundary
    assert (sg := s.particles()[2]).sum() == pytest.approx(so.sum(), abs=2)


@pytest.mark.parametrize("nsteps", [0, 1, 63, 64, 65, 130])  # graph boundaries and partial flushes
def test_step_counts_and_partial_dft_flush_fp64(P, nsteps):
    w = W.scaled(W.c1(), 64, 24, 40, 512, nsteps)
    o, s = run_pair(P, w, nsteps, P.PIC_FP64)
    if nsteps:
        compare_fields(o, s, 1e-10)
        Fo, Fg = o.probe_read(), s.probe_read()
        assert np.linalg.norm(Fg - Fo) <= 1e-10 * max(np.linalg.norm(Fo), 1e-300)
    assert s.stats().step == nsteps


def test_probe_read_midway_then_continue(P):
    w = W.scaled(W.c1(), 64, 24, 40, 256, 0)
    o, s = run_pair(P, w, 37, P.PIC_FP64)
    s.probe_read()  # partial flush in the middle of a block
    o.step(100)
    s.step(100)
    Fo, Fg = o.probe_read(), s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= 1e-10 * np.linalg.norm(Fo)


def test_periodic_particles_fp64(P):
    # particles cross a periodic face; metal slab absorbs some of them
    nx, ny, nz = 32, 16, 24
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[4:7] = 1
    bc = (W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_CPML, W.BC_CPML)
    w = box_workload(nx, ny, nz, bc=bc, material=mat, table=W.drude_table())
    w.cpml_cells = 6
    rng = np.random.default_rng(3)
    n = 300
    w.xyz = np.stack([rng.uniform(0, nx, n), rng.uniform(0, ny, n), rng.uniform(9, 13, n)], 1) * w.dx
    w.u = np.zeros((n, 3))
    w.u[:, 0] = -W.electron_momentum(50.0)
    w.u[:, 1] = 0.3 * W.electron_momentum(50.0)
    w.u[:, 2] = -0.2 * W.electron_momentum(50.0)
    w.q_macro = -1e-17
    w.m_macro = W.ME * 1e-17 / W.QE
    o, s = run_pair(P, w, 200, P.PIC_FP64, probes=False)
    compare_fields(o, s, 1e-10)
    xo, _, so = o.particles()
    xg, _, sg = s.particles()
    assert np.array_equal(so, sg) and so.sum() > 0
    assert np.abs(xg - xo).max() <= 1e-12 * w.dx


def test_gpu_gauss_law_fp64(P):
    nx, ny, nz = 24, 16, 20
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[3:6] = 1
    bc = (W.BC_PEC, W.BC_PEC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PEC, W.BC_PEC)
    w = box_workload(nx, ny, nz, bc=bc, material=mat, table=W.drude_table())
    rng = np.random.default_rng(5)
    n = 200
    w.xyz = np.stack([rng.uniform(3, 12, n), rng.uniform(0, ny, n), rng.uniform(7, 10, n)], 1) * w.dx
    w.u = np.zeros((n, 3))
    w.u[:, 0] = W.electron_momentum(30.0)
    w.u[:, 2] = -0.5 * W.electron_momentum(30.0)
    w.q_macro, w.m_macro = -2e-17, W.ME * 2e-17 / W.QE
    s = P.Simulation(w, P.PIC_FP64, probes=False)
    mask = interior_node_mask(w, 1)
    x0 = s.particles()[0]
    E0 = [s.field(c) for c in range(3)]
    worst = 0.0
    for _ in range(30):
        s.step(1)
        x1 = s.particles()[0]
        E1 = [s.field(c) for c in range(3)]
        Jp = [s.field(P.PIC_JPX + c) for c in range(3)]
        lhs = W.EPS0 * node_divergence(w, *[E1[c] - E0[c] for c in range(3)]) + w.dt * node_divergence(w, *Jp)
        drho = cic_charge(w, x1, w.q_macro) - cic_charge(w, x0, w.q_macro)
        worst = max(worst, np.abs((lhs - drho)[mask]).max() / np.abs(drho).max())
        x0, E0 = x1, E1
    assert worst < 1e-9


def test_add_particles_rejects_forbidden_positions(P):
    w = W.c1(nsteps=0)
    s = P.Simulation(w, P.PIC_FP32, particles=False, probes=False, max_particles=10)
    bad = np.array([[1.0 * w.dx, 16 * w.dy, 30 * w.dz],      # inside the 2-cell margin
                    [40 * w.dx, 16 * w.dy, 12 * w.dz]])      # inside the film
    with pytest.raises(P.PicError) as e:
        P.pic_add_particles(s.h, bad, np.zeros((2, 3)), w.q_macro, w.m_macro)
    assert e.value.code == -1
    with pytest.raises(P.PicError) as e:
        P.pic_add_particles(s.h, np.tile(w.xyz[:1], (11, 1)), np.zeros((11, 3)), w.q_macro, w.m_macro)
    assert e.value.code == -3
    assert s.stats().n_particles == 0


def test_library_allocated_memory_path(P):
    # the same C1 slice without a caller workspace (library cudaMalloc)
    w = W.scaled(W.c1(), 64, 24, 40, 512, 80)
    a = P.Simulation(w, P.PIC_FP64, torch_memory=False)
    b = P.Simulation(w, P.PIC_FP64, torch_memory=True)
    a.step(80)
    b.step(80)
    fa = [a.field(c) for c in range(6)]
    fb = [b.field(c) for c in range(6)]
    # atomics may sum in a different order: compare to rounding, not bitwise
    assert rel_l2(fa[:3], fb[:3]) <= 1e-13 and rel_l2(fa[3:], fb[3:]) <= 1e-13
