"""Host logic of bench.py on the CPU: the algorithmic byte counts behind the
roofline figures, checked against counts written out by hand for small
grids (a film of whole planes, CPML slabs on every face)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1505_04007_gb300 import workloads as W  # noqa: E402


def _film(n=16, L=4, k0=6, k1=9):
    w = W.Workload(name="t", nx=n, ny=n, nz=n, dx=2e-9, dy=2e-9, dz=2e-9, dt=W.yee_dt(2e-9, 2e-9, 2e-9),
                   nsteps=0, bc=(W.BC_CPML,) * 6)
    w.cpml_cells = L
    w.material = W.slab_material(n, n, n, k0, k1)
    w.table = W.drude_table()
    return w


def test_field_update_bytes_by_hand():
    n, L, k0, k1 = 16, 4, 6, 9
    w = _film(n, L, k0, k1)
    ab = bench.algorithmic_bytes(w, 4)
    N = n ** 3
    slab = 3 * (2 * L) * n * n  # cells of each axis' two slabs, summed over the axes
    psi = slab * 2 * 2 * 4  # two psi components, read and written, FP32
    # metal edges: x and y edges touch the film on planes k0..k1 (cell below or
    # above in the film), z edges on the film planes themselves
    metal = 2 * (k1 - k0 + 1) * n * n + (k1 - k0) * n * n
    assert ab["slab_cells"] == slab
    assert ab["metal_edges"] == metal
    assert ab["update_H"] == N * 36 + psi
    # edge classes (one byte per edge, three per cell) are read on the planes
    # holding metal edges, k0..k1, only
    assert ab["class_bytes"] == (k1 - k0 + 1) * n * n * 3
    assert ab["update_E"] == N * 36 + (k1 - k0 + 1) * n * n * 3 + psi + metal * 8


def test_fp64_doubles_the_state_bytes():
    w = _film()
    a4, a8 = bench.algorithmic_bytes(w, 4), bench.algorithmic_bytes(w, 8)
    assert a8["update_H"] == 2 * a4["update_H"]
    assert a8["update_E"] - 2 * a4["update_E"] == -a4["class_bytes"]  # class ids stay one byte per edge


def test_adjoint_step_bytes_by_hand():
    from paper_1505_04007_gb300 import adjoint as A
    cfg = A.film_config(nx=24, ny=16, nz=24, design=(8, 11), nsteps=10, cpml=4)
    fwd, bwd = bench.adjoint_bytes(cfg, 4)
    N = 24 * 16 * 24
    slab = N * 8 // 24 + N * 8 // 16 + N * 8 // 24
    planes = (11 + 1) - (8 - 1)  # planes 7..11 hold design edges
    edges = 24 * 16 * (2 * (11 - 8 + 1) + (11 - 8))
    assert fwd == 18 * 4 * N + 8 * 4 * slab + 12 * 24 * 16 * planes + 5 * 4 * edges
    assert bwd == fwd + 32 * edges


def test_measured_peak_reads_the_driver_file_or_falls_back():
    peak, kind = bench.measured_peak()
    assert peak > 1000.0 and kind in ("measured", "fallback")
    if not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert (peak, kind) == (bench.FALLBACK_HBM_GBS, "fallback")
