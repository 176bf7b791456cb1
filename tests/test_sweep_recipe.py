"""The seeded sweep recipe (inputs of the batched stepping): deterministic,
within the stated ranges, every electron in an allowed cell."""
import numpy as np

from paper_1505_04007_gb300 import workloads as W

SMALL = dict(sizes=((64, 96), (32, 48), (48, 64)), nparticles=384)


def test_sweep_recipe():
    ws = W.sweep(n=6, seed=11, nsteps=100, **SMALL)
    again = W.sweep(n=6, seed=11, nsteps=100, **SMALL)
    for w, v in zip(ws, again):
        assert (w.nx, w.ny, w.nz) == (v.nx, v.ny, v.nz) and np.array_equal(w.xyz, v.xyz)
        assert w.nx % 32 == 0 and w.ny % 16 == 0 and w.nz % 16 == 0
        assert 10e-9 <= w.info["thickness"] <= 60e-9 and 5e-9 <= w.info["gap"] <= 20e-9
        assert 10.0 <= w.info["kev"] <= 100.0
        assert W.allowed(w, w.xyz).all()


def test_bench_workloads_take_the_four_cell_kernels():
    """Every workload the bench and the NEXT-row studies time has nx a multiple
    of 4 and, with CPML along x, a CPML width that is one too, so the FP32
    four-cells-per-thread field kernels (and the adjoint's) run on it rather
    than the one-cell kernels."""
    from paper_1505_04007_gb300 import adjoint as A
    ws = [W.c1(nsteps=0), W.c2(nsteps=0), W.c3(nsteps=0)] + W.sweep() + W.table1(64)
    for w in ws:
        assert w.nx % 4 == 0, w.name
        if w.bc[0] == W.BC_CPML or w.bc[1] == W.BC_CPML:
            assert w.cpml_cells % 4 == 0, w.name
    cfg = A.film_config()
    assert cfg.nx % 4 == 0 and cfg.cpml_cells % 4 == 0
