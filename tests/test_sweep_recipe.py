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
