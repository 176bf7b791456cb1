"""The seeded inputs of the three single-run sizes (the paper's setup, Sec.
III, with the unstated details as the design notes read them): grid, film,
bunch and probes as stated, deterministic under the seed, every electron in
an allowed cell, and the bunch statistics those of the stated Gaussian up to
sampling and the rejection of points in the metal and the face margins."""
import math

import numpy as np
import pytest

from paper_1505_04007_gb300 import workloads as W

ME_KEV = 510.99895

SPEC = {  # name: grid, dx, film planes, electrons, charge, keV, centre (x, z above top), sigma, probes
    "c1": ((128, 32, 48), 2e-9, (8, 18), 4096, 1e-15, 30.0, (20e-9, 10e-9), 5e-9, 1),
    "c2": ((384, 128, 128), 2e-9, (8, 28), 100000, 1e-15, 50.0, (44e-9, 15e-9), 8e-9, 64),
    "c3": ((768, 256, 256), 1e-9, (8, 18), 1000000, 2e-15, 30.0, (25e-9, 5e-9), 5e-9, 1),
}


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_single_run_recipe(name):
    (nx, ny, nz), dx, (k0, k1), npart, charge, kev, (x0, gap), sigma, nprobe = SPEC[name]
    w = W.WORKLOADS[name](nsteps=0)
    assert (w.nx, w.ny, w.nz, w.dx) == (nx, ny, nz, dx)
    assert w.dt == pytest.approx(0.5 * dx / (W.C0 * math.sqrt(3.0)), rel=1e-15)
    # film: silver planes k0..k1-1 over the whole x-y extent, vacuum elsewhere
    wp = w.table[:, 0][w.material]
    assert (wp[k0:k1] == W.AG_WP).all() and (wp[:k0] == 0).all() and (wp[k1:] == 0).all()
    # bunch
    assert w.nparticles == npart
    assert w.q_macro * npart == pytest.approx(-charge, rel=1e-12)
    g = 1.0 + kev / ME_KEV
    assert np.allclose(w.u[:, 0], W.C0 * math.sqrt(g * g - 1.0), rtol=1e-12) and not w.u[:, 1:].any()
    assert W.allowed(w, w.xyz).all()
    top = k1 * dx
    centre = np.array([x0, 0.5 * ny * dx, top + gap])
    mean, std = w.xyz.mean(axis=0), w.xyz.std(axis=0)
    # x and y are untouched by the film (only far tails are cut): mean and spread as drawn
    assert abs(mean[0] - centre[0]) < 5 * sigma / math.sqrt(npart) + 0.02 * sigma
    assert abs(mean[1] - centre[1]) < 5 * sigma / math.sqrt(npart) + 0.02 * sigma
    assert std[1] == pytest.approx(sigma, rel=0.05)
    # z: points below the film top were redrawn, so the mean sits at or above the centre
    assert centre[2] - 0.01 * sigma <= mean[2] < centre[2] + 0.5 * sigma
    # probes 5 nm above the film top
    assert w.probes.shape == (nprobe, 3)
    assert np.allclose(w.probes[:, 2], top + 5e-9, rtol=1e-12)


def test_recipes_are_deterministic():
    a, b = W.c1(nsteps=0), W.c1(nsteps=0)
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.material, b.material)
    c = W.c1(seed=7, nsteps=0)
    assert not np.array_equal(a.xyz, c.xyz)
