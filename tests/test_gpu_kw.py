"""k-omega readout of the probe line (pic_probe_kw; the dispersion picture of
Sec. II / Fig. 2).

1. Parity: on the same seeded inputs the FP64 CUDA path's probe spectra match
   the FP64 oracle's, and the device k-omega map equals the definition
   |sum_p F_p exp(-i k x_p)|^2 evaluated in numpy on the oracle's spectra.
2. Physics: a short current pulse above a free 40 nm silver film launches
   surface plasmons over a range of k; along the k-omega map the strongest
   frequency on each side of the midpoint between the branches lies within
   1.5% of the thin-film dispersion (oracle/theory_imi.branch_omega, pinned in
   tests/test_theory.py) for k = 2e7 .. 9e7 rad/m.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import theory_imi as T
from paper_1505_04007_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


def pulse(w):
    """Ez current pulse (derivative of a Gaussian, tau = 100 dt) on one cell
    column just above the film, 100 cells in from the x-low face."""
    k1 = w.info["film_cells"][1]
    return (2, (100, 101, 0, w.ny, k1 + 1, k1 + 2), 1e15, 400 * w.dt, 100 * w.dt, 0.0)


def kw_definition(F, xp, k):
    return np.abs(np.einsum("pf,qp->qf", F, np.exp(-1j * np.outer(k, xp)))) ** 2


def test_kw_parity_fp64(P):
    w = W.film_line(10, 400, nx=256, nprobes=16, first=40, spacing=8)
    src = pulse(w)
    o = O.from_workload(w, with_particles=False)
    o.add_source(*src)
    o.step(400)
    s = P.Simulation(w, P.PIC_FP64, particles=False)
    P.pic_add_source(s.h, *src)
    s.step(400)
    Fo, Fg = o.probe_read(), s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= 1e-10 * np.linalg.norm(Fo)
    k = np.linspace(1e7, 1.4e8, 27)
    want = kw_definition(Fo[:, 2, :], w.probes[:, 0], k)
    got = s.probe_kw(2, k)
    assert np.abs(got - want).max() <= 1e-10 * want.max()
    s.close()


def test_kw_dispersion_ridge(P):
    thick = 20  # cells: a 40 nm film
    w = W.film_line(thick, 32768)
    s = P.Simulation(w, P.PIC_FP32, particles=False)
    P.pic_add_source(s.h, *pulse(w))
    s.step(32768)
    k = np.linspace(2e7, 9e7, 8)
    kw = s.probe_kw(2, k)
    # the device map is the definition applied to the device's own spectra
    assert np.abs(kw - kw_definition(s.probe_read()[:, 2, :], w.probes[:, 0], k)).max() <= 1e-12 * kw.max()
    f = w.freqs
    for q in range(k.size):
        lo = T.branch_omega(W.TABLE1_WP, thick * 2e-9, k[q], "lower") / (2 * np.pi)
        hi = T.branch_omega(W.TABLE1_WP, thick * 2e-9, k[q], "upper") / (2 * np.pi)
        mid = 0.5 * (lo + hi)
        for band, want in (((f[0], mid), lo), ((mid, f[-1]), hi)):
            idx = np.nonzero((f >= band[0]) & (f <= band[1]))[0]
            got = f[idx[np.argmax(kw[q, idx])]]
            assert abs(got / want - 1) <= 0.015, (k[q], got, want)
    s.close()
