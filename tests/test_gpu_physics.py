"""The same surface-plasmon runs as tests/test_oracle_physics.py on the CUDA
path (FP32 and FP64): each dominant spectral peak within 1% of the film
theory and within 0.2% of the FP64 oracle's peak for the same inputs."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import theory_imi as T

from _helpers import FILM_CASES, film_spp_workload, spectral_peak

pytestmark = pytest.mark.gpu
WP = 1.2e16


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


@pytest.mark.parametrize("case", FILM_CASES, ids=lambda c: f"{c[0] * 2}nm")
def test_film_plasmon_peaks_gpu(P, case):
    thick, steps, band = case
    w = film_spp_workload(thick, steps)
    o = O.from_workload(w)
    o.step(w.nsteps)
    Fo = o.probe_read()[0]
    if thick == 75:
        f_theory = T.thick_film_omega(WP, 100.0) / (2 * math.pi)
    else:
        f_theory = T.film_modes(WP, thick * 2e-9, 100.0)[1] / (2 * math.pi)
    for prec in (P.PIC_FP32, P.PIC_FP64):
        s = P.Simulation(w, prec)
        s.step(w.nsteps)
        Fg = s.probe_read()[0]
        s.close()
        for c in (0, 2):
            pg = spectral_peak(w.freqs, np.abs(Fg[c]) ** 2, band)
            po = spectral_peak(w.freqs, np.abs(Fo[c]) ** 2, band)
            assert abs(pg / f_theory - 1) < 0.01, (prec, c, pg, f_theory)
            assert abs(pg / po - 1) < 2e-3, (prec, c, pg, po)
