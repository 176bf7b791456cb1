"""The whole method on the oracle against the paper's theory (Sec. IV).

A 100 keV electron sheet moving parallel to a silver film (the paper's wp and
gamma) excites surface plasmons; the spectrum of the field 5 nm above the
film peaks where the electron line crosses the film dispersion:
* thick film (150 nm): the single-interface value wp/sqrt(1+gamma_L^2)
  (1225.25 THz, the paper's 150 nm entry of Table 1), within 1%;
* thin films (20 nm, 40 nm): the dominant peak is the upper (tanh) branch of
  the film theory, within 1%, and the branches move apart as the film thins.
Quasi-2D (periodic y) runs of 8000-24000 steps, about 30 s in all.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import theory_imi as T

from _helpers import FILM_CASES, film_spp_workload, spectral_peak

WP = 1.2e16


@pytest.fixture(scope="module")
def peaks():
    out = {}
    for thick, steps, band in FILM_CASES:
        w = film_spp_workload(thick, steps)
        o = O.from_workload(w)
        o.step(w.nsteps)
        F = o.probe_read()[0]
        out[thick] = {name: spectral_peak(w.freqs, np.abs(F[c]) ** 2, band) for c, name in ((0, "Ex"), (2, "Ez"))}
    return out


def test_thick_film_plasmon_frequency(peaks):
    f_theory = T.thick_film_omega(WP, 100.0) / (2 * math.pi)
    for name in ("Ex", "Ez"):
        assert abs(peaks[75][name] / f_theory - 1) < 0.01, (name, peaks[75][name], f_theory)


@pytest.mark.parametrize("thick", [10, 20])
def test_thin_film_upper_branch(peaks, thick):
    _, hi = T.film_modes(WP, thick * 2e-9, 100.0)
    f_hi = hi / (2 * math.pi)
    for name in ("Ex", "Ez"):
        assert abs(peaks[thick][name] / f_hi - 1) < 0.01, (name, peaks[thick][name], f_hi)


def test_split_shrinks_with_thickness(peaks):
    assert peaks[10]["Ez"] > peaks[20]["Ez"] > peaks[75]["Ez"]
