"""Host logic of the Table 1 readout (paper_1505_04007_gb300/table1.py) on
synthetic spectra: the parabolic refinement is exact on a parabola, the
smoothing keeps the area and the centre of a line, and the two strongest
lines of a two-line spectrum are found at their frequencies."""
import numpy as np
import pytest

pytest.importorskip("torch")  # the package imports torch lazily; the helpers do not need a GPU
from paper_1505_04007_gb300 import table1 as T  # noqa: E402


def test_refine_is_exact_on_a_parabola():
    f = 1.0e15 + 1.0e12 * np.arange(50)
    f0 = 1.0e15 + 23.37e12
    p = 5.0 - ((f - f0) / 1e12) ** 2
    m = int(np.argmax(p))
    assert T.refine(f, p, m) == pytest.approx(f0, abs=1e-3)
    assert T.refine(f, p, 0) == f[0]  # no neighbour on one side: the sample itself


def test_smoothing_keeps_area_and_centre():
    f = 0.7e15 + 1.0e12 * np.arange(901)
    p = np.zeros_like(f)
    p[450] = 1.0
    s = T.smooth(f, p)
    assert s.sum() == pytest.approx(1.0, rel=1e-12)
    assert (s * f).sum() / s.sum() == pytest.approx(f[450], rel=1e-15)
    assert np.array_equal(T.smooth(f, p, 0.0), p)


def test_two_lines_found_at_their_frequencies():
    f = 0.7e15 + 1.0e12 * np.arange(901)
    lines = (1.1234e15, 1.3056e15)
    p = sum(a * np.exp(-0.5 * ((f - fl) / 3e12) ** 2) for a, fl in zip((1.0, 0.4), lines))
    p = p + 1e-3 * np.exp(-((f - 0.9e15) / 50e12) ** 2)  # a broad weak background
    pk = T.top_peaks(f, p, 2)
    assert pk[0] == pytest.approx(lines[0], abs=0.2e12)
    assert pk[1] == pytest.approx(lines[1], abs=0.2e12)
    assert T.peak_in(f, p, (1.2e15, 1.4e15)) == pytest.approx(lines[1], abs=0.2e12)
