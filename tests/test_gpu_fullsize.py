"""Checks at the full sizes, in the launch configuration the bench times
(FP32 state, graph replays of 64 steps, sorted deposit, launch settings
chosen by pic_tune on the run's first steps, as bench.py does).

Field values at these sizes have no closed form and the oracle cannot follow
the runs step by step, so they are checked through properties that hold at
any size (the discrete continuity / Gauss law of every step), and, for the
paper-scale run, through the probe spectrum against the stored spectrum of
the FP64 oracle (tests/golden/c2_spectrum.json, written by
tests/golden/make_golden_c2.py, which calls only the oracle).
"""
import json
import os

import numpy as np
import pytest

from paper_1505_04007_gb300 import workloads as W

from _helpers import cic_charge_fast, interior_node_mask, node_divergence, spectral_peak

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c2_spectrum.json")


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


def gauss_residual(P, s, w, mask):
    """max |eps0 div(dE) + dt div(Jp) - drho| / max |drho| over one step."""
    x0 = s.particles()[0]
    E0 = [s.field(c) for c in range(3)]
    s.step(1)
    x1 = s.particles()[0]
    E1 = [s.field(c) for c in range(3)]
    Jp = [s.field(P.PIC_JPX + c) for c in range(3)]
    lhs = W.EPS0 * node_divergence(w, *[E1[c] - E0[c] for c in range(3)]) + w.dt * node_divergence(w, *Jp)
    drho = cic_charge_fast(w, x1, w.q_macro) - cic_charge_fast(w, x0, w.q_macro)
    return np.abs((lhs - drho)[mask]).max() / np.abs(drho).max()


@pytest.mark.parametrize("name,steps", [("c2", 640), ("c3", 128)])
def test_gauss_law_full_size_fp32(P, name, steps):
    w = W.WORKLOADS[name](nsteps=0)
    s = P.Simulation(w, P.PIC_FP32)
    s.tune(rounds=2)  # as the bench: real steps under every candidate, then the fastest
    s.step(steps)  # graph replays (64-step blocks) under the chosen settings
    st = s.stats()
    assert st.device_error == 0 and st.n_frozen < w.nparticles
    mask = interior_node_mask(w, margin=1)
    res = gauss_residual(P, s, w, mask)
    s.close()
    # FP32: the residual is rounding of E (~1e-7 relative) seen through a
    # difference quotient, far below the charge moved in one step
    assert res < 1e-3, res


@pytest.mark.skipif(not os.path.exists(GOLD), reason="stored oracle spectrum not generated")
def test_c2_plasmon_peak_vs_oracle_fp32(P):
    gold = json.load(open(GOLD))
    w = W.c2()
    s = P.Simulation(w, P.PIC_FP32)
    rep = s.tune(rounds=2)  # the tuning steps are steps of the run
    s.step(w.nsteps - rep["steps"])
    F = s.probe_read()
    st = s.stats()
    s.close()
    assert st.step == w.nsteps and st.device_error == 0
    band = tuple(gold["band_hz"])
    for c, name in ((0, "Ex"), (2, "Ez")):
        power = (np.abs(F[:, c, :]) ** 2).sum(axis=0)
        peak = spectral_peak(w.freqs, power, band)
        ref = gold[f"{name}_sum_peak_hz"]
        assert abs(peak / ref - 1) <= 0.005, (name, peak, ref)
        sel = (w.freqs >= band[0]) & (w.freqs <= band[1])
        ref_band = np.array(gold[f"{name}_sum_band_power"])
        assert np.linalg.norm(power[sel] - ref_band) <= 2e-3 * np.linalg.norm(ref_band)
