"""The paper's film-mode study (Sec. IV, Table 1) on the CUDA path.

Eight quasi-2D runs, one per film thickness (20-80 nm and 150 nm, silver with
the paper's Drude parameters, a 100 keV electron sheet 20 nm above the film),
stepped together through one pic_batch; the Ez spectrum 5 nm above each film
is read from the probe DFT and its strongest peaks are the film modes where
the electron line crosses the two branches of the thin-film dispersion.

    python -m paper_1505_04007_gb300.table1 [--steps 65536] [--nx 2048]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import pic
from . import workloads as W


def run(nsteps: int = 65536, nx: int = 2048, precision: int = pic.PIC_FP32):
    """Step the thickness series together; returns (workloads, freqs,
    [|Ez(f)|^2 per thickness], seconds)."""
    ws = W.table1(nsteps, nx=nx)
    sims = [pic.Simulation(w, precision) for w in ws]
    b = pic.Batch(sims)
    t0 = time.perf_counter()
    b.step(nsteps)
    b.sync()
    secs = time.perf_counter() - t0
    power = [np.abs(s.probe_read()[0][2]) ** 2 for s in sims]
    b.close()
    for s in sims:
        s.close()
    return ws, ws[0].freqs, power, secs


def refine(freqs, power, m: int) -> float:
    """Frequency of sample m refined by the vertex of the parabola through it
    and its two neighbours."""
    if 0 < m < len(power) - 1:
        y0, y1, y2 = power[m - 1], power[m], power[m + 1]
        den = y0 - 2 * y1 + y2
        shift = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        return float(freqs[m] + shift * (freqs[1] - freqs[0]))
    return float(freqs[m])


SMOOTH_HZ = 4e12  # about half the 1/T resolution of a 65 536-step (126 fs) record


def smooth(freqs, power, width_hz: float = SMOOTH_HZ):
    """power convolved with a normalised Gaussian of rms width width_hz: a
    record of length T resolves lines only to ~1/T, and the side lobes of a
    line cut off by the end of the record can outgrow its centre sample."""
    if width_hz <= 0:
        return np.asarray(power, np.float64)
    s = width_hz / (freqs[1] - freqs[0])
    half = int(4 * s) + 1
    x = np.arange(-half, half + 1)
    k = np.exp(-0.5 * (x / s) ** 2)
    return np.convolve(np.asarray(power, np.float64), k / k.sum(), mode="same")


def peak_in(freqs, power, band, width_hz: float = SMOOTH_HZ) -> float:
    """Refined frequency of the largest sample of the smoothed power inside
    band = (f_lo, f_hi)."""
    p = smooth(freqs, power, width_hz)
    idx = np.nonzero((freqs >= band[0]) & (freqs <= band[1]))[0]
    return refine(freqs, p, int(idx[np.argmax(p[idx])]))


def top_peaks(freqs, power, n: int = 2, width_hz: float = SMOOTH_HZ) -> list:
    """The n largest local maxima of the smoothed power, refined, in
    increasing frequency."""
    p = smooth(freqs, power, width_hz)
    lm = [i for i in range(1, len(p) - 1) if p[i] > p[i - 1] and p[i] >= p[i + 1]]
    lm = sorted(lm, key=lambda i: -p[i])[:n]
    return sorted(refine(freqs, p, i) for i in lm)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=65536)
    ap.add_argument("--nx", type=int, default=2048)
    args = ap.parse_args()
    ws, f, power, secs = run(args.steps, args.nx)
    rows = []
    for w, p in zip(ws, power):
        d_nm = round(w.info["thickness"] * 1e9)
        pk = [x / 1e12 for x in top_peaks(f, p, 2)]
        rows.append({"thickness_nm": d_nm, "peaks_thz": [round(x, 1) for x in pk]})
        print(f"{d_nm:4d} nm: " + "  ".join(f"{x:7.1f} THz" for x in pk), flush=True)
    cells = sum(w.ncells for w in ws)
    print(json.dumps({"steps": args.steps, "nx": args.nx, "seconds": secs,
                      "gcell_upd_per_s": cells * args.steps / secs / 1e9, "modes": rows}))


if __name__ == "__main__":
    main()
