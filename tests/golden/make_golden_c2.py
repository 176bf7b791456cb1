"""Write tests/golden/c2_spectrum.json from the FP64 oracle.

The 384x128x128-cell, 8000-step silver-film run (40 nm film, 1e5 electrons at
50 keV, 64 probes 5 nm above the film) is too long for a test to run on the
oracle, so its spectrum is stored: for the probe-summed power of Ex and of Ez
the peak inside the surface-plasmon band, the band spectrum itself, and each
probe's own peak.  Run: python tests/golden/make_golden_c2.py [threads]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as O  # noqa: E402
from paper_1505_04007_gb300 import workloads as W  # noqa: E402
from _helpers import spectral_peak  # noqa: E402

BAND = (1.2e15, 1.8e15)


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    O.set_threads(threads)
    w = W.c2()
    o = O.from_workload(w)
    t0 = time.time()
    chunk = 500
    done = 0
    while done < w.nsteps:
        n = min(chunk, w.nsteps - done)
        o.step(n)
        done += n
        print(f"{done}/{w.nsteps} steps, {time.time() - t0:.0f} s", flush=True)
    F = o.probe_read()  # [64][3][nf]
    x, u, s = o.particles()
    out = {"workload": "c2 384x128x128, dx=2 nm, 8000 steps, FP64 oracle",
           "band_hz": BAND, "freq_hz": [float(w.freqs[0]), float(w.freqs[1] - w.freqs[0]), int(w.freqs.size)],
           "n_frozen": int(s.sum()), "seconds": time.time() - t0}
    sel = (w.freqs >= BAND[0]) & (w.freqs <= BAND[1])
    for c, name in ((0, "Ex"), (2, "Ez")):
        power = (np.abs(F[:, c, :]) ** 2).sum(axis=0)
        out[f"{name}_sum_peak_hz"] = float(spectral_peak(w.freqs, power, BAND))
        out[f"{name}_sum_band_power"] = [float(v) for v in power[sel]]
        out[f"{name}_probe_peaks_hz"] = [float(spectral_peak(w.freqs, np.abs(F[p, c]) ** 2, BAND))
                                        for p in range(F.shape[0])]
    with open(os.path.join(HERE, "c2_spectrum.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("peaks Ex %.4e Ez %.4e" % (out["Ex_sum_peak_hz"], out["Ez_sum_peak_hz"]))


if __name__ == "__main__":
    main()
