"""pic_dft_fold_static, the probe-DFT fold that allocates no device memory.

Callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or a cudaMalloc would stall a latency-critical loop) get the same
probe spectrum from caller-owned arrays, with the phase table held in a fixed
array inside the library.  This test feeds it the probe series of a short
FP64 run and checks the result against what the handle's own path
(pic_probe_read) accumulated, over two calls in a row that continue one
series, and again on a fresh accumulator.  It sits in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _interp(E, xi, c):
    """E component c at a point given in cell units (staggered trilinear)."""
    nz, ny, nx = E.shape
    s = np.array(xi, dtype=np.float64) - np.array([0.5 if a == c else 0.0 for a in range(3)])
    b = np.floor(s).astype(int)
    f = s - b
    v = 0.0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                wgt = (f[0] if di else 1 - f[0]) * (f[1] if dj else 1 - f[1]) * (f[2] if dk else 1 - f[2])
                v += wgt * E[b[2] + dk, b[1] + dj, b[0] + di]
    return v


def test_static_fold_matches_probe_read_over_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic as P
    from paper_1505_04007_gb300 import workloads as W

    w = W.scaled(W.c1(), 64, 24, 40, 256, 0)
    probes = np.array([w.probes[0], [30.3 * w.dx, 11.6 * w.dy, 20.7 * w.dz]])
    freqs = w.freqs[::7].copy()          # 286 frequencies
    mask = 0b101
    s = P.Simulation(w, P.PIC_FP64, probes=False, max_probes=2)
    s.probe_dft(probes, freqs, mask)
    d = np.array([w.dx, w.dy, w.dz])
    K = 150                              # two full 64-sample chunks and a ragged tail
    series = np.zeros((K, len(probes), 3))
    for n in range(K):
        s.step(1)
        E = [s.field(c) for c in range(3)]
        for p, x in enumerate(probes):
            for c in range(3):
                if mask & (1 << c):
                    series[n, p, c] = _interp(E[c], x / d, c)
    F_ref = s.probe_read()               # complex [np][3][nf]
    s.close()

    dev = torch.device("cuda")
    st = torch.cuda.Stream()
    samples = torch.tensor(series, dtype=torch.float64, device=dev)
    fr = torch.tensor(freqs, dtype=torch.float64, device=dev)
    F = torch.zeros((len(probes), 3, len(freqs), 2), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    # two calls in a row continue one series: steps 0..99, then 100..149
    cut = 100
    P.pic_dft_fold_static(samples.data_ptr(), cut, len(probes), mask, fr.data_ptr(), len(freqs), 0, w.dt,
                          F.data_ptr(), st.cuda_stream)
    P.pic_dft_fold_static(samples[cut:].data_ptr(), K - cut, len(probes), mask, fr.data_ptr(), len(freqs), cut,
                          w.dt, F.data_ptr(), st.cuda_stream)
    st.synchronize()
    got = F.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    scale = np.linalg.norm(F_ref)
    assert scale > 0
    assert np.linalg.norm(got - F_ref) <= 1e-10 * scale
    # and the DFT definition applied in numpy to the same series:
    # F[p][c][f] = dt sum_s x[s][p][c] exp(+i 2 pi f (s+1) dt)
    t = (np.arange(K) + 1) * w.dt
    ph = np.exp(1j * 2 * np.pi * np.outer(t, freqs))          # [K][nf]
    F_def = np.einsum("spc,sf->pcf", series, ph) * w.dt
    assert np.linalg.norm(got - F_def) <= 1e-10 * np.linalg.norm(F_def)
    assert np.all(got[:, 1] == 0)        # component outside the mask untouched

    # a fresh accumulator, the whole series in one call: same spectrum
    F2 = torch.zeros_like(F)
    P.pic_dft_fold_static(samples.data_ptr(), K, len(probes), mask, fr.data_ptr(), len(freqs), 0, w.dt,
                          F2.data_ptr(), st.cuda_stream)
    st.synchronize()
    g2 = F2.cpu().numpy()
    g2 = g2[..., 0] + 1j * g2[..., 1]
    assert np.linalg.norm(g2 - F_ref) <= 1e-10 * scale

    # beyond the fixed table: rejected before any device work
    big = 2049
    with pytest.raises(P.PicError) as e:
        P.pic_dft_fold_static(samples.data_ptr(), K, len(probes), mask, fr.data_ptr(), big, 0, w.dt,
                              F2.data_ptr(), st.cuda_stream)
    assert e.value.code == -1 and "2048" in str(e.value)
