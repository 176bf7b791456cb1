"""Adjoint gradients (include/pic_adjoint.h) on the GPU.

- Against the FP64 oracle (oracle/adjoint_oracle.py: the same forward model
  in plain PyTorch CPU ops, differentiated by reverse mode) on a 24x16x24
  study of 120 steps: loss and every mask cell's gradient within 1e-10 (FP64
  path, rel. L2) and 1e-3 (FP32 path).
- Against central finite differences of the library's own forward model, in
  FP64, on a 48x24x40 study (6-plane design slab, 400 steps, 40 keV rigid
  bunch, Ez probe at wp/sqrt(2), seeded mask in [0.2, 0.8]): the mask gradient
  at 32 cells (drawn from the 200 with the largest gradient), d/dwp and
  d/dgamma within 1e-5 of the largest mask gradient (mask) or of the
  derivative itself (wp, gamma), at a relative step of 1e-4.
- The FP32 path's gradient against the FP64 one, and the torch.autograd
  wrapper against the direct call.
- The FP32 kernels with four x cells per thread (nx and the CPML width
  multiples of 4) against the one-cell FP32 kernels (flags bit 0) and the
  FP64 path on the same study.
- Checkpoint mode (flags bit 1: segments of 64 steps recomputed from field
  checkpoints, here 6 whole segments and a partial one) against the default
  mode: the same loss bit for bit, gradients within the atomic-order rounding.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WP, GAMMA = 1.2e16, 1.45e13


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import adjoint
    adjoint.load()
    return adjoint


def small(A, precision):
    from paper_1505_04007_gb300 import pic
    prec = pic.PIC_FP64 if precision == "fp64" else pic.PIC_FP32
    return A.Adjoint(A.film_config(nx=48, ny=24, nz=40, design=(10, 16), nsteps=400, sigma=4e-9, cpml=6,
                                   precision=prec))


@pytest.fixture(scope="module")
def fp64_grad(A):
    st = small(A, "fp64")
    mask = np.random.default_rng(7).uniform(0.2, 0.8, st.n)
    loss = st.forward(mask, WP, GAMMA)
    dm, dwp, dga = st.backward()
    return st, mask, loss, dm, dwp, dga


def test_mask_gradient_matches_central_differences(fp64_grad):
    st, mask, loss, dm, _, _ = fp64_grad
    assert loss > 0 and np.isfinite(dm).all()
    rng = np.random.default_rng(11)
    cells = rng.choice(np.argsort(-np.abs(dm))[:200], 32, replace=False)
    for c in cells:
        h = 1e-4 * mask[c]
        mp, mm = mask.copy(), mask.copy()
        mp[c] += h
        mm[c] -= h
        fd = (st.forward(mp, WP, GAMMA) - st.forward(mm, WP, GAMMA)) / (2 * h)
        assert abs(fd - dm[c]) <= 1e-5 * np.abs(dm).max(), (c, fd, dm[c])


def test_wp_and_gamma_gradients_match_central_differences(fp64_grad):
    st, mask, loss, _, dwp, dga = fp64_grad
    for val, grad, f in ((WP, dwp, lambda v: st.forward(mask, v, GAMMA)),
                         (GAMMA, dga, lambda v: st.forward(mask, WP, v))):
        h = 1e-4 * val
        fd = (f(val + h) - f(val - h)) / (2 * h)
        assert abs(fd - grad) <= 1e-5 * abs(grad), (fd, grad)


def test_fp32_gradient_close_to_fp64(A, fp64_grad):
    _, mask, loss64, dm64, dwp64, dga64 = fp64_grad
    st = small(A, "fp32")
    loss = st.forward(mask, WP, GAMMA)
    dm, dwp, dga = st.backward()
    st.close()
    assert abs(loss / loss64 - 1) <= 1e-4
    assert np.linalg.norm(dm - dm64) <= 1e-3 * np.linalg.norm(dm64)
    assert abs(dwp / dwp64 - 1) <= 1e-3 and abs(dga / dga64 - 1) <= 1e-3


def test_autograd_wrapper(A, fp64_grad):
    import torch
    st, mask, loss, dm, dwp, dga = fp64_grad
    f = A.plasmon_loss(st)
    m = torch.tensor(mask, dtype=torch.float64, requires_grad=True)
    w = torch.tensor(WP, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(GAMMA, dtype=torch.float64, requires_grad=True)
    out = f(m, w, g)
    (3.0 * out).backward()
    # a second forward/backward: equal up to the order of the atomic sums
    assert float(out.detach()) == pytest.approx(loss, rel=1e-12)
    assert np.abs(m.grad.numpy() - 3.0 * dm).max() <= 1e-9 * 3.0 * np.abs(dm).max()
    assert float(w.grad) == pytest.approx(3.0 * dwp, rel=1e-9)
    assert float(g.grad) == pytest.approx(3.0 * dga, rel=1e-9)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-3)])
def test_gradient_matches_the_oracle(A, precision, tol):
    from oracle import adjoint_oracle as AO
    from paper_1505_04007_gb300 import pic
    prec = pic.PIC_FP64 if precision == "fp64" else pic.PIC_FP32
    cfg = A.film_config(nx=24, ny=16, nz=24, design=(8, 11), nsteps=120, sigma=4e-9, cpml=4, precision=prec)
    st = A.Adjoint(cfg)
    mask = np.random.default_rng(13).uniform(0.2, 0.8, st.n)
    loss = st.forward(mask, WP, GAMMA)
    dm, dwp, dga = st.backward()
    st.close()
    L0, dm0, dwp0, dga0 = AO.loss_and_grad(cfg, mask, WP, GAMMA)
    assert abs(loss / L0 - 1) <= tol, (loss, L0)
    assert np.linalg.norm(dm - dm0) <= tol * np.linalg.norm(dm0)
    assert abs(dwp / dwp0 - 1) <= tol, (dwp, dwp0)
    assert abs(dga / dga0 - 1) <= tol, (dga, dga0)


def test_four_cell_fp32_kernels_match_one_cell_and_fp64(A):
    from paper_1505_04007_gb300 import pic
    res = {}
    for name, prec, flags in (("four", pic.PIC_FP32, 0), ("one", pic.PIC_FP32, 1), ("fp64", pic.PIC_FP64, 0)):
        cfg = A.film_config(nx=48, ny=24, nz=40, design=(10, 16), nsteps=400, sigma=4e-9, cpml=8, precision=prec)
        cfg.flags = flags
        st = A.Adjoint(cfg)
        mask = np.random.default_rng(17).uniform(0.2, 0.8, st.n)
        loss = st.forward(mask, WP, GAMMA)
        res[name] = (loss, *st.backward())
        st.close()
    for ref, tol in (("one", 1e-4), ("fp64", 1e-3)):
        L0, dm0, dw0, dg0 = res[ref]
        L, dm, dw, dg = res["four"]
        assert abs(L / L0 - 1) <= tol / 10, (ref, L, L0)
        assert np.linalg.norm(dm - dm0) <= tol * np.linalg.norm(dm0), ref
        assert abs(dw / dw0 - 1) <= tol and abs(dg / dg0 - 1) <= tol, (ref, dw, dw0, dg, dg0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_checkpoint_mode_equals_stored_steps(A, precision, tol):
    from paper_1505_04007_gb300 import pic
    prec = pic.PIC_FP64 if precision == "fp64" else pic.PIC_FP32
    res = {}
    for flags in (0, 2):
        cfg = A.film_config(nx=48, ny=24, nz=40, design=(10, 16), nsteps=400, sigma=4e-9, cpml=8, precision=prec)
        cfg.flags = flags
        st = A.Adjoint(cfg)
        mask = np.random.default_rng(19).uniform(0.2, 0.8, st.n)
        loss = st.forward(mask, WP, GAMMA)
        res[flags] = (loss, *st.backward())
        st.close()
    L0, dm0, dw0, dg0 = res[0]
    L2, dm2, dw2, dg2 = res[2]
    assert L2 == L0
    assert np.linalg.norm(dm2 - dm0) <= tol * np.linalg.norm(dm0)
    assert abs(dw2 / dw0 - 1) <= tol and abs(dg2 / dg0 - 1) <= tol
