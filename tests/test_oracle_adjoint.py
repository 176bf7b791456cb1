"""Pins of the adjoint oracle (oracle/adjoint_oracle.py) to things other than
itself, on the CPU:

- its field step (H with CPML, Eq. 6, Eq. 8 with CPML, held faces, four-cell
  edge averaging of the mask) and probe DFT equal the C oracle's field step
  and probe from the same random state, with the mask expressed as a material
  table (the C oracle is pinned by the tests of test_oracle_pins.py);
- the bunch current integrates to q v over the grid and is centred on
  x0 + v t (closed forms of the Gaussian);
- its gradient equals central differences of its own forward model;
- without metal, L does not depend on wp or gamma (zero derivatives).
"""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint_oracle as AO
from oracle import oracle as O

EPS0, MU0 = 8.8541878128e-12, 1.25663706212e-6
C0 = 1.0 / math.sqrt(EPS0 * MU0)
WP, GAMMA = 1.2e16, 1.45e13


class Cfg:
    """The fields of pic_adj_config for a small film study."""

    def __init__(self, nx=20, ny=14, nz=22, dx=2e-9, cpml=4, kappa_max=1.0, design=(8, 11), nsteps=60,
                 kev=40.0, sigma=4e-9, gap=6e-9, comp=2):
        self.nx, self.ny, self.nz, self.dx = nx, ny, nz, dx
        self.dt = 0.5 * dx / (C0 * math.sqrt(3.0))
        self.cpml_cells, self.cpml_order, self.cpml_sigma_fac = cpml, 3.0, 0.8
        self.cpml_kappa_max, self.cpml_alpha_max = kappa_max, 0.05 * EPS0 * WP
        self.eps0, self.mu0 = EPS0, MU0
        self.design_k0, self.design_k1 = design
        g = 1.0 + kev / 510.99895
        self.bunch_q, self.bunch_sigma = -1e-15, sigma
        self.bunch_v = C0 * math.sqrt(1.0 - 1.0 / g ** 2)
        top = design[1] * dx
        self.bunch_x0, self.bunch_y0, self.bunch_z0 = (cpml + 2) * dx, 0.5 * ny * dx, top + gap
        self.probe = [0.7 * nx * dx, 0.5 * ny * dx + 0.3 * dx, top + 2.6 * dx]
        self.probe_comp = comp
        self.omega0 = WP / math.sqrt(2.0)
        self.nsteps = nsteps


class _W:
    """Workload-like description of the same grid for the C oracle."""

    def __init__(self, cfg, material, table):
        self.nx, self.ny, self.nz = cfg.nx, cfg.ny, cfg.nz
        self.dx = self.dy = self.dz = cfg.dx
        self.dt = cfg.dt
        self.bc = (0,) * 6  # CPML on every face
        self.cpml_cells, self.cpml_order = cfg.cpml_cells, cfg.cpml_order
        self.cpml_sigma_fac, self.cpml_kappa_max = cfg.cpml_sigma_fac, cfg.cpml_kappa_max
        self.cpml_alpha_max = cfg.cpml_alpha_max
        self.material, self.table = material, table


@pytest.mark.parametrize("kappa_max", [1.0, 2.5])
def test_field_step_and_probe_equal_the_c_oracle(kappa_max):
    cfg = Cfg(kappa_max=kappa_max)
    rng = np.random.default_rng(3)
    nz, ny, nx = cfg.nz, cfg.ny, cfg.nx
    k0, k1 = cfg.design_k0, cfg.design_k1
    levels = np.array([0.25, 0.5, 0.75, 1.0])
    pick = rng.integers(0, 4, (k1 - k0, ny, nx))
    mask = levels[pick]
    material = np.zeros((nz, ny, nx), np.uint8)
    material[k0:k1] = pick + 1
    table = np.array([[0.0, 0.0, 1.0]] + [[WP * math.sqrt(m), GAMMA, 1.0] for m in levels])
    model = AO.FilmModel(cfg)
    beta, _ = model.drude(torch.tensor(mask.reshape(-1)), WP, GAMMA)
    # random state; held tangential E zero, J only on metal edges
    st = model.zero_state()
    eta0 = math.sqrt(MU0 / EPS0)
    fields = {}
    for c in range(3):
        e = rng.standard_normal((nz, ny, nx)) * model.upd[c].numpy()
        h = rng.standard_normal((nz, ny, nx)) / eta0
        j = rng.standard_normal((nz, ny, nx)) * 1e12 * (beta[c].numpy() > 0)
        fields[c] = (e, h, j)
        st["E"][c], st["H"][c], st["J"][c] = (torch.tensor(v) for v in (e, h, j))
    orc = O.Oracle(_W(cfg, material, table), eps0=EPS0, mu0=MU0)
    for c in range(3):
        e, h, j = fields[c]
        orc.set_field(O.E_X + c, e)
        orc.set_field(O.H_X + c, h)
        orc.set_field(O.JP_X + c, j)
    orc.probe_dft(np.array(cfg.probe), np.array([cfg.omega0 / (2 * math.pi)]), comp_mask=1 << cfg.probe_comp)
    nst = 5
    orc.step(nst)
    with torch.no_grad():
        Fr, Fi, st = model.run(torch.tensor(mask.reshape(-1)), WP, GAMMA, nsteps=nst, state=st, with_bunch=False)
    for c in range(3):
        for name, which in (("E", O.E_X), ("H", O.H_X), ("J", O.JP_X)):
            ref = orc.get_field(which + c)
            got = st[name][c].numpy()
            assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref), (name, c)
    F = orc.probe_read()[0, cfg.probe_comp, 0]
    assert abs(complex(float(Fr), float(Fi)) - F) <= 1e-13 * abs(F)


def test_bunch_current_integrates_to_qv_and_is_centred():
    """The prescribed current is the whole Gaussian: on a lattice of spacing
    dx = sigma/2 the lattice sums of a Gaussian equal its integrals up to
    terms of order exp(-2 pi^2 sigma^2/dx^2) ~ 1e-34 (Poisson summation), and
    the centre lies more than 7 sigma inside every face (tails below 1e-12),
    so the charge flux, centroid and variance match the closed forms to
    rounding.  A truncation at six rms radii (2e-8 of the charge) fails."""
    cfg = Cfg(nx=40, ny=36, nz=36, sigma=4e-9)
    cfg.bunch_x0, cfg.bunch_y0, cfg.bunch_z0 = 17.3 * cfg.dx, 17.6 * cfg.dx, 18.2 * cfg.dx
    model = AO.FilmModel(cfg)
    t = 7.5 * cfg.dt
    js = model.bunch(t).numpy()
    dV = cfg.dx ** 3
    total = js.sum() * dV
    assert total == pytest.approx(cfg.bunch_q * cfg.bunch_v, rel=1e-11)
    x = (np.arange(cfg.nx) + 0.5) * cfg.dx
    y = np.arange(cfg.ny) * cfg.dx
    z = np.arange(cfg.nz) * cfg.dx
    w = js / js.sum()
    assert (w.sum(axis=(0, 1)) * x).sum() == pytest.approx(cfg.bunch_x0 + cfg.bunch_v * t, abs=1e-10 * cfg.dx)
    assert (w.sum(axis=(0, 2)) * y).sum() == pytest.approx(cfg.bunch_y0, abs=1e-10 * cfg.dx)
    assert (w.sum(axis=(1, 2)) * z).sum() == pytest.approx(cfg.bunch_z0, abs=1e-10 * cfg.dx)
    # the second moment along each axis is sigma^2 (the normalisation's width)
    var_y = (w.sum(axis=(0, 2)) * (y - cfg.bunch_y0) ** 2).sum()
    var_x = (w.sum(axis=(0, 1)) * (x - cfg.bunch_x0 - cfg.bunch_v * t) ** 2).sum()
    assert var_y == pytest.approx(cfg.bunch_sigma ** 2, rel=1e-10)
    assert var_x == pytest.approx(cfg.bunch_sigma ** 2, rel=1e-10)
    # no cut: the current is positive (q v < 0 scaled) on every edge of the grid
    assert np.all(js * np.sign(cfg.bunch_q * cfg.bunch_v) > 0)


@pytest.fixture(scope="module")
def grad_case():
    cfg = Cfg()
    n = cfg.nx * cfg.ny * (cfg.design_k1 - cfg.design_k0)
    mask = np.random.default_rng(5).uniform(0.2, 0.8, n)
    return cfg, mask, AO.loss_and_grad(cfg, mask, WP, GAMMA)


def test_gradient_matches_central_differences(grad_case):
    cfg, mask, (L, dm, dw, dg) = grad_case
    assert L > 0 and np.isfinite(dm).all()
    cells = np.argsort(-np.abs(dm))[[0, 3, 17, 60]]
    for c in cells:
        h = 1e-4 * mask[c]
        mp, mm = mask.copy(), mask.copy()
        mp[c] += h
        mm[c] -= h
        fd = (AO.loss(cfg, mp, WP, GAMMA) - AO.loss(cfg, mm, WP, GAMMA)) / (2 * h)
        assert abs(fd - dm[c]) <= 1e-6 * np.abs(dm).max(), (c, fd, dm[c])
    for val, grad, f in ((WP, dw, lambda v: AO.loss(cfg, mask, v, GAMMA)),
                         (GAMMA, dg, lambda v: AO.loss(cfg, mask, WP, v))):
        h = 1e-4 * val
        fd = (f(val + h) - f(val - h)) / (2 * h)
        assert abs(fd - grad) <= 1e-6 * abs(grad), (fd, grad)


def test_without_metal_wp_and_gamma_do_not_matter():
    cfg = Cfg(nsteps=30)
    n = cfg.nx * cfg.ny * (cfg.design_k1 - cfg.design_k0)
    L, dm, dw, dg = AO.loss_and_grad(cfg, np.zeros(n), WP, GAMMA)
    assert L > 0
    assert dw == 0.0 and dg == 0.0
    assert np.abs(dm).max() > 0.0
