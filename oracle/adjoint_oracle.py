"""FP64 CPU oracle of the film design study: the forward model behind the
gradient API and its gradient with respect to the per-cell Drude mask, wp and
gamma.

TEST INFRASTRUCTURE ONLY: tests may import this module; the CUDA library
never does, and nothing here calls it.

Forward model, one step n -> n+1 on the Yee grid (plain PyTorch CPU ops in
float64, every array full size [nz][ny][nx], x fastest):
  H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n              (Sec. II; CPML on all faces)
  J^{n+1}   = kJ J^n + bJ E^n                          (Eq. 6, E at level n)
  E^{n+1}   = E^n + dt/eps0 [curl H^{n+1/2} - J^{n+1} - Js^{n+1/2}]   (Eq. 8)
with kJ = (2 - gamma dt)/(2 + gamma dt), bJ = 2 dt eps0 wp_e^2/(2 + gamma dt)
(the coefficients of Eq. 6), wp_e^2 = wp^2 times the mean of the mask over
the four cells around the edge (cells below a face clamped to the face; the
mask is zero outside the design slab), eps_inf = 1.  Tangential E on the six
faces stays zero, E beyond a high face reads as zero.  Js is the current of a
rigid Gaussian bunch moving along +x, on every Ex edge (not truncated):
  Js_x = q v (2 pi s^2)^{-3/2} exp(-r^2 / (2 s^2)),  r measured from
  (x0 + v t, y0, z0) to the Ex edge, t = (n + 1/2) dt.
Loss L = |F|^2 with F = sum_n E_c(x_p, (n+1) dt) exp(+i w0 (n+1) dt) dt, E_c
interpolated trilinearly on its own staggered lattice (the probe DFT at one
frequency).

CPML (Roden-Gedney) as the main oracle: depth rho in cells, sigma =
sigma_fac (m+1)/(eta0 dx) (rho/L)^m, kappa = 1 + (kappa_max-1)(rho/L)^m,
alpha = alpha_max (1 - rho/L), b = exp(-(sigma/kappa + alpha) dt/eps0),
a = sigma (b-1)/(sigma kappa + kappa^2 alpha); psi <- b psi + a dF and the
curl uses dF/kappa + psi.

The gradient is reverse-mode differentiation of this forward model
(torch.autograd); no transposed step is written by hand here.  The forward
step is pinned to the C oracle's field step, and the gradient to central
differences of the forward model.

The configuration is duck-typed: any object with the fields of
pic_adj_config (nx, ny, nz, dx, dt, cpml_cells, cpml_order, cpml_sigma_fac,
cpml_kappa_max, cpml_alpha_max, eps0, mu0, design_k0, design_k1, bunch_q,
bunch_sigma, bunch_v, bunch_x0, bunch_y0, bunch_z0, probe[3], probe_comp,
omega0, nsteps).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64


def cpml_profile(n, L, order, sigma_fac, kappa_max, alpha_max, dx, dt, eps0, mu0, shift):
    """(b, a, 1/kappa) at positions x + shift, x = 0..n-1 (cell units), for
    absorbing slabs of L cells on both faces of an axis of n cells."""
    b = np.ones(n)
    a = np.zeros(n)
    ik = np.ones(n)
    eta0 = math.sqrt(mu0 / eps0)
    for x in range(n):
        pos = x + shift
        rho = 0.0
        if pos < L:
            rho = L - pos
        if pos > n - L:
            rho = max(rho, pos - (n - L))
        if rho <= 0.0:
            continue
        r = rho / L
        sigma = sigma_fac * (order + 1.0) / (eta0 * dx) * r ** order
        kappa = 1.0 + (kappa_max - 1.0) * r ** order
        alpha = alpha_max * (1.0 - r)
        bb = math.exp(-(sigma / kappa + alpha) * dt / eps0)
        den = sigma * kappa + kappa * kappa * alpha
        b[x] = bb
        a[x] = sigma * (bb - 1.0) / den if (sigma > 0.0 and den > 0.0) else 0.0
        ik[x] = 1.0 / kappa
    return b, a, ik


def _dim(axis):
    """Array dimension of grid axis 0=x, 1=y, 2=z in a [nz][ny][nx] array."""
    return 2 - axis


def _next(X, axis):
    """X at index + 1 along the axis; zero beyond the high face."""
    d = _dim(axis)
    zero = torch.zeros_like(X.narrow(d, 0, 1))
    return torch.cat([X.narrow(d, 1, X.shape[d] - 1), zero], dim=d)


def _prev(X, axis):
    """X at index - 1 along the axis; index 0 reads itself (clamped)."""
    d = _dim(axis)
    return torch.cat([X.narrow(d, 0, 1), X.narrow(d, 0, X.shape[d] - 1)], dim=d)


class FilmModel:
    """The forward model of one configuration (see the module docstring)."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.n = (int(cfg.nx), int(cfg.ny), int(cfg.nz))
        self.shape = (self.n[2], self.n[1], self.n[0])
        L = int(cfg.cpml_cells)
        args = (L, cfg.cpml_order, cfg.cpml_sigma_fac, cfg.cpml_kappa_max, cfg.cpml_alpha_max,
                cfg.dx, cfg.dt, cfg.eps0, cfg.mu0)
        self.prof = {}
        for a in range(3):
            for field, shift in (("E", 0.0), ("H", 0.5)):
                b, aa, ik = cpml_profile(self.n[a], *args, shift)
                view = [1, 1, 1]
                view[_dim(a)] = self.n[a]
                self.prof[field, a] = tuple(torch.tensor(v, dtype=F64).reshape(view) for v in (b, aa, ik))
        nz, ny, nx = self.shape
        k = torch.arange(nz, dtype=F64).reshape(nz, 1, 1)
        j = torch.arange(ny, dtype=F64).reshape(1, ny, 1)
        i = torch.arange(nx, dtype=F64).reshape(1, 1, nx)
        # updated (not held) edges of each component
        self.upd = ((j > 0) & (k > 0)).expand(self.shape), ((i > 0) & (k > 0)).expand(self.shape), \
                   ((i > 0) & (j > 0)).expand(self.shape)
        self.ijk = (i, j, k)
        # probe: trilinear weights on the component's staggered lattice
        c = int(cfg.probe_comp)
        self.pidx, self.pw = [], []
        for corner in range(8):
            idx, w = [], 1.0
            for a in range(3):
                s = cfg.probe[a] / cfg.dx - (0.5 if a == c else 0.0)
                fl = math.floor(s)
                bit = (corner >> a) & 1
                idx.append(min(max(int(fl) + bit, 0), self.n[a] - 1))
                w *= (s - fl) if bit else 1.0 - (s - fl)
            self.pidx.append((idx[2], idx[1], idx[0]))
            self.pw.append(w)

    def zero_state(self):
        z = lambda: torch.zeros(self.shape, dtype=F64)  # noqa: E731
        return {"E": [z() for _ in range(3)], "H": [z() for _ in range(3)], "J": [z() for _ in range(3)],
                "psiE": [[z(), z()] for _ in range(3)], "psiH": [[z(), z()] for _ in range(3)]}

    def cell_mask(self, mask):
        """The mask on the full grid of cells (zero outside the design slab)."""
        cfg = self.cfg
        nz, ny, nx = self.shape
        k0, k1 = int(cfg.design_k0), int(cfg.design_k1)
        m = mask.reshape(k1 - k0, ny, nx)
        return torch.cat([torch.zeros(k0, ny, nx, dtype=F64), m, torch.zeros(nz - k1, ny, nx, dtype=F64)], dim=0)

    def edge_mean(self, M, comp):
        """Mean of the cell values M over the four cells sharing each edge of
        the component (offsets -1, 0 along the two transverse axes)."""
        a1, a2 = (comp + 1) % 3, (comp + 2) % 3
        return 0.25 * (M + _prev(M, a1) + _prev(M, a2) + _prev(_prev(M, a1), a2))

    def drude(self, mask, wp, gamma):
        """(bJ per component, kJ) of Eq. 6."""
        cfg = self.cfg
        dt = cfg.dt
        M = self.cell_mask(mask)
        den = 2.0 + gamma * dt
        beta = [2.0 * dt * cfg.eps0 * wp * wp * self.edge_mean(M, c) / den for c in range(3)]
        kJ = (2.0 - gamma * dt) / den
        return beta, kJ

    def bunch(self, t):
        """Js_x on the Ex edges at time t."""
        cfg = self.cfg
        i, j, k = self.ijk
        s = cfg.bunch_sigma
        x = (i + 0.5) * cfg.dx - (cfg.bunch_x0 + cfg.bunch_v * t)
        y = j * cfg.dx - cfg.bunch_y0
        z = k * cfg.dx - cfg.bunch_z0
        r2 = x * x + y * y + z * z
        amp = cfg.bunch_q * cfg.bunch_v / (2.0 * math.pi * s * s) ** 1.5
        return amp * torch.exp(-r2 / (2.0 * s * s))

    def step_H(self, st):
        cfg = self.cfg
        E, H, P = st["E"], st["H"], st["psiH"]
        r = 1.0 / cfg.dx
        cH = cfg.dt / cfg.mu0
        # dF[(field comp, derivative axis)]: forward differences of E
        dF = {}
        for c in range(3):
            for a in range(3):
                if a != c:
                    dF[c, a] = (_next(E[c], a) - E[c]) * r
        # Hx: +dEz/dy - dEy/dz ; Hy: +dEx/dz - dEz/dx ; Hz: +dEy/dx - dEx/dy
        for c in range(3):
            a1, a2 = (c + 1) % 3, (c + 2) % 3
            b1, aa1, ik1 = self.prof["H", a1]
            b2, aa2, ik2 = self.prof["H", a2]
            d1 = dF[a2, a1]  # derivative along a1 of E_{a2}
            d2 = dF[a1, a2]  # derivative along a2 of E_{a1}
            P[c][0] = b1 * P[c][0] + aa1 * d1
            P[c][1] = b2 * P[c][1] + aa2 * d2
            curl = ik1 * d1 + P[c][0] - ik2 * d2 - P[c][1]
            H[c] = H[c] - cH * curl

    def step_E(self, st, beta, kJ, js):
        cfg = self.cfg
        E, H, J, P = st["E"], st["H"], st["J"], st["psiE"]
        r = 1.0 / cfg.dx
        cE = cfg.dt / cfg.eps0
        # Ex: +dHz/dy - dHy/dz ; Ey: +dHx/dz - dHz/dx ; Ez: +dHy/dx - dHx/dy
        for c in range(3):
            a1, a2 = (c + 1) % 3, (c + 2) % 3
            b1, aa1, ik1 = self.prof["E", a1]
            b2, aa2, ik2 = self.prof["E", a2]
            d1 = (H[a2] - _prev(H[a2], a1)) * r
            d2 = (H[a1] - _prev(H[a1], a2)) * r
            u = self.upd[c]
            p1 = b1 * P[c][0] + aa1 * d1
            p2 = b2 * P[c][1] + aa2 * d2
            curl = ik1 * d1 + p1 - ik2 * d2 - p2
            Jn = kJ * J[c] + beta[c] * E[c]
            En = E[c] + cE * (curl - Jn - (js if c == 0 else 0.0))
            P[c][0] = torch.where(u, p1, P[c][0])
            P[c][1] = torch.where(u, p2, P[c][1])
            J[c] = torch.where(u, Jn, J[c])
            E[c] = torch.where(u, En, E[c])

    def probe(self, E):
        c = int(self.cfg.probe_comp)
        v = 0.0
        for (k, j, i), w in zip(self.pidx, self.pw):
            v = v + w * E[c][k, j, i]
        return v

    def run(self, mask, wp, gamma, nsteps=None, state=None, with_bunch=True, n0=0):
        """Step from `state` (zero fields by default) for nsteps (the
        configuration's by default), starting at step index n0.  Returns
        (Re F, Im F, state)."""
        cfg = self.cfg
        nsteps = int(cfg.nsteps) if nsteps is None else int(nsteps)
        st = self.zero_state() if state is None else state
        beta, kJ = self.drude(mask, wp, gamma)
        dt, w0 = cfg.dt, cfg.omega0
        Fr = torch.zeros((), dtype=F64)
        Fi = torch.zeros((), dtype=F64)
        for n in range(n0, n0 + nsteps):
            self.step_H(st)
            js = self.bunch((n + 0.5) * dt) if with_bunch else 0.0
            self.step_E(st, beta, kJ, js)
            t = (n + 1) * dt
            v = self.probe(st["E"])
            Fr = Fr + v * math.cos(w0 * t) * dt
            Fi = Fi + v * math.sin(w0 * t) * dt
        return Fr, Fi, st


def loss(cfg, mask, wp, gamma):
    """L = |F|^2 of the forward model from zero fields (float)."""
    model = FilmModel(cfg)
    with torch.no_grad():
        Fr, Fi, _ = model.run(torch.as_tensor(np.asarray(mask, np.float64)), float(wp), float(gamma))
    return float(Fr * Fr + Fi * Fi)


def loss_and_grad(cfg, mask, wp, gamma):
    """(L, dL/dmask, dL/dwp, dL/dgamma) by reverse-mode differentiation of the
    forward model (mask ordered [k][j][i] over the design slab)."""
    model = FilmModel(cfg)
    m = torch.tensor(np.asarray(mask, np.float64), requires_grad=True)
    w = torch.tensor(float(wp), dtype=F64, requires_grad=True)
    g = torch.tensor(float(gamma), dtype=F64, requires_grad=True)
    Fr, Fi, _ = model.run(m, w, g)
    L = Fr * Fr + Fi * Fi
    dm, dw, dg = torch.autograd.grad(L, [m, w, g])
    return float(L.detach()), dm.numpy().copy(), float(dw), float(dg)
