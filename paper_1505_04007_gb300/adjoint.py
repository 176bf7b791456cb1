"""Python binding of include/pic_adjoint.h (argument marshalling only) and a
torch.autograd.Function around it.

The gradient of the plasmon probe's spectral energy L = |F(omega0)|^2 with
respect to the per-cell Drude mask of a design slab, wp and gamma comes from
the library's hand-written adjoint (the transposed field step run backward
in time); nothing here differentiates anything.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import pic as _pic
from . import workloads as W

ADJ_EXPORTS = ("pic_adj_create", "pic_adj_mask_size", "pic_adj_forward", "pic_adj_backward", "pic_adj_destroy")


class pic_adj_config(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64), ("dx", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int32), ("cpml_cells", C.c_int32),
                ("cpml_order", C.c_double), ("cpml_sigma_fac", C.c_double), ("cpml_kappa_max", C.c_double),
                ("cpml_alpha_max", C.c_double), ("eps0", C.c_double), ("mu0", C.c_double),
                ("design_k0", C.c_int64), ("design_k1", C.c_int64),
                ("bunch_q", C.c_double), ("bunch_sigma", C.c_double), ("bunch_v", C.c_double),
                ("bunch_x0", C.c_double), ("bunch_y0", C.c_double), ("bunch_z0", C.c_double),
                ("probe", C.c_double * 3), ("probe_comp", C.c_int32), ("flags", C.c_int32),
                ("omega0", C.c_double), ("nsteps", C.c_int64)]


_bound = False


def load():
    global _bound
    L = _pic.load()
    if not _bound:
        h = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.pic_adj_create.argtypes = [C.POINTER(pic_adj_config), C.POINTER(h)]
        L.pic_adj_mask_size.argtypes = [h, C.POINTER(C.c_int64)]
        L.pic_adj_forward.argtypes = [h, dp, C.c_double, C.c_double, dp]
        L.pic_adj_backward.argtypes = [h, dp, dp, dp]
        L.pic_adj_destroy.argtypes = [h]
        _bound = True
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def pic_adj_create(cfg: pic_adj_config) -> C.c_void_p:
    out = C.c_void_p()
    _pic._check(load().pic_adj_create(C.byref(cfg), C.byref(out)), "pic_adj_create")
    return out


def pic_adj_mask_size(h) -> int:
    n = C.c_int64()
    _pic._check(load().pic_adj_mask_size(h, C.byref(n)), "pic_adj_mask_size")
    return n.value


def pic_adj_forward(h, mask, wp: float, gamma: float) -> float:
    m = np.ascontiguousarray(mask, dtype=np.float64)
    loss = C.c_double()
    _pic._check(load().pic_adj_forward(h, _dp(m), wp, gamma, C.byref(loss)), "pic_adj_forward")
    return loss.value


def pic_adj_backward(h, n: int):
    dm = np.empty(n)
    dwp, dga = C.c_double(), C.c_double()
    _pic._check(load().pic_adj_backward(h, _dp(dm), C.byref(dwp), C.byref(dga)), "pic_adj_backward")
    return dm, dwp.value, dga.value


def pic_adj_destroy(h) -> None:
    _pic._check(load().pic_adj_destroy(h), "pic_adj_destroy")


def film_config(nx=192, ny=96, nz=96, dx=2e-9, design=(16, 31), nsteps=4000, kev=40.0, sigma=6e-9, charge=1e-15,
                gap=10e-9, precision=_pic.PIC_FP32, cpml=8, wp_ref=W.TABLE1_WP):
    """The adjoint study of a film: a design slab of cell planes [design)
    (30 nm at the defaults), a rigid Gaussian electron bunch (kev, sigma,
    charge) moving +x `gap` above the slab top, a probe of Ez 5 nm above the
    slab top at 3/4 of x, loss frequency wp_ref/sqrt(2)."""
    c = pic_adj_config()
    c.nx, c.ny, c.nz, c.dx = nx, ny, nz, dx
    c.dt = W.yee_dt(dx, dx, dx)
    c.precision = precision
    c.cpml_cells = cpml
    c.cpml_order, c.cpml_sigma_fac, c.cpml_kappa_max = 3.0, 0.8, 1.0
    c.cpml_alpha_max = 0.05 * W.EPS0 * wp_ref
    c.eps0, c.mu0 = W.EPS0, W.MU0
    c.design_k0, c.design_k1 = design
    top = design[1] * dx
    c.bunch_q = -charge
    c.bunch_sigma = sigma
    c.bunch_v = W.electron_momentum(kev) / np.sqrt(1 + (W.electron_momentum(kev) / W.C0) ** 2)
    c.bunch_x0 = (cpml + 2) * dx + 3 * sigma
    c.bunch_y0 = 0.5 * ny * dx
    c.bunch_z0 = top + gap
    c.probe[0], c.probe[1], c.probe[2] = 0.75 * nx * dx, 0.5 * ny * dx, top + 5e-9
    c.probe_comp = 2
    c.omega0 = wp_ref / np.sqrt(2.0)
    c.nsteps = nsteps
    return c


class Adjoint:
    """One adjoint study (a pic_adj handle) for a configuration."""

    def __init__(self, cfg: pic_adj_config):
        self.cfg = cfg
        self.h = pic_adj_create(cfg)
        self.n = pic_adj_mask_size(self.h)

    def forward(self, mask, wp, gamma) -> float:
        return pic_adj_forward(self.h, mask, wp, gamma)

    def backward(self):
        return pic_adj_backward(self.h, self.n)

    def close(self):
        if getattr(self, "h", None):
            pic_adj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plasmon_loss(study: Adjoint):
    """torch.autograd.Function for this study: f(mask, wp, gamma) -> L, with
    the backward pass taken from the library's adjoint (FP64 tensors)."""
    import torch

    class _PlasmonLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, mask, wp, gamma):
            loss = study.forward(mask.detach().cpu().double().numpy(), float(wp), float(gamma))
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            dm, dwp, dga = study.backward()
            g = float(g)
            return (torch.from_numpy(dm * g), torch.tensor(dwp * g, dtype=torch.float64),
                    torch.tensor(dga * g, dtype=torch.float64))

    return _PlasmonLoss.apply
