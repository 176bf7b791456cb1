"""Seeded synthetic inputs for the PIC/FDTD-Drude time step.

This module builds the inputs that both the CUDA library and the FP64 CPU
oracle consume: grid sizes, time step, the per-cell material map with its
Drude table, the electron bunch (positions and momenta), the probe points and
the DFT frequency grid.  It holds none of the method's arithmetic (no field
update, push, deposit or transform); it only draws and lays out inputs.

The workloads stand in for the paper's setup (Sec. III: an electron bunch
moving parallel to a silver film, Drude parameters per cell, absorbing
boundaries, an E-field probe above the film whose spectrum shows the surface
plasmon modes).  The paper gives no grid, time step or particle count, so the
sizes below are the three single-instance workloads the project benchmarks:

* ``c1`` 128x32x48 cells, dx=2 nm, 1000 steps, 20 nm film, 4096 electrons
  at 30 keV, one probe (FP64 parity size).
* ``c2`` 384x128x128 cells, dx=2 nm, 8000 steps, 40 nm film, 1e5 electrons
  at 50 keV, a line of 64 probes (paper-scale run, the timed workload).
* ``c3`` 768x256x256 cells, dx=1 nm, 12000 steps, 10 nm film, 1e6 electrons
  at 30 keV, one probe (streaming-limit size).
* ``sweep`` 48 independent instances on uneven grids (128..320 x 64..128 x
  64..96 cells), films 10-60 nm, 10-100 keV, gaps 5-20 nm, 2e4 electrons
  each, 4000 steps (batched stepping).

Positions come from ``numpy.random.default_rng(seed)`` (PCG64) with a fixed
rejection order, so every consumer sees identical arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 constants, passed verbatim to both implementations.
C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
QE = 1.602176634e-19
ME = 9.1093837015e-31
MEC2_KEV = 510.99895

# Boundary codes per face (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi).
BC_CPML, BC_PEC, BC_PERIODIC = 0, 1, 2

# Silver Drude parameters used by the workloads (rad/s, 1/s).
AG_WP = 1.37e16
AG_GAMMA = 3.2e13

# The particle margin: non-periodic axes keep electrons this many cells away
# from the outer faces (the freeze rule uses the same number).
MARGIN_CELLS = 2


@dataclasses.dataclass
class Workload:
    """Everything one simulation instance needs, in SI units.

    ``material`` is uint8 [nz][ny][nx] (x fastest); ``table`` is float64
    [n_materials][3] holding (wp [rad/s], gamma [1/s], eps_inf) per id.
    ``xyz`` and ``u`` are float64 [n][3] (metres and gamma*v in m/s).
    """
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    dt: float
    nsteps: int
    bc: tuple = (BC_CPML,) * 6
    cpml_cells: int = 8
    cpml_order: float = 3.0
    cpml_sigma_fac: float = 0.8
    cpml_kappa_max: float = 1.0
    cpml_alpha_max: float = 0.0
    material: np.ndarray = None
    table: np.ndarray = None
    xyz: np.ndarray = None
    u: np.ndarray = None
    q_macro: float = 0.0
    m_macro: float = 0.0
    probes: np.ndarray = None
    comp_mask: int = 0b111
    freqs: np.ndarray = None
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nparticles(self) -> int:
        return 0 if self.xyz is None else int(self.xyz.shape[0])


def yee_dt(dx: float, dy: float, dz: float, courant: float = 0.5) -> float:
    """dt = courant * dx / (c*sqrt(3)) for a cubic grid (general form
    courant / (c*sqrt(1/dx^2+1/dy^2+1/dz^2)))."""
    return courant / (C0 * math.sqrt(1.0 / dx**2 + 1.0 / dy**2 + 1.0 / dz**2))


def electron_momentum(kinetic_kev: float) -> float:
    """gamma*v [m/s] of an electron of the given kinetic energy."""
    g = 1.0 + kinetic_kev / MEC2_KEV
    beta = math.sqrt(1.0 - 1.0 / (g * g))
    return g * beta * C0


def slab_material(nx: int, ny: int, nz: int, k0: int, k1: int) -> np.ndarray:
    """uint8 map with id 1 in cell planes k0..k1-1 (a film spanning x and y)."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[k0:k1] = 1
    return m


def drude_table(wp: float = AG_WP, gamma: float = AG_GAMMA, eps_inf: float = 1.0) -> np.ndarray:
    return np.array([[0.0, 0.0, 1.0], [wp, gamma, eps_inf]], dtype=np.float64)


def allowed(w: Workload, pts: np.ndarray) -> np.ndarray:
    """Mask of positions an electron may occupy: inside the margin on every
    non-periodic axis and not in a cell whose material has wp > 0."""
    n = (w.nx, w.ny, w.nz)
    d = (w.dx, w.dy, w.dz)
    ok = np.ones(pts.shape[0], dtype=bool)
    cells = []
    for a in range(3):
        xi = pts[:, a] / d[a]
        periodic = w.bc[2 * a] == BC_PERIODIC
        if periodic:
            xi = np.mod(xi, n[a])
        else:
            ok &= (xi >= MARGIN_CELLS) & (xi < n[a] - MARGIN_CELLS)
        cells.append(np.clip(np.floor(xi).astype(np.int64), 0, n[a] - 1))
    metal = w.table[w.material[cells[2], cells[1], cells[0]], 0] > 0.0
    return ok & ~metal


def gaussian_bunch(w: Workload, n: int, centre, sigma, seed: int = 1505) -> np.ndarray:
    """n positions drawn from an isotropic Gaussian, rejected points redrawn
    in batches (fixed order: draw, keep allowed, repeat) until n are kept."""
    rng = np.random.default_rng(seed)
    centre = np.asarray(centre, dtype=np.float64)
    out = np.empty((0, 3))
    drawn = 0
    while out.shape[0] < n:
        need = n - out.shape[0]
        pts = centre + sigma * rng.standard_normal((need, 3))
        drawn += need
        out = np.concatenate([out, pts[allowed(w, pts)]], axis=0)
    w.info["bunch_drawn"] = drawn
    w.info["bunch_rejected_fraction"] = 1.0 - n / drawn
    return out[:n]


def freq_grid(f0: float = 0.5e15, f1: float = 2.5e15, df: float = 1.0e12) -> np.ndarray:
    nf = int(round((f1 - f0) / df)) + 1
    return f0 + df * np.arange(nf, dtype=np.float64)


def _bunch_workload(name, nx, ny, nz, dx, nsteps, film_k0, film_k1, npart, charge, kev,
                    centre, sigma, probes, seed=1505, nfreq_step=1.0e12):
    w = Workload(name=name, nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dx,
                 dt=yee_dt(dx, dx, dx), nsteps=nsteps)
    w.cpml_alpha_max = 0.05 * EPS0 * AG_WP
    w.material = slab_material(nx, ny, nz, film_k0, film_k1)
    w.table = drude_table()
    w.q_macro = -charge / max(npart, 1)
    w.m_macro = ME * (charge / max(npart, 1)) / QE
    if npart:
        w.xyz = gaussian_bunch(w, npart, centre, sigma, seed=seed)
        w.u = np.zeros_like(w.xyz)
        w.u[:, 0] = electron_momentum(kev)
    w.probes = np.asarray(probes, dtype=np.float64).reshape(-1, 3)
    w.freqs = freq_grid(df=nfreq_step)
    w.info.update(film_cells=(film_k0, film_k1), kev=kev, charge=charge)
    return w


def c1(seed: int = 1505, nsteps: int = 1000) -> Workload:
    """128x32x48, dx=2 nm, 20 nm film at cell planes 8..17, 4096 electrons,
    sigma 5 nm, 1 fC, 30 keV along +x, centred 10 nm above the film top at
    x=20 nm; one probe 5 nm above the top, 3/4 of the way along the interior."""
    dx = 2e-9
    nx, ny, nz = 128, 32, 48
    top = 18 * dx
    L = 8
    probe = [(L + 0.75 * (nx - 2 * L)) * dx, 0.5 * ny * dx, top + 5e-9]
    return _bunch_workload("c1", nx, ny, nz, dx, nsteps, 8, 18, 4096, 1e-15, 30.0,
                           (20e-9, 0.5 * ny * dx, top + 10e-9), 5e-9, [probe], seed)


def c2(seed: int = 1505, nsteps: int = 8000, nparticles: int = 100000) -> Workload:
    """384x128x128, dx=2 nm, 40 nm film at cell planes 8..27, 1e5 electrons,
    sigma 8 nm, 1 fC, 50 keV, 15 nm above the top, x centre 44 nm; a line of
    64 probes 5 nm above the top along x."""
    dx = 2e-9
    nx, ny, nz = 384, 128, 128
    top = 28 * dx
    L = 8
    lo, length = L * dx, (nx - 2 * L) * dx
    probes = [[lo + (p + 0.5) * length / 64, 0.5 * ny * dx, top + 5e-9] for p in range(64)]
    return _bunch_workload("c2", nx, ny, nz, dx, nsteps, 8, 28, nparticles, 1e-15, 50.0,
                           (44e-9, 0.5 * ny * dx, top + 15e-9), 8e-9, probes, seed)


def c3(seed: int = 1505, nsteps: int = 12000, nparticles: int = 1000000) -> Workload:
    """768x256x256, dx=1 nm, 10 nm film at cell planes 8..17, 1e6 electrons,
    sigma 5 nm, 2 fC, 30 keV, 5 nm above the top, x centre 25 nm; one probe."""
    dx = 1e-9
    nx, ny, nz = 768, 256, 256
    top = 18 * dx
    L = 8
    probe = [(L + 0.75 * (nx - 2 * L)) * dx, 0.5 * ny * dx, top + 5e-9]
    return _bunch_workload("c3", nx, ny, nz, dx, nsteps, 8, 18, nparticles, 2e-15, 30.0,
                           (25e-9, 0.5 * ny * dx, top + 5e-9), 5e-9, [probe], seed)


def sweep(n: int = 48, seed: int = 1505, nsteps: int = 4000, nparticles: int = 20000,
          sizes: tuple = ((128, 320), (64, 128), (64, 96))) -> list:
    """A sweep of n independent film instances for batched stepping: silver
    films 10-60 nm thick (uniform), electrons of 10-100 keV (log-uniform),
    bunch centres 5-20 nm above the film (uniform), grids of uneven sizes in
    the given (lo, hi) cell ranges per axis (x a multiple of 32, y and z of
    16; z raised where the film, gap and bunch need it), dx = 2 nm, 1 fC and
    `nparticles` electrons per bunch (sigma 5 nm), one probe 5 nm above the
    film top.  Draws come from one PCG64 stream in a fixed order per
    instance: nx, ny, nz, thickness, energy, gap; instance i's bunch uses
    seed + 1 + i."""
    rng = np.random.default_rng(seed)
    dx = 2e-9
    L = 8
    sigma = 5e-9
    out = []
    for i in range(n):
        nx = 32 * int(rng.integers(sizes[0][0] // 32, sizes[0][1] // 32 + 1))
        ny = 16 * int(rng.integers(sizes[1][0] // 16, sizes[1][1] // 16 + 1))
        nz = 16 * int(rng.integers(sizes[2][0] // 16, sizes[2][1] // 16 + 1))
        d = rng.uniform(10e-9, 60e-9)
        kev = float(np.exp(rng.uniform(np.log(10.0), np.log(100.0))))
        gap = rng.uniform(5e-9, 20e-9)
        k0 = L
        k1 = k0 + max(1, int(round(d / dx)))
        top = k1 * dx
        need = int(np.ceil((top + gap + 3 * sigma) / dx)) + MARGIN_CELLS + 1 + L
        nz = max(nz, 16 * ((need + 15) // 16))
        probe = [(L + 0.75 * (nx - 2 * L)) * dx, 0.5 * ny * dx, top + 5e-9]
        centre = ((L + MARGIN_CELLS) * dx + 3 * sigma, 0.5 * ny * dx, top + gap)
        w = _bunch_workload(f"sweep{i:02d}", nx, ny, nz, dx, nsteps, k0, k1, nparticles, 1e-15, kev,
                            centre, sigma, [probe], seed + 1 + i)
        w.info.update(thickness=d, gap=gap)
        out.append(w)
    return out


# The paper's film model for its mode study (Sec. IV, Table 1): silver with
# these Drude parameters, a 100 keV bunch, films 20-150 nm thick.
TABLE1_WP = 1.2e16
TABLE1_GAMMA = 1.45e13
TABLE1_KEV = 100.0
TABLE1_THICKNESS_NM = (20, 30, 40, 50, 60, 70, 80, 150)


def film_plasmon(thick_cells: int, nsteps: int, nx: int = 256, npart: int = 1024, charge: float = 1e-18,
                 wp: float = TABLE1_WP, gamma: float = TABLE1_GAMMA, kev: float = TABLE1_KEV, seed: int = 5,
                 freqs=None, comp_mask: int = 0b101, below: int = 0) -> Workload:
    """Quasi-2D version of the paper's film model (Sec. III-IV): a silver film
    of thick_cells x 2 nm, `below` vacuum cells above the z-low CPML (0: on
    it), periodic in y (2 cells), and a sheet of electrons at kev moving +x
    20 nm above it (small total charge: linear response, no Coulomb
    explosion); one probe 5 nm above the film at 3/4 of the x extent."""
    dx = 2e-9
    k0 = 8 + below
    k1 = k0 + thick_cells
    ny = 2
    nz = k1 + 32 + 8
    w = Workload(name=f"film{2 * thick_cells}nm", nx=nx, ny=ny, nz=nz, dx=dx, dy=dx, dz=dx,
                 dt=yee_dt(dx, dx, dx), nsteps=nsteps,
                 bc=(BC_CPML, BC_CPML, BC_PERIODIC, BC_PERIODIC, BC_CPML, BC_CPML))
    w.cpml_alpha_max = 0.05 * EPS0 * wp
    w.material = slab_material(nx, ny, nz, k0, k1)
    w.table = np.array([[0.0, 0.0, 1.0], [wp, gamma, 1.0]])
    rng = np.random.default_rng(seed)
    x = rng.normal(30 * dx, 8 * dx, npart)
    y = rng.uniform(0, ny * dx, npart)
    z = rng.normal((k1 + 10) * dx, 1.0 * dx, npart)
    w.xyz = np.stack([x, y, z], 1)
    w.u = np.zeros_like(w.xyz)
    w.u[:, 0] = electron_momentum(kev)
    w.q_macro = -charge / max(npart, 1)
    w.m_macro = ME * (charge / max(npart, 1)) / QE
    w.probes = np.array([[0.75 * nx * dx, 0.5 * ny * dx, k1 * dx + 5e-9]])
    w.freqs = np.arange(1.0e15, 1.5e15, 1e12) if freqs is None else np.asarray(freqs, np.float64)
    w.comp_mask = comp_mask
    w.info.update(film_cells=(k0, k1), kev=kev, wp=wp, thickness=thick_cells * dx)
    return w


def film_line(thick_cells: int, nsteps: int, nx: int = 1024, nprobes: int = 64, first: int = 200,
              spacing: int = 11, below: int = 24, freqs=None) -> Workload:
    """A free film (film_plasmon geometry, no electrons) with a line of
    nprobes probes along x, 5 nm above the film, from cell `first` every
    `spacing` cells: the input of the k-omega readout (Fig. 2 analogue).  The
    excitation is left to the caller (a prescribed source pulse)."""
    fq = np.arange(0.5e15, 1.7e15 + 0.5e12, 2e12) if freqs is None else freqs
    w = film_plasmon(thick_cells, nsteps, nx=nx, npart=0, freqs=fq, comp_mask=0b100, below=below)
    w.xyz = np.zeros((0, 3))
    w.u = np.zeros((0, 3))
    top = w.info["film_cells"][1] * w.dx
    w.probes = np.array([[(first + spacing * p) * w.dx, 0.5 * w.ny * w.dx, top + 5e-9] for p in range(nprobes)])
    w.name = f"film_line{2 * thick_cells}nm"
    return w


def table1(nsteps: int, nx: int = 2048, below: int = 24) -> list:
    """The paper's thickness series: one film_plasmon instance per thickness
    of TABLE1_THICKNESS_NM, Ez probed from 0.7 to 1.6 PHz in 1 THz steps.
    The film is a free film in vacuum (the theory the paper compares with
    has vacuum on both sides): `below` vacuum cells separate it from the
    z-low CPML, which also keeps the Drude metal away from the absorbing
    layer (with the metal on the CPML the late-time fields grow)."""
    freqs = np.arange(0.7e15, 1.6e15 + 0.5e12, 1e12)
    return [film_plasmon(d // 2, nsteps, nx=nx, freqs=freqs, comp_mask=0b100, below=below)
            for d in TABLE1_THICKNESS_NM]


def scaled(w: Workload, nx: int, ny: int, nz: int, nparticles: int, nsteps: int,
           seed: int = 1505) -> Workload:
    """A smaller instance with the same film planes, bunch recipe and probe
    rule as ``w`` (used for parity cases the oracle finishes in seconds)."""
    k0, k1 = w.info["film_cells"]
    dx = w.dx
    top = k1 * dx
    L = w.cpml_cells
    gap = (w.info.get("gap", None) or (10e-9 if w.name == "c1" else 5e-9))
    probe = [(L + 0.75 * (nx - 2 * L)) * dx, 0.5 * ny * dx, top + 5e-9]
    return _bunch_workload(w.name + "_scaled", nx, ny, nz, dx, nsteps, k0, k1, nparticles,
                           w.info["charge"], w.info["kev"],
                           ((L + 4) * dx, 0.5 * ny * dx, top + gap), 5e-9, [probe], seed)


WORKLOADS = {"c1": c1, "c2": c2, "c3": c3}
