"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an exact discrete identity, or a textbook definition computed here from
scratch.  A plausible slip in the oracle (a dropped term, a wrong sign or
time level, a transposed index) breaks at least one of them:

* Drude ADE + Ampere (Eqs. 6, 8): the uniform plasma oscillation obeys the
  discrete dispersion relation Omega (Omega + i gamma cos(w dt/2)) = wp^2,
  Omega = (2/dt) sin(w dt/2); its continuum limit is Eq. 1 (eps(w) = 0).
* Yee curls + Drude + Ampere: with gamma = 0 the discrete energy changes
  only by the work of the free current (exact to round-off).
* Deposit + E update: Gauss's law residual stays constant (discrete
  continuity), per particle and for the whole step.
* Boris: exact |u| in pure B, rotation angle 2 atan|t|, exact impulse in
  pure E, E x B drift.
* CPML: reflection below -40 dB against a larger domain.
* Probe DFT: equals the direct sum of the recorded probe series, and the
  closed-form geometric series of the plasma oscillation.
* Bulk Drude permittivity (Eq. 1) recovered from a plane wave in a metal:
  the two-probe ratio gives the numerical wavenumber, and
  eps = (c K/Omega)^2 must equal the discrete Drude-Yee permittivity
  1 - wp^2/(Omega(Omega + i gamma cos(w dt/2))) and, to O((w dt)^2), Eq. 1.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04007_gb300 import workloads as W

from _helpers import box_workload, cic_charge, edge_wp2, interior_node_mask, node_divergence

WP, GAM = W.AG_WP, W.AG_GAMMA


# ----------------------------------------------------------- Eqs. 6 and 8 --
def _plasma_series(gamma, nsteps=300, eps_inf=1.0):
    w = box_workload(4, 4, 4, bc=(W.BC_PERIODIC,) * 6,
                     material=np.ones((4, 4, 4), np.uint8),
                     table=[[0, 0, 1], [WP, gamma, eps_inf]])
    o = O.Oracle(w)
    o.set_field(O.E_X, np.full((4, 4, 4), 1.0e6))
    e = [1.0e6]
    j = [0.0]
    for _ in range(nsteps):
        o.step(1)
        ex = o.get_field(O.E_X)
        assert np.ptp(ex) == 0.0  # stays uniform: the curl of a uniform field is zero
        e.append(ex[0, 0, 0])
        j.append(o.get_field(O.JP_X)[0, 0, 0])
    return w, np.array(e), np.array(j), o


def _two_root_fit(e):
    # e[n+1] = a e[n] + b e[n-1]: exact for a two-state linear recurrence
    A = np.stack([e[1:-1], e[:-2]], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, e[2:], rcond=None)
    resid = np.abs(A @ np.array([a, b]) - e[2:]).max() / np.abs(e).max()
    z = np.roots([1.0, -a, -b])
    return z, resid


@pytest.mark.parametrize("gamma", [0.0, GAM, 40 * GAM])
def test_plasma_oscillation_discrete_dispersion(gamma):
    w, e, _, _ = _plasma_series(gamma)
    z, resid = _two_root_fit(e)
    assert resid < 1e-12, "E^n is not a two-state recurrence (wrong time level in Eq. 6?)"
    dt = w.dt
    # z = exp(-i w dt) with the paper's convention i w = -d/dt (Eq. 3 -> Eq. 4)
    for zz in z:
        om = 1j * np.log(zz) / dt
        if om.real < 0:
            continue
        Om = 2.0 / dt * np.sin(om * dt / 2)
        res = Om * (Om + 1j * gamma * np.cos(om * dt / 2)) - WP**2
        assert abs(res) / WP**2 < 1e-9
        # continuum limit (Eq. 1, eps(w) = 0): w^2 + i gamma w = wp^2
        cont = math.sqrt(WP**2 - gamma**2 / 4)
        assert abs(om.real / cont - 1) < 1e-4
        assert abs(-om.imag - gamma / 2) <= 1e-3 * max(gamma, 1e10)
        return
    pytest.fail("no positive-frequency root")


def test_plasma_oscillation_eps_inf():
    # With eps_inf the uniform mode obeys eps_inf Omega(Omega + i g cos) = wp^2.
    w, e, _, _ = _plasma_series(GAM, eps_inf=2.5)
    z, resid = _two_root_fit(e)
    assert resid < 1e-12
    om = [1j * np.log(zz) / w.dt for zz in z if (1j * np.log(zz)).real > 0][0]
    Om = 2.0 / w.dt * np.sin(om * w.dt / 2)
    assert abs(2.5 * Om * (Om + 1j * GAM * np.cos(om * w.dt / 2)) - WP**2) / WP**2 < 1e-9


def test_probe_dft_matches_direct_and_closed_form():
    w = box_workload(4, 4, 4, bc=(W.BC_PERIODIC,) * 6, material=np.ones((4, 4, 4), np.uint8),
                     table=[[0, 0, 1], [WP, GAM, 1.0]])
    o = O.Oracle(w)
    freqs = np.linspace(1.0e15, 3.0e15, 41)
    o.probe_dft([[3.1e-9, 2.7e-9, 4.4e-9]], freqs, 0b001)
    o.set_field(O.E_X, np.full((4, 4, 4), 1.0e6))
    e = [1.0e6]
    N = 400
    for _ in range(N):
        o.step(1)
        e.append(o.get_field(O.E_X)[0, 0, 0])
    e = np.array(e)
    F = o.probe_read()[0, 0]
    t = np.arange(1, N + 1) * w.dt
    direct = (e[1:, None] * np.exp(2j * np.pi * freqs[None, :] * t[:, None])).sum(0) * w.dt
    assert np.abs(F - direct).max() <= 1e-12 * np.abs(direct).max()
    # closed form: e[n] = c1 z1^n + c2 z2^n  ->  sum of two geometric series
    z, _ = _two_root_fit(e)
    V = np.stack([z**0, z**1], axis=0)
    c = np.linalg.solve(V, e[:2].astype(complex))
    cf = np.zeros_like(freqs, dtype=complex)
    for ck, zk in zip(c, z):
        r = zk * np.exp(2j * np.pi * freqs * w.dt)
        cf += ck * r * (1 - r**N) / (1 - r)
    cf *= w.dt
    assert np.abs(F - cf).max() <= 1e-9 * np.abs(cf).max()
    # untouched components stay zero
    assert np.all(o.probe_read()[0, 1:] == 0)


def test_bulk_drude_permittivity_from_plane_wave():
    # Metal everywhere, periodic x and y (plane wave along z), absorbing z ends
    # far away; a sheet current launches a pulse centred at 3.5 PHz whose
    # spectrum stays well above the plasma frequency (2.18 PHz), so nothing
    # rings near cut-off inside the window.
    nz = 4000
    bc = (W.BC_PERIODIC,) * 4 + (W.BC_CPML, W.BC_CPML)
    w = box_workload(2, 2, nz, bc=bc, material=np.ones((nz, 2, 2), np.uint8), table=[[0, 0, 1], [WP, GAM, 1.0]])
    o = O.Oracle(w)
    zs, z1, z2 = 1500, 1600, 1610
    o.add_source(0, (0, 2, 0, 2, zs, zs + 1), 1e16, 1800 * w.dt, 420 * w.dt, 3.5e15)
    freqs = np.linspace(3.1e15, 3.9e15, 41)
    o.probe_dft([[0.5 * w.dx, 0, z1 * w.dz], [0.5 * w.dx, 0, z2 * w.dz]], freqs, 0b001)
    prev = O.set_threads(0)
    O.set_threads(2)  # a 2x2-cell cross-section: more threads only add overhead
    try:
        o.step(12000)  # the reflections from the z ends have not come back yet
    finally:
        O.set_threads(prev)
    F = o.probe_read()[:, 0, :]
    kt = -1j * np.log(F[1] / F[0]) / ((z2 - z1) * w.dz)   # exp(+i k z) with the e^{-i w t} convention
    K = 2 / w.dz * np.sin(kt * w.dz / 2)
    om = 2 * np.pi * freqs
    Om = 2 / w.dt * np.sin(om * w.dt / 2)
    eps = (W.C0 * K / Om) ** 2
    eps_num = 1 - WP**2 / (Om * (Om + 1j * GAM * np.cos(om * w.dt / 2)))
    eps_eq1 = 1 - WP**2 / (om * (om + 1j * GAM))
    assert np.abs(eps - eps_num).max() <= 1e-5 * np.abs(eps_num).min()
    # the collision term (imaginary part, ~1e-3) is resolved too
    assert np.abs(eps.imag - eps_num.imag).max() <= 0.02 * np.abs(eps_num.imag).min()
    assert (np.abs(eps - eps_eq1) / np.abs(1 - eps_eq1)).max() <= 1e-3


# ----------------------------------------------------------------- energy --
def _energy_run(with_particles, nsteps=60, eps_inf_metal=2.0):
    nx, ny, nz = 14, 12, 12
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[3:6, :, 4:11] = 1
    bc = (W.BC_PEC, W.BC_PEC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PEC, W.BC_PEC)
    # anisotropic cells: a transposed spacing in any curl breaks the identity
    w = box_workload(nx, ny, nz, bc=bc, material=mat, table=[[0, 0, 1], [WP, 0.0, eps_inf_metal]],
                     dx=2e-9, dy=2.6e-9, dz=1.7e-9)
    o = O.Oracle(w)
    if with_particles:
        rng = np.random.default_rng(7)
        n = 64
        xyz = np.stack([rng.uniform(4, 8, n) * w.dx, rng.uniform(0, ny, n) * w.dy,
                        rng.uniform(7.5, 9.5, n) * w.dz], 1)
        u = np.zeros((n, 3))
        u[:, 0] = W.electron_momentum(30.0)
        u[:, 2] = -0.3 * W.electron_momentum(30.0)
        q = -1e-16
        o.add_particles(xyz, u, q, W.ME * 1e-16 / W.QE)
    else:
        o.add_source(2, (6, 8, 5, 7, 8, 9), 1e17, 20 * w.dt, 6 * w.dt, 1.2e15)
    return w, o, nsteps


@pytest.mark.parametrize("with_particles", [False, True])
def test_energy_identity_lossless(with_particles):
    w, o, N = _energy_run(with_particles)
    V = w.dx * w.dy * w.dz
    eps0, mu0 = W.EPS0, W.MU0
    wp2 = [edge_wp2(w, c) for c in range(3)]
    einf = [edge_wp2(w, c, values=w.table[:, 2]) for c in range(3)]
    snaps = [dict(E=[np.zeros(o.shape)] * 3, H=[np.zeros(o.shape)] * 3, J=[np.zeros(o.shape)] * 3)]
    jf = []
    for _ in range(N):
        o.step(1)
        snaps.append(dict(E=[o.get_field(c) for c in range(3)], H=[o.get_field(3 + c) for c in range(3)],
                          J=[o.get_field(6 + c) for c in range(3)]))
        jf.append([o.get_field(9 + c) for c in range(3)])

    def W_at(n):
        # snaps[n] holds E^n, H^{n-1/2}, J^{n-1/2}; snaps[n+1] holds H^{n+1/2}, J^{n+1/2}
        a, b = snaps[n], snaps[n + 1]
        we = sum(0.5 * eps0 * (einf[c] * a["E"][c] ** 2).sum() for c in range(3))
        wh = sum(0.5 * mu0 * (a["H"][c] * b["H"][c]).sum() for c in range(3))
        wj = 0.0
        for c in range(3):
            m = wp2[c] > 0
            wj += (a["J"][c][m] * b["J"][c][m] / (2 * eps0 * wp2[c][m])).sum()
        return V * (we + wh + wj)

    Ws = [W_at(n) for n in range(N)]
    scale = max(abs(x) for x in Ws)
    assert scale > 0
    worst = 0.0
    for n in range(N - 1):
        work = -w.dt * V * sum((jf[n][c] * (snaps[n]["E"][c] + snaps[n + 1]["E"][c]) / 2).sum() for c in range(3))
        worst = max(worst, abs(Ws[n + 1] - Ws[n] - work) / scale)
    assert worst < 1e-12, worst


def test_energy_decays_with_collisions():
    nx = ny = nz = 10
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[3:7, 3:7, 3:7] = 1
    w = box_workload(nx, ny, nz, material=mat, table=[[0, 0, 1], [WP, 5e14, 1.0]])
    o = O.Oracle(w)
    E0 = np.zeros(o.shape)
    E0[4:6, 4:6, 4:6] = 1e8
    o.set_field(O.E_X, E0)
    V = w.dx**3
    prev = None
    energies = []
    for _ in range(200):
        o.step(1)
        e = sum((o.get_field(c) ** 2).sum() for c in range(3)) * 0.5 * W.EPS0 * V
        h = sum((o.get_field(3 + c) ** 2).sum() for c in range(3)) * 0.5 * W.MU0 * V
        energies.append(e + h)
    # field energy oscillates but its envelope must decay (collisions only remove energy)
    first = max(energies[:50])
    last = max(energies[-50:])
    assert last < first


# ------------------------------------------------------------------ Gauss --
def test_gauss_law_residual_constant_with_particles_and_metal():
    nx, ny, nz = 20, 14, 14
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[3:6] = 1
    bc = (W.BC_PEC, W.BC_PEC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PEC, W.BC_PEC)
    w = box_workload(nx, ny, nz, bc=bc, material=mat, table=[[0, 0, 1], [WP, GAM, 1.0]],
                     dx=2e-9, dy=1.5e-9, dz=2.4e-9)
    o = O.Oracle(w)
    rng = np.random.default_rng(11)
    n = 80
    xyz = np.stack([rng.uniform(3, 9, n) * w.dx, rng.uniform(0, ny, n) * w.dy,
                    rng.uniform(6.2, 8.5, n) * w.dz], 1)
    u = np.zeros((n, 3))
    u[:, 0] = W.electron_momentum(30.0)
    u[:, 2] = -0.5 * W.electron_momentum(30.0)  # some electrons reach the metal and freeze
    q = -2e-17
    o.add_particles(xyz, u, q, W.ME * 2e-17 / W.QE)
    mask = interior_node_mask(w, margin=1)
    x0, _, _ = o.particles()
    E0 = [o.get_field(c) for c in range(3)]
    worst = 0.0
    frozen_seen = 0
    for _ in range(40):
        o.step(1)
        x1, _, st = o.particles()
        frozen_seen = int(st.sum())
        E1 = [o.get_field(c) for c in range(3)]
        Jp = [o.get_field(6 + c) for c in range(3)]
        dE = [E1[c] - E0[c] for c in range(3)]
        lhs = W.EPS0 * node_divergence(w, *dE) + w.dt * node_divergence(w, *Jp)
        drho = cic_charge(w, x1, q) - cic_charge(w, x0, q)
        scale = np.abs(drho).max()
        worst = max(worst, np.abs((lhs - drho)[mask]).max() / scale)
        x0, E0 = x1, E1
    assert worst < 1e-9, worst
    assert frozen_seen > 0  # the freeze rule was exercised


def test_esirkepov_single_particle_continuity_and_total_current():
    w = box_workload(10, 10, 10, bc=(W.BC_PERIODIC,) * 6)
    o = O.Oracle(w)
    q = -1e-18
    x0 = np.array([[4.9, 5.02, 6.97]]) * w.dx  # crosses cell faces in x and z
    u = np.array([[0.6, -0.2, 0.3]]) * W.C0
    o.add_particles(x0, u, q, W.ME * 1e-18 / W.QE)
    for _ in range(3):
        xa, _, _ = o.particles()
        o.step(1)
        xb, _, _ = o.particles()
        J = [o.get_field(9 + c) for c in range(3)]
        drho = cic_charge(w, xb, q) - cic_charge(w, xa, q)
        res = drho + w.dt * node_divergence(w, *J)
        assert np.abs(res).max() <= 1e-12 * np.abs(drho).max()
        # sum of J V = q * displacement / dt (dipole-moment rate), per axis
        disp = xb[0] - xa[0]
        L = np.array([w.nx, w.ny, w.nz]) * w.dx
        disp -= np.round(disp / L) * L
        V = w.dx**3
        for c in range(3):
            assert abs(J[c].sum() * V - q * disp[c] / w.dt) <= 1e-12 * abs(q) * W.C0


# ------------------------------------------------------------------ Boris --
def test_boris_pure_magnetic_rotation():
    qm = -W.QE / W.ME
    dt = 2e-18
    u = np.array([0.5, 0.2, 0.1]) * W.C0
    B = np.array([0.0, 0.0, 3.0e3])
    g = math.sqrt(1 + (u @ u) / W.C0**2)
    un = O.boris(u, [0, 0, 0], B, qm, dt, W.C0)
    assert abs(np.linalg.norm(un) / np.linalg.norm(u) - 1) < 1e-15
    assert un[2] == u[2]
    t = abs(0.5 * qm * dt * B[2] / g)
    ang = math.atan2(u[0] * un[1] - u[1] * un[0], u[0] * un[0] + u[1] * un[1])
    assert abs(abs(ang) - 2 * math.atan(t)) < 1e-12 * 2 * math.atan(t) + 1e-16
    # electrons (q < 0) gyrate counter-clockwise about +B
    assert ang > 0


def test_boris_pure_electric_impulse():
    qm = -W.QE / W.ME
    dt = 2e-18
    u = np.array([1e7, -2e6, 3e5])
    E = np.array([1e10, 2e9, -5e9])
    un = O.boris(u, E, [0, 0, 0], qm, dt, W.C0)
    assert np.allclose(un, u + qm * E * dt, rtol=0, atol=1e-15 * W.C0)


def test_boris_exb_drift():
    qm = -W.QE / W.ME
    B = np.array([0.0, 0.0, 1.0e4])
    E = np.array([0.0, 1.0e11, 0.0])
    vd = np.cross(E, B) / (B @ B)  # E x B / B^2 = (1e7, 0, 0) m/s
    wc = abs(qm) * B[2]
    dt = 2 * math.pi / wc / 200
    u = np.zeros(3)
    xs = []
    x = np.zeros(3)
    for _ in range(20000):
        u = O.boris(u, E, B, qm, dt, W.C0)
        g = math.sqrt(1 + (u @ u) / W.C0**2)
        x = x + dt * u / g
        xs.append(x.copy())
    T = 20000 * dt
    v_mean = (xs[-1] - xs[0]) / (T - dt)
    assert abs(v_mean[0] / vd[0] - 1) < 2e-3
    assert abs(v_mean[1]) < 2e-3 * vd[0]


def test_gyration_in_static_field_closed_form():
    # A test electron (no deposit) in a uniform static Hz: each Boris step
    # rotates u by the fixed angle 2 atan|t|, so x_N - x_0 is the geometric
    # sum dt/gamma * sum_{n=1..N} R^n u_0 (closed form, no integration).
    w = box_workload(12, 12, 12, bc=(W.BC_PERIODIC,) * 6, dx=2e-9, dy=1.6e-9, dz=2.3e-9)
    o = O.Oracle(w)
    H0 = 2.0e9  # A/m (mu0 H ~ 2.5e3 T keeps the orbit a few cells wide)
    o.set_field(O.H_Z, np.full(o.shape, H0))
    o.set_deposit(False)
    x0 = np.array([[5.3 * w.dx, 6.1 * w.dy, 4.4 * w.dz]])
    u0 = np.array([[0.2 * W.C0, 0.05 * W.C0, 0.01 * W.C0]])
    q = -1e-19
    o.add_particles(x0, u0, q, W.ME * 1e-19 / W.QE)
    N = 40
    o.step(N)
    x, u, st = o.particles()
    assert st[0] == 0
    assert np.all(o.get_field(O.H_Z) == H0)  # curl of a uniform field vanishes
    qm = -W.QE / W.ME
    g = math.sqrt(1 + (u0[0] @ u0[0]) / W.C0**2)
    t = 0.5 * qm * w.dt * W.MU0 * H0 / g
    th = -2 * math.atan(t)  # rotation angle about +z per step
    c, s_ = math.cos(th), math.sin(th)
    R = np.array([[c, -s_], [s_, c]])
    v = u0[0, :2].copy()
    disp = np.zeros(2)
    for _ in range(N):
        v = R @ v
        disp += w.dt * v / g
    L = np.array([w.nx * w.dx, w.ny * w.dy])
    got = x[0, :2] - x0[0, :2]
    got -= np.round((got - disp) / L) * L
    assert np.allclose(got, disp, rtol=0, atol=1e-12 * np.abs(disp).max())
    assert abs(x[0, 2] - x0[0, 2] - N * w.dt * u0[0, 2] / g) < 1e-12 * w.dz
    assert np.allclose(u[0, :2], v, rtol=1e-12)


def test_gather_and_probe_staggering_on_linear_fields():
    # Curl-free linear fields F_c = g_c * (position of component c along
    # axis c) are reproduced exactly by trilinear interpolation on the
    # component's own staggered lattice, so one push gives the Boris result
    # for the exact local E and B, and the probe sees the exact local E.
    w = box_workload(10, 10, 10, dx=2e-9, dy=1.7e-9, dz=2.2e-9)
    o = O.Oracle(w)
    gE = np.array([3e18, -2e18, 5e18])   # V/m per m
    gH = np.array([4e17, 6e17, -3e17])   # A/m per m
    k, j, i = np.meshgrid(np.arange(10), np.arange(10), np.arange(10), indexing="ij")
    pos = [i * w.dx, j * w.dy, k * w.dz]
    d = (w.dx, w.dy, w.dz)
    for c in range(3):
        o.set_field(c, gE[c] * (pos[c] + 0.5 * d[c]))   # E_c sits half a cell along axis c
        o.set_field(3 + c, gH[c] * pos[c])              # H_c sits on the node along axis c
    o.set_deposit(False)
    xp = np.array([4.37 * w.dx, 5.81 * w.dy, 4.12 * w.dz])
    probe = np.array([5.64 * w.dx, 3.29 * w.dy, 6.71 * w.dz])
    freqs = np.array([1e15, 2e15])
    o.probe_dft([probe], freqs, 0b111)
    u0 = np.array([0.3 * W.C0, -0.1 * W.C0, 0.05 * W.C0])
    q = -1e-19
    o.add_particles(xp[None], u0[None], q, W.ME * 1e-19 / W.QE)
    o.step(1)
    _, u, _ = o.particles()
    want = O.boris(u0, gE * xp, W.MU0 * gH * xp, -W.QE / W.ME, w.dt, W.C0)
    assert np.allclose(u[0], want, rtol=1e-13, atol=0)
    F = o.probe_read()[0]
    ph = np.exp(2j * np.pi * freqs * w.dt) * w.dt
    for c in range(3):
        assert np.allclose(F[c], gE[c] * probe[c] * ph, rtol=1e-12, atol=0)


def test_magnetic_field_time_centring():
    # E_y = g x (static, curl_z E = g) makes H_z uniform and linear in time:
    # H^{n+1/2} = H^{n-1/2} - g dt/mu0 exactly.  The push at step n must use
    # B^n = mu0 H(t_n), the mean of the two half-step fields.
    bc = (W.BC_PEC, W.BC_PEC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC)
    w = box_workload(10, 8, 8, bc=bc)
    o = O.Oracle(w)
    g = 2e18
    H0 = 1.0e9
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(10), indexing="ij")
    o.set_field(O.E_Y, g * i * w.dx)
    o.set_field(O.H_Z, np.full(o.shape, H0))
    o.set_deposit(False)
    xp = np.array([4.6 * w.dx, 3.3 * w.dy, 2.2 * w.dz])
    u0 = np.array([0.2 * W.C0, 0.1 * W.C0, 0.0])
    o.add_particles(xp[None], u0[None], -1e-19, W.ME * 1e-19 / W.QE)
    o.step(1)
    _, u, _ = o.particles()
    Hz = o.get_field(O.H_Z)
    assert np.allclose(Hz[:, :, :8], H0 - g * w.dt / W.MU0, rtol=1e-14, atol=0)
    B = np.array([0, 0, W.MU0 * H0 - 0.5 * g * w.dt])
    want = O.boris(u0, [0, g * xp[0], 0], B, -W.QE / W.ME, w.dt, W.C0)
    assert np.allclose(u[0], want, rtol=1e-13, atol=0)
    wrong = O.boris(u0, [0, g * xp[0], 0], [0, 0, W.MU0 * H0 - g * w.dt], -W.QE / W.ME, w.dt, W.C0)
    assert np.abs(want - wrong).max() > 1e3 * 1e-13 * np.abs(want).max()


# ------------------------------------------------------------------- CPML --
def _cpml_run(n, nsteps, probes):
    # CPML on all six faces; two oblique current sources excite every field
    # component, so every psi term of the absorbing layers is exercised.
    w = box_workload(n, n, n, bc=(W.BC_CPML,) * 6, dx=2e-9, dy=2.2e-9, dz=1.8e-9)
    o = O.Oracle(w)
    c = n // 2
    o.add_source(2, (c, c + 1, c, c + 1, c, c + 1), 1e18, 30 * w.dt, 8 * w.dt, 0.0)
    o.add_source(0, (c + 1, c + 2, c - 1, c, c + 1, c + 2), 7e17, 34 * w.dt, 8 * w.dt, 0.0)
    rec = []
    for _ in range(nsteps):
        o.step(1)
        f = [o.get_field(q) for q in range(6)]
        rec.append([f[q][p[2] + c, p[1] + c, p[0] + c] for p in probes for q in range(6)])
    return np.array(rec)


def test_cpml_reflection_below_40db():
    small, big, N = 28, 76, 140
    r = small // 2 - 8 - 2  # probes two cells inside each slab's inner face
    probes = [(r, 0, 0), (-r, 1, 0), (0, r, 1), (1, -r, 0), (0, 1, r), (-1, 0, -r), (r, r, -r)]
    a = _cpml_run(small, N, probes)
    b = _cpml_run(big, N, probes)
    scale = np.abs(b).reshape(N, len(probes), 6).max(axis=(0, 1))  # per field component
    err = (np.abs(a - b).reshape(N, len(probes), 6).max(axis=(0, 1)) / scale).max()
    db = 20 * math.log10(err)
    assert db < -40.0, db


def test_edge_material_average_on_film():
    w = W.c1(nsteps=0)
    o = O.Oracle(w)
    bJ = o.coeff(1, 0)[:, 20, 60]  # Ex beta_J along z at one column
    full = bJ[12]
    assert full > 0
    for k in range(9, 18):
        assert bJ[k] == pytest.approx(full, rel=1e-15)
    assert bJ[8] == pytest.approx(0.5 * full, rel=1e-15)
    assert bJ[18] == pytest.approx(0.5 * full, rel=1e-15)
    assert bJ[7] == 0.0 and bJ[19] == 0.0
    bz = o.coeff(1, 2)[:, 20, 60]  # Ez edges sit between planes k and k+1
    assert all(bz[k] == pytest.approx(full, rel=1e-15) for k in range(8, 18))
    assert bz[7] == 0.0 and bz[18] == 0.0
    kJ = o.coeff(0, 0)[12, 20, 60]
    g = W.AG_GAMMA * w.dt
    assert kJ == pytest.approx((2 - g) / (2 + g), rel=1e-15)


# ------------------------------------------------------- freeze rule (R11) --
@pytest.mark.parametrize("target", ["metal", "face"])
def test_freeze_rule_stops_the_step_that_would_enter(target):
    """With the deposit off and no fields an electron moves ballistically,
    x^{n+1} = x^n + dt u / gamma.  It must freeze on exactly the step whose
    new position would lie in a metal cell (film below it, moving -z) or
    within two cells of a non-periodic face (moving +x), keep the position it
    had, and never move again."""
    n = 24
    mat = np.zeros((n, n, n), np.uint8)
    mat[:8] = 1  # metal planes z < 8 cells
    w = box_workload(n, n, n, bc=(W.BC_PEC,) * 6, material=mat, table=W.drude_table())
    o = O.Oracle(w)
    o.set_deposit(False)
    d = w.dx
    x0 = np.array([[11.3 * d, 12.5 * d, 12.7 * d]])
    speed = 0.6 * W.C0  # |u| = gamma beta c
    gam = math.sqrt(1.0 + (speed / W.C0) ** 2)
    u = np.array([[0.0, 0.0, -speed]]) if target == "metal" else np.array([[speed, 0.0, 0.0]])
    o.add_particles(x0, u, -1e-19, W.ME)
    v = u[0] / gam
    # the step whose new position is the first one not allowed
    x = x0[0].copy()
    stop = None
    for step in range(200):
        nxt = x + w.dt * v
        if target == "metal":
            bad = nxt[2] < 8 * d
        else:
            bad = nxt[0] >= (n - 2) * d  # the allowed region ends two cells before the face
        if bad:
            stop = step
            break
        x = nxt
    assert stop is not None
    o.step(stop)
    xs, _, s = o.particles()
    assert s[0] == 0 and np.allclose(xs[0], x, rtol=0, atol=1e-12 * d)
    o.step(1)
    xs, _, s = o.particles()
    assert s[0] == 1 and np.allclose(xs[0], x, rtol=0, atol=1e-12 * d)
    o.step(5)
    xs2, _, s2 = o.particles()
    assert s2[0] == 1 and np.array_equal(xs2, xs)


# --------------------------------------------------------- prescribed current --
@pytest.mark.parametrize("f0", [0.0, 1.2e15])
def test_source_current_first_step_closed_form(f0):
    """From zero fields, one step of a prescribed current J in vacuum gives
    E^1 = -dt/eps0 J(t_1/2) on the source edges (curl H^1/2 = 0) and leaves
    every other edge at zero: J = amp exp(-s^2) sin(2 pi f0 (t - t0)) for
    f0 > 0, amp (-2 s) exp(-s^2) for f0 = 0, s = (t - t0)/tau, t = dt/2."""
    w = box_workload(12, 12, 12, bc=(W.BC_PEC,) * 6)
    o = O.Oracle(w)
    amp, t0, tau = 3.0e9, 2.0 * w.dt, 1.5 * w.dt
    box = (4, 7, 5, 8, 3, 9)
    o.add_source(1, box, amp, t0, tau, f0)
    o.step(1)
    t = 0.5 * w.dt
    sarg = (t - t0) / tau
    J = amp * math.exp(-sarg * sarg) * (math.sin(2 * math.pi * f0 * (t - t0)) if f0 > 0 else -2.0 * sarg)
    ey = o.get_field(O.E_Y)
    expect = np.zeros_like(ey)
    expect[box[4]:box[5], box[2]:box[3], box[0]:box[1]] = -w.dt / W.EPS0 * J
    assert np.allclose(ey, expect, rtol=1e-14, atol=0)
    for c in (O.E_X, O.E_Z, O.H_X, O.H_Y, O.H_Z):
        assert not o.get_field(c).any()


# ------------------------------------------------------ edge materials (R6) --
def test_edge_coefficients_follow_the_four_cell_rule():
    """Random map of three materials on a grid periodic in y, absorbing in x,
    conducting in z: every edge's (kJ, bJ, dt/(eps0 eps_inf)) equals the rule
    written out here from the cell means -- wp^2 averaged over the four cells
    around the edge (wrapped on the periodic axis, clamped on the others),
    gamma weighted by wp^2, eps_inf averaged -- through the coefficients of
    Eq. 6 and Eq. 8."""
    rng = np.random.default_rng(23)
    table = np.array([[0.0, 0.0, 1.0], [1.3e16, 3.0e13, 1.0], [0.9e16, 1.1e14, 2.5]])
    mat = rng.integers(0, 3, (6, 8, 20)).astype(np.uint8)
    w = box_workload(20, 8, 6, bc=(W.BC_CPML, W.BC_CPML, W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PEC, W.BC_PEC),
                     material=mat, table=table)
    w.cpml_cells = 4
    o = O.Oracle(w)
    dt = w.dt
    for c in range(3):
        wp2 = edge_wp2(w, c)
        wp2g = edge_wp2(w, c, values=table[:, 0] ** 2 * table[:, 1])
        einf = edge_wp2(w, c, values=table[:, 2])
        gam = np.where(wp2 > 0, wp2g / np.where(wp2 > 0, wp2, 1.0), 0.0)
        kJ = (2 - gam * dt) / (2 + gam * dt)
        bJ = 2 * dt * W.EPS0 * wp2 / (2 + gam * dt)
        cE = dt / (W.EPS0 * einf)
        metal = wp2 > 0
        assert np.allclose(o.coeff(1, c), bJ, rtol=1e-13, atol=0)
        assert np.allclose(o.coeff(0, c)[metal], kJ[metal], rtol=1e-13, atol=0)
        assert np.allclose(o.coeff(2, c), cE, rtol=1e-13, atol=0)


def test_oracle_result_does_not_depend_on_thread_count():
    """The oracle's cell loops run on OpenMP threads and its particles one by
    one in input order, so the fields and particles after some steps are the
    same bit for bit on one thread and on several."""
    w = W.scaled(W.c1(), 48, 24, 40, 256, 30)
    out = []
    for threads in (1, 4):
        O.set_threads(threads)
        o = O.from_workload(w)
        o.step(30)
        out.append(([o.get_field(c) for c in range(6)], o.particles()[0], o.probe_read()))
    O.set_threads(len(__import__("os").sched_getaffinity(0)))
    (f1, x1, p1), (f4, x4, p4) = out
    assert all(np.array_equal(a, b) for a, b in zip(f1, f4))
    assert np.array_equal(x1, x4) and np.array_equal(p1, p4)
