"""Small synthetic cases and textbook diagnostics shared by the tests.

The diagnostics here are written from their definitions (cloud-in-cell charge
at grid nodes, the node divergence of edge fields, the discrete field energy)
and are independent of both the oracle and the CUDA library.
"""
import numpy as np

from paper_1505_04007_gb300 import workloads as W


def box_workload(nx, ny, nz, dx=2e-9, bc=(W.BC_PEC,) * 6, material=None, table=None,
                 courant=0.5, name="box", dy=None, dz=None):
    dy = dx if dy is None else dy
    dz = dx if dz is None else dz
    w = W.Workload(name=name, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
                   dt=W.yee_dt(dx, dy, dz, courant), nsteps=0, bc=tuple(bc))
    w.material = np.zeros((nz, ny, nx), np.uint8) if material is None else material.astype(np.uint8)
    w.table = W.drude_table() if table is None else np.asarray(table, np.float64)
    w.cpml_alpha_max = 0.05 * W.EPS0 * W.AG_WP
    return w


def periodic_axes(w):
    return [w.bc[2 * a] == W.BC_PERIODIC for a in range(3)]


def cic_charge(w, xyz, q):
    """Charge density at nodes [nz][ny][nx] from linear node shapes."""
    rho = np.zeros((w.nz, w.ny, w.nx))
    d = np.array([w.dx, w.dy, w.dz])
    n = np.array([w.nx, w.ny, w.nz])
    per = periodic_axes(w)
    V = w.dx * w.dy * w.dz
    for p in range(xyz.shape[0]):
        xi = xyz[p] / d
        b = np.floor(xi).astype(int)
        f = xi - b
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    idx = [b[0] + di, b[1] + dj, b[2] + dk]
                    ok = True
                    for a in range(3):
                        if per[a]:
                            idx[a] %= n[a]
                        elif not (0 <= idx[a] < n[a]):
                            ok = False
                    if not ok:
                        continue
                    wgt = (f[0] if di else 1 - f[0]) * (f[1] if dj else 1 - f[1]) * (f[2] if dk else 1 - f[2])
                    rho[idx[2], idx[1], idx[0]] += q * wgt / V
    return rho


def node_divergence(w, fx, fy, fz):
    """div at node (i,j,k) of edge fields: (Fx(i+1/2)-Fx(i-1/2))/dx + ...;
    arrays [nz][ny][nx], x edge i+1/2 stored at index i.  On non-periodic
    axes the value below index 0 is taken as zero (result at index 0 is only
    meaningful on periodic axes)."""
    per = periodic_axes(w)

    def back(a, axis):
        if per[axis]:
            return np.roll(a, 1, axis=2 - axis)
        b = np.zeros_like(a)
        sl = [slice(None)] * 3
        sl2 = [slice(None)] * 3
        sl[2 - axis] = slice(1, None)
        sl2[2 - axis] = slice(0, -1)
        b[tuple(sl)] = a[tuple(sl2)]
        return b

    return (fx - back(fx, 0)) / w.dx + (fy - back(fy, 1)) / w.dy + (fz - back(fz, 2)) / w.dz


def interior_node_mask(w, margin=1):
    """Nodes at least ``margin`` cells (plus the CPML slab) away from every
    non-periodic face."""
    m = np.ones((w.nz, w.ny, w.nx), bool)
    per = periodic_axes(w)
    n = (w.nx, w.ny, w.nz)
    for a in range(3):
        if per[a]:
            continue
        lo = margin + (w.cpml_cells if W.BC_CPML in (w.bc[2 * a], w.bc[2 * a + 1]) else 0)
        idx = np.arange(n[a])
        keep = (idx >= lo) & (idx < n[a] - lo)
        shape = [1, 1, 1]
        shape[2 - a] = n[a]
        m &= keep.reshape(shape)
    return m


def edge_wp2(w, comp, values=None):
    """Mean of wp^2 (or of a per-material ``values`` table) over the four
    cells sharing each edge of component comp (clamped at non-periodic faces,
    wrapped on periodic ones)."""
    wp2 = ((w.table[:, 0] ** 2) if values is None else np.asarray(values))[w.material]
    per = periodic_axes(w)
    a1, a2 = (comp + 1) % 3, (comp + 2) % 3

    def shift_back(a, axis):
        if per[axis]:
            return np.roll(a, 1, axis=2 - axis)
        out = a.copy()
        sl = [slice(None)] * 3
        sl2 = [slice(None)] * 3
        sl[2 - axis] = slice(1, None)
        sl2[2 - axis] = slice(0, -1)
        out[tuple(sl)] = a[tuple(sl2)]
        return out

    s1 = shift_back(wp2, a1)
    return 0.25 * (wp2 + s1 + shift_back(wp2, a2) + shift_back(s1, a2))


def spectral_peak(freqs, power, band=None):
    """Frequency of the largest value of power (optionally inside band =
    (f_lo, f_hi)), refined by the vertex of the parabola through the
    maximum and its two neighbours."""
    f = np.asarray(freqs, np.float64)
    p = np.asarray(power, np.float64)
    idx = np.arange(f.size)
    if band is not None:
        idx = idx[(f >= band[0]) & (f <= band[1])]
    m = idx[np.argmax(p[idx])]
    if 0 < m < f.size - 1:
        y0, y1, y2 = p[m - 1], p[m], p[m + 1]
        den = y0 - 2 * y1 + y2
        shift = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        return f[m] + shift * (f[1] - f[0])
    return f[m]


def cic_charge_fast(w, xyz, q):
    """Vectorised cic_charge (same definition: linear node shapes)."""
    rho = np.zeros(w.nx * w.ny * w.nz)
    d = np.array([w.dx, w.dy, w.dz])
    n = np.array([w.nx, w.ny, w.nz])
    per = periodic_axes(w)
    xi = xyz / d
    b = np.floor(xi).astype(np.int64)
    f = xi - b
    V = w.dx * w.dy * w.dz
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                idx = []
                ok = np.ones(xyz.shape[0], bool)
                for a, off in enumerate((di, dj, dk)):
                    ia = b[:, a] + off
                    if per[a]:
                        ia = np.mod(ia, n[a])
                    else:
                        ok &= (ia >= 0) & (ia < n[a])
                        ia = np.clip(ia, 0, n[a] - 1)
                    idx.append(ia)
                wgt = ((f[:, 0] if di else 1 - f[:, 0]) * (f[:, 1] if dj else 1 - f[:, 1]) *
                       (f[:, 2] if dk else 1 - f[:, 2]))
                lin = (idx[2] * n[1] + idx[1]) * n[0] + idx[0]
                np.add.at(rho, lin[ok], q * wgt[ok] / V)
    return rho.reshape(w.nz, w.ny, w.nx)


def film_spp_workload(thick_cells, nsteps, nx=256, npart=1024, charge=1e-18, wp=1.2e16, gamma=1.45e13,
                      kev=100.0, seed=5):
    """The quasi-2D film model of workloads.film_plasmon with Ex and Ez probed
    from 1.0 to 1.5 PHz."""
    w = W.film_plasmon(thick_cells, nsteps, nx=nx, npart=npart, charge=charge, wp=wp, gamma=gamma, kev=kev,
                       seed=seed)
    w.name = "film_spp"
    return w


# (film cells, steps, band searched for the dominant peak): thick film and two thin films
FILM_CASES = [(75, 8000, (1.1e15, 1.35e15)), (10, 24000, (1.2e15, 1.49e15)), (20, 24000, (1.2e15, 1.49e15))]
