"""ctypes wrapper around the FP64 CPU oracle (pic_oracle.c).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline leg may use it.  The CUDA library never imports it.  The wrapper
only marshals arrays; every step of the method runs in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pic_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

_lock = threading.Lock()
_lib = None

E_X, E_Y, E_Z, H_X, H_Y, H_Z, JP_X, JP_Y, JP_Z, JF_X, JF_Y, JF_Z = range(12)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over cells; particles stay serial)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
               SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = P
            L.orc_create.argtypes = [C.POINTER(C.c_long), dp, C.c_double, C.c_double, C.c_double,
                                     C.POINTER(C.c_int), C.c_int, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.POINTER(C.c_uint8), C.c_int, dp, C.POINTER(C.c_int)]
            L.orc_destroy.argtypes = [P]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            L.orc_get_field.argtypes = [P, C.c_int, dp]
            L.orc_set_field.argtypes = [P, C.c_int, dp]
            L.orc_add_particles.argtypes = [P, C.c_long, dp, dp, C.c_double, C.c_double, C.POINTER(C.c_long)]
            L.orc_get_particles.argtypes = [P, dp, dp, C.POINTER(C.c_uint8)]
            L.orc_num_particles.argtypes = [P]
            L.orc_num_particles.restype = C.c_long
            L.orc_set_deposit.argtypes = [P, C.c_int]
            L.orc_add_source.argtypes = [P, C.c_int, C.POINTER(C.c_long), C.c_double, C.c_double,
                                         C.c_double, C.c_double]
            L.orc_probe_dft.argtypes = [P, C.c_int, dp, C.c_uint, C.c_int, dp]
            L.orc_probe_read.argtypes = [P, dp]
            L.orc_step.argtypes = [P, C.c_long]
            L.orc_get_step.argtypes = [P]
            L.orc_get_step.restype = C.c_long
            L.orc_get_coeff.argtypes = [P, C.c_int, C.c_int, dp]
            L.orc_boris.argtypes = [dp, dp, dp, C.c_double, C.c_double, C.c_double]
            L.orc_boris.restype = None
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def boris(u, E, B, qm, dt, c):
    """One relativistic Boris step of the oracle on a single momentum."""
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    e = np.ascontiguousarray(E, dtype=np.float64)
    b = np.ascontiguousarray(B, dtype=np.float64)
    lib().orc_boris(_dp(uu), _dp(e), _dp(b), qm, dt, c)
    return uu


class Oracle:
    """One oracle simulation built from a workload-like object (duck-typed:
    nx, ny, nz, dx, dy, dz, dt, bc, cpml_*, material, table)."""

    def __init__(self, w, eps0=None, mu0=None):
        L = lib()
        eps0 = 8.8541878128e-12 if eps0 is None else eps0
        mu0 = 1.25663706212e-6 if mu0 is None else mu0
        self.shape = (w.nz, w.ny, w.nx)
        self.n = w.nx * w.ny * w.nz
        n = (C.c_long * 3)(w.nx, w.ny, w.nz)
        d = np.array([w.dx, w.dy, w.dz], dtype=np.float64)
        bc = (C.c_int * 6)(*w.bc)
        mat = np.ascontiguousarray(w.material, dtype=np.uint8)
        assert mat.shape == self.shape
        tab = np.ascontiguousarray(w.table, dtype=np.float64)
        st = C.c_int(0)
        h = L.orc_create(n, _dp(d), w.dt, eps0, mu0, bc, int(w.cpml_cells), float(w.cpml_order),
                         float(w.cpml_sigma_fac), float(w.cpml_kappa_max), float(w.cpml_alpha_max),
                         mat.ctypes.data_as(C.POINTER(C.c_uint8)), int(tab.shape[0]), _dp(tab),
                         C.byref(st))
        if not h:
            raise OracleError(f"orc_create failed with status {st.value}")
        self.h = C.c_void_p(h)
        self.nprobe = 0
        self.nfreq = 0

    def close(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def get_field(self, which: int) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        _check(lib().orc_get_field(self.h, which, _dp(out)), "orc_get_field")
        return out.reshape(self.shape)

    def set_field(self, which: int, arr) -> None:
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
        assert a.size == self.n
        _check(lib().orc_set_field(self.h, which, _dp(a)), "orc_set_field")

    def coeff(self, which: int, comp: int) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        _check(lib().orc_get_coeff(self.h, which, comp, _dp(out)), "orc_get_coeff")
        return out.reshape(self.shape)

    def add_particles(self, xyz, u, q, m) -> None:
        x = np.ascontiguousarray(xyz, dtype=np.float64)
        v = np.ascontiguousarray(u, dtype=np.float64)
        bad = C.c_long(0)
        rc = lib().orc_add_particles(self.h, x.shape[0], _dp(x), _dp(v), q, m, C.byref(bad))
        if rc != 0:
            raise OracleError(f"orc_add_particles: {bad.value} particles outside the allowed region")

    def particles(self):
        n = lib().orc_num_particles(self.h)
        x = np.empty((n, 3)); u = np.empty((n, 3)); s = np.empty(n, dtype=np.uint8)
        lib().orc_get_particles(self.h, _dp(x), _dp(u), s.ctypes.data_as(C.POINTER(C.c_uint8)))
        return x, u, s

    def set_deposit(self, on: bool) -> None:
        lib().orc_set_deposit(self.h, int(bool(on)))

    def add_source(self, comp, box, amp, t0, tau, f0=0.0) -> None:
        b = (C.c_long * 6)(*box)
        _check(lib().orc_add_source(self.h, comp, b, amp, t0, tau, f0), "orc_add_source")

    def probe_dft(self, xyz, freqs, comp_mask=0b111) -> None:
        p = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        f = np.ascontiguousarray(freqs, dtype=np.float64)
        _check(lib().orc_probe_dft(self.h, p.shape[0], _dp(p), comp_mask, f.size, _dp(f)), "orc_probe_dft")
        self.nprobe, self.nfreq = p.shape[0], f.size

    def probe_read(self) -> np.ndarray:
        """Complex [nprobe][3][nfreq]."""
        out = np.empty(self.nprobe * 3 * self.nfreq * 2)
        _check(lib().orc_probe_read(self.h, _dp(out)), "orc_probe_read")
        z = out.reshape(self.nprobe, 3, self.nfreq, 2)
        return z[..., 0] + 1j * z[..., 1]

    def step(self, n: int = 1) -> None:
        _check(lib().orc_step(self.h, int(n)), "orc_step")

    @property
    def step_index(self) -> int:
        return lib().orc_get_step(self.h)


def from_workload(w, with_particles=True, with_probes=True) -> Oracle:
    o = Oracle(w)
    if with_particles and w.nparticles:
        o.add_particles(w.xyz, w.u, w.q_macro, w.m_macro)
    if with_probes and w.probes is not None and w.freqs is not None:
        o.probe_dft(w.probes, w.freqs, w.comp_mask)
    return o
