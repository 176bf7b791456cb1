"""Python binding of libpic (include/pic.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method; all of the time step runs in the CUDA kernels of
libpic.  The library must be built for the GPU (``build.build()``); if it is
missing or cannot be loaded, loading raises instead of falling back to
anything else.

``Simulation`` is a convenience wrapper that builds a ``pic_config`` from a
``workloads.Workload``, takes its device memory from PyTorch (one uint8
tensor handed to the library as its workspace) and runs on a PyTorch stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PIC_OK = 0
PIC_FP32, PIC_FP64 = 0, 1
PIC_FLAG_SPLIT_FIELDS = 1  # keep separate H and E updates where the fused pass would run
PIC_FLAG_STAGED_UPLOAD = 2  # copy host arrays through the runtime rather than read them with kernels
PIC_EX, PIC_EY, PIC_EZ, PIC_HX, PIC_HY, PIC_HZ, PIC_JPX, PIC_JPY, PIC_JPZ, PIC_JFX, PIC_JFY, PIC_JFZ = range(12)

ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_CFL", -3: "PIC_ERR_OOM", -4: "PIC_ERR_CUDA", -5: "PIC_ERR_NONFINITE",
          -6: "PIC_ERR_STATE", -7: "PIC_ERR_UNSUPPORTED", -8: "PIC_ERR_DEVICE"}

# Names the header declares; tests check the library exports each of them.
EXPORTS = ("pic_last_error", "pic_workspace_size", "pic_create", "pic_destroy", "pic_set_stream",
           "pic_add_particles", "pic_get_particles", "pic_set_deposit", "pic_add_source", "pic_probe_dft",
           "pic_step", "pic_sync", "pic_probe_read", "pic_get_field", "pic_set_field", "pic_get_stats",
           "pic_save", "pic_load", "pic_profile_steps", "pic_dft_fold_static", "pic_batch_create",
           "pic_batch_step", "pic_batch_sync", "pic_batch_destroy", "pic_probe_kw", "pic_get_tuning",
           "pic_set_tuning", "pic_tune", "pic_batch_tune", "pic_batch_set_lanes", "pic_batch_set_joint")


class pic_material(C.Structure):
    _fields_ = [("wp", C.c_double), ("gamma", C.c_double), ("eps_inf", C.c_double)]


class pic_config(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
                ("eps0", C.c_double), ("mu0", C.c_double),
                ("precision", C.c_int32), ("bc", C.c_int32 * 6),
                ("cpml_cells", C.c_int32), ("cpml_order", C.c_double), ("cpml_sigma_fac", C.c_double),
                ("cpml_kappa_max", C.c_double), ("cpml_alpha_max", C.c_double),
                ("material_id", C.POINTER(C.c_uint8)), ("materials", C.POINTER(pic_material)),
                ("n_materials", C.c_int32), ("max_particles", C.c_int64), ("max_probes", C.c_int32),
                ("max_freqs", C.c_int32), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("stream", C.c_void_p), ("flags", C.c_uint64)]


class pic_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_particles", C.c_int64), ("n_frozen", C.c_int64),
                ("device_error", C.c_int32), ("n_edge_classes", C.c_int32), ("kernel_launches", C.c_int64),
                ("field_path", C.c_int32), ("reserved", C.c_int32)]


class pic_tuning(C.Structure):
    _fields_ = [("dep_smem_bytes", C.c_int32), ("sort_every", C.c_int32), ("field_block", C.c_int32),
                ("field_path", C.c_int32)]


PIC_TUNE_MAX_CANDIDATES = 20


class pic_tune_report(C.Structure):
    _fields_ = [("best", pic_tuning), ("n", C.c_int32), ("cand", pic_tuning * PIC_TUNE_MAX_CANDIDATES),
                ("us_per_step", C.c_double * PIC_TUNE_MAX_CANDIDATES), ("steps", C.c_int64),
                ("best_lanes", C.c_int32), ("lanes", C.c_int32 * PIC_TUNE_MAX_CANDIDATES)]


class PicError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib.pic_last_error().decode() if _lib is not None else ""
        super().__init__(f"{where}: {ERRORS.get(code, code)} {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libpic (building it first if sources are newer).  Raises if the
    library cannot be built or loaded: there is no other implementation."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libpic not found at {path}")
    L = C.CDLL(path)
    h = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.pic_last_error.restype = C.c_char_p
    L.pic_workspace_size.argtypes = [C.POINTER(pic_config), C.POINTER(C.c_size_t)]
    L.pic_create.argtypes = [C.POINTER(pic_config), C.POINTER(h)]
    L.pic_destroy.argtypes = [h]
    L.pic_set_stream.argtypes = [h, C.c_void_p]
    L.pic_add_particles.argtypes = [h, C.c_int64, dp, dp, C.c_double, C.c_double, C.POINTER(C.c_int64)]
    L.pic_get_particles.argtypes = [h, dp, dp, C.POINTER(C.c_uint8)]
    L.pic_set_deposit.argtypes = [h, C.c_int]
    L.pic_add_source.argtypes = [h, C.c_int, C.POINTER(C.c_int64), C.c_double, C.c_double, C.c_double, C.c_double]
    L.pic_probe_dft.argtypes = [h, C.c_int, dp, C.c_uint32, C.c_int, dp]
    L.pic_step.argtypes = [h, C.c_int64]
    L.pic_sync.argtypes = [h]
    L.pic_probe_read.argtypes = [h, dp]
    L.pic_get_field.argtypes = [h, C.c_int, dp]
    L.pic_set_field.argtypes = [h, C.c_int, dp]
    L.pic_get_stats.argtypes = [h, C.POINTER(pic_stats)]
    L.pic_profile_steps.argtypes = [h, C.c_int64, dp]
    L.pic_get_tuning.argtypes = [h, C.POINTER(pic_tuning)]
    L.pic_set_tuning.argtypes = [h, C.POINTER(pic_tuning)]
    L.pic_tune.argtypes = [h, C.c_int32, C.POINTER(pic_tune_report)]
    L.pic_batch_tune.argtypes = [h, C.c_int32, C.POINTER(pic_tune_report)]
    L.pic_batch_set_lanes.argtypes = [h, C.c_int32]
    L.pic_batch_set_joint.argtypes = [h, C.c_int32]
    L.pic_save.argtypes = [h, C.c_char_p]
    L.pic_load.argtypes = [h, C.c_char_p]
    L.pic_dft_fold_static.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_uint32, C.c_void_p, C.c_int,
                                      C.c_int64, C.c_double, C.c_void_p, C.c_void_p]
    L.pic_probe_kw.argtypes = [h, C.c_int, C.c_int, C.c_int, dp, dp]
    L.pic_batch_create.argtypes = [C.c_int, C.POINTER(h), C.c_void_p, C.POINTER(h)]
    L.pic_batch_step.argtypes = [h, C.c_int64]
    L.pic_batch_sync.argtypes = [h]
    L.pic_batch_destroy.argtypes = [h]
    _lib = L
    return L


def _check(rc, where):
    if rc != PIC_OK:
        raise PicError(rc, where)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------- C names --
def pic_last_error() -> str:
    return load().pic_last_error().decode()


def pic_workspace_size(cfg: pic_config) -> int:
    n = C.c_size_t(0)
    _check(load().pic_workspace_size(C.byref(cfg), C.byref(n)), "pic_workspace_size")
    return n.value


def pic_create(cfg: pic_config) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().pic_create(C.byref(cfg), C.byref(h)), "pic_create")
    return h


def pic_destroy(h) -> None:
    _check(load().pic_destroy(h), "pic_destroy")


def pic_set_stream(h, stream: int | None) -> None:
    _check(load().pic_set_stream(h, C.c_void_p(stream or None)), "pic_set_stream")


def pic_add_particles(h, xyz: np.ndarray, u: np.ndarray, q_macro: float, m_macro: float) -> None:
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, 3)
    bad = C.c_int64(0)
    _check(load().pic_add_particles(h, x.shape[0], _dp(x), _dp(v), q_macro, m_macro, C.byref(bad)),
           "pic_add_particles")


def pic_get_particles(h, n: int):
    x = np.empty((n, 3)); u = np.empty((n, 3)); s = np.empty(n, dtype=np.uint8)
    _check(load().pic_get_particles(h, _dp(x), _dp(u), s.ctypes.data_as(C.POINTER(C.c_uint8))),
           "pic_get_particles")
    return x, u, s


def pic_set_deposit(h, on: bool) -> None:
    _check(load().pic_set_deposit(h, int(bool(on))), "pic_set_deposit")


def pic_add_source(h, comp, box, amp, t0, tau, f0=0.0) -> None:
    b = (C.c_int64 * 6)(*[int(v) for v in box])
    _check(load().pic_add_source(h, int(comp), b, amp, t0, tau, f0), "pic_add_source")


def pic_probe_dft(h, xyz, comp_mask, freqs) -> None:
    p = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    _check(load().pic_probe_dft(h, p.shape[0], _dp(p), int(comp_mask), f.size, _dp(f)), "pic_probe_dft")


def pic_step(h, nsteps: int) -> None:
    _check(load().pic_step(h, int(nsteps)), "pic_step")


def pic_sync(h) -> None:
    _check(load().pic_sync(h), "pic_sync")


def pic_probe_read(h, nprobe: int, nfreq: int) -> np.ndarray:
    out = np.empty(nprobe * 3 * nfreq * 2)
    _check(load().pic_probe_read(h, _dp(out)), "pic_probe_read")
    z = out.reshape(nprobe, 3, nfreq, 2)
    return z[..., 0] + 1j * z[..., 1]


def pic_probe_kw(h, comp: int, k, nfreq: int, axis: int = 0) -> np.ndarray:
    k = np.ascontiguousarray(k, dtype=np.float64)
    out = np.empty((k.size, nfreq))
    _check(load().pic_probe_kw(h, comp, axis, k.size, _dp(k), _dp(out)), "pic_probe_kw")
    return out


def pic_get_field(h, which: int, shape) -> np.ndarray:
    out = np.empty(int(np.prod(shape)))
    _check(load().pic_get_field(h, int(which), _dp(out)), "pic_get_field")
    return out.reshape(shape)


def pic_set_field(h, which: int, arr) -> None:
    a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
    _check(load().pic_set_field(h, int(which), _dp(a)), "pic_set_field")


def pic_get_stats(h) -> pic_stats:
    s = pic_stats()
    _check(load().pic_get_stats(h, C.byref(s)), "pic_get_stats")
    return s


def pic_save(h, path: str) -> None:
    _check(load().pic_save(h, os.fsencode(path)), "pic_save")


def pic_load(h, path: str) -> None:
    _check(load().pic_load(h, os.fsencode(path)), "pic_load")


def pic_profile_steps(h, nsteps: int, fused: bool = False) -> dict:
    """Per-step phase durations (us).  fused: the handle is on the fused field
    path (pic_stats.field_path 1), whose phases are named after what they run."""
    out = np.zeros(6)
    _check(load().pic_profile_steps(h, int(nsteps), _dp(out)), "pic_profile_steps")
    if fused:
        keys = ("field_pass", "push_deposit", "jf_correction", "step_tail", "dft_flush", "step")
    else:
        keys = ("update_H", "push_deposit", "update_E", "step_tail", "dft_flush", "step")
    return dict(zip(keys, out.tolist()))


def pic_get_tuning(h) -> tuple:
    """(dep_smem_bytes, sort_every, field_block, field_path)."""
    t = pic_tuning()
    _check(load().pic_get_tuning(h, C.byref(t)), "pic_get_tuning")
    return t.dep_smem_bytes, t.sort_every, t.field_block, t.field_path


def pic_set_tuning(h, dep_smem_bytes: int, sort_every: int, field_block: int = 256, field_path: int = 1) -> None:
    t = pic_tuning(int(dep_smem_bytes), int(sort_every), int(field_block), int(field_path))
    _check(load().pic_set_tuning(h, C.byref(t)), "pic_set_tuning")


def _report(r: pic_tune_report) -> dict:
    tup = lambda t: (t.dep_smem_bytes, t.sort_every, t.field_block, t.field_path)  # noqa: E731
    out = {"best": tup(r.best), "steps": r.steps,
           "candidates": [(tup(r.cand[i]), r.us_per_step[i]) for i in range(r.n)]}
    if r.best_lanes >= 0:
        out["best_lanes"] = r.best_lanes
        out["lanes"] = [r.lanes[i] for i in range(r.n)]
    return out


def pic_batch_set_lanes(b, lanes: int) -> None:
    _check(load().pic_batch_set_lanes(b, int(lanes)), "pic_batch_set_lanes")


def pic_batch_set_joint(b, joint: int) -> None:
    _check(load().pic_batch_set_joint(b, int(joint)), "pic_batch_set_joint")


def pic_tune(h, rounds: int = 1) -> dict:
    r = pic_tune_report()
    _check(load().pic_tune(h, int(rounds), C.byref(r)), "pic_tune")
    return _report(r)


def pic_batch_tune(b, rounds: int = 1) -> dict:
    r = pic_tune_report()
    _check(load().pic_batch_tune(b, int(rounds), C.byref(r)), "pic_batch_tune")
    return _report(r)


def pic_dft_fold_static(samples_ptr: int, count: int, np_: int, comp_mask: int, freq_ptr: int, nf: int,
                        first_step: int, dt: float, F_ptr: int, stream: int | None = None) -> None:
    """Allocation-free probe-DFT fold on caller device arrays (raw device
    addresses, e.g. ``tensor.data_ptr()``); see include/pic.h."""
    _check(load().pic_dft_fold_static(C.c_void_p(samples_ptr), int(count), int(np_), int(comp_mask),
                                      C.c_void_p(freq_ptr), int(nf), int(first_step), float(dt),
                                      C.c_void_p(F_ptr), C.c_void_p(stream or None)), "pic_dft_fold_static")


# ------------------------------------------------------------ convenience --
def pic_batch_create(handles, stream: int | None = None) -> C.c_void_p:
    arr = (C.c_void_p * len(handles))(*[hh.value if isinstance(hh, C.c_void_p) else hh for hh in handles])
    out = C.c_void_p()
    _check(load().pic_batch_create(len(handles), arr, C.c_void_p(stream) if stream else None, C.byref(out)),
           "pic_batch_create")
    return out


def pic_batch_step(b, nsteps: int) -> None:
    _check(load().pic_batch_step(b, int(nsteps)), "pic_batch_step")


def pic_batch_sync(b) -> None:
    _check(load().pic_batch_sync(b), "pic_batch_sync")


def pic_batch_destroy(b) -> None:
    _check(load().pic_batch_destroy(b), "pic_batch_destroy")


def make_config(w, precision=PIC_FP32, max_particles=None, max_probes=None, max_freqs=None,
                eps0=None, mu0=None, flags=0) -> tuple[pic_config, tuple]:
    """pic_config for a Workload; returns (cfg, keepalive) where keepalive
    holds the host arrays the config points to."""
    from . import workloads as W
    mat = np.ascontiguousarray(w.material, dtype=np.uint8)
    tab = (pic_material * len(w.table))(*[pic_material(*map(float, r)) for r in w.table])
    cfg = pic_config()
    cfg.nx, cfg.ny, cfg.nz = w.nx, w.ny, w.nz
    cfg.dx, cfg.dy, cfg.dz, cfg.dt = w.dx, w.dy, w.dz, w.dt
    cfg.eps0 = W.EPS0 if eps0 is None else eps0
    cfg.mu0 = W.MU0 if mu0 is None else mu0
    cfg.precision = precision
    cfg.bc = (C.c_int32 * 6)(*w.bc)
    cfg.cpml_cells = w.cpml_cells
    cfg.cpml_order = w.cpml_order
    cfg.cpml_sigma_fac = w.cpml_sigma_fac
    cfg.cpml_kappa_max = w.cpml_kappa_max
    cfg.cpml_alpha_max = w.cpml_alpha_max
    cfg.material_id = mat.ctypes.data_as(C.POINTER(C.c_uint8))
    cfg.materials = tab
    cfg.n_materials = len(w.table)
    cfg.max_particles = w.nparticles if max_particles is None else max_particles
    nprobe = 0 if w.probes is None else len(w.probes)
    nfreq = 0 if w.freqs is None else len(w.freqs)
    cfg.max_probes = nprobe if max_probes is None else max_probes
    cfg.max_freqs = nfreq if max_freqs is None else max_freqs
    cfg.flags = int(flags)
    return cfg, (mat, tab)


class Simulation:
    """One libpic handle for a Workload, with PyTorch-owned device memory."""

    def __init__(self, w, precision=PIC_FP32, particles=True, probes=True, torch_memory=True,
                 stream=None, **cap):
        import torch
        self.w = w
        self.shape = (w.nz, w.ny, w.nx)
        cfg, self._keep = make_config(w, precision, **cap)
        self._ws = None
        if torch_memory:
            nbytes = pic_workspace_size(cfg)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            aligned = (base + 255) & ~255
            cfg.workspace = C.c_void_p(aligned)
            cfg.workspace_bytes = nbytes
        if stream is None:
            self._stream = torch.cuda.Stream()
        else:
            self._stream = stream
        cfg.stream = C.c_void_p(self._stream.cuda_stream)
        self.h = pic_create(cfg)
        self.n = 0
        self.nprobe = 0
        self.nfreq = 0
        if particles and w.nparticles:
            self.add_particles(w.xyz, w.u, w.q_macro, w.m_macro)
        if probes and w.probes is not None and w.freqs is not None:
            self.probe_dft(w.probes, w.freqs, w.comp_mask)

    @property
    def stream(self):
        return self._stream

    def add_particles(self, xyz, u, q, m):
        pic_add_particles(self.h, xyz, u, q, m)
        self.n += len(xyz)

    def probe_dft(self, xyz, freqs, mask=0b111):
        pic_probe_dft(self.h, xyz, mask, freqs)
        self.nprobe, self.nfreq = len(np.asarray(xyz).reshape(-1, 3)), len(freqs)

    def step(self, n=1):
        pic_step(self.h, n)

    def sync(self):
        pic_sync(self.h)

    def field(self, which):
        return pic_get_field(self.h, which, self.shape)

    def set_field(self, which, arr):
        pic_set_field(self.h, which, arr)

    def particles(self):
        return pic_get_particles(self.h, self.n)

    def probe_read(self):
        return pic_probe_read(self.h, self.nprobe, self.nfreq)

    def probe_kw(self, comp, k, axis=0):
        return pic_probe_kw(self.h, comp, k, self.nfreq, axis)

    def stats(self):
        return pic_get_stats(self.h)

    def profile(self, nsteps):
        return pic_profile_steps(self.h, nsteps, fused=self.stats().field_path == 1)

    @property
    def tuning(self):
        return pic_get_tuning(self.h)

    def set_tuning(self, dep_smem_bytes, sort_every, field_block=256, field_path=1):
        pic_set_tuning(self.h, dep_smem_bytes, sort_every, field_block, field_path)

    def tune(self, rounds=1):
        """Time the deposit box, sort interval and field block candidates on
        real steps of this simulation and keep the fastest (the simulation
        advances)."""
        return pic_tune(self.h, rounds)

    def save(self, path):
        pic_save(self.h, path)

    def load(self, path):
        pic_load(self.h, path)

    def close(self):
        if getattr(self, "h", None):
            pic_destroy(self.h)
            self.h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Simulations stepped together through one pic_batch."""

    def __init__(self, sims, stream=None):
        import torch
        self.sims = list(sims)
        self._stream = stream if stream is not None else torch.cuda.Stream()
        self.b = pic_batch_create([x.h for x in self.sims], self._stream.cuda_stream)

    @property
    def stream(self):
        return self._stream

    def step(self, n):
        pic_batch_step(self.b, n)

    def sync(self):
        pic_batch_sync(self.b)

    def tune(self, rounds=1):
        """pic_tune over the whole batch (every instance advances)."""
        return pic_batch_tune(self.b, rounds)

    def set_lanes(self, lanes):
        pic_batch_set_lanes(self.b, lanes)

    def set_joint(self, joint):
        """1: one joint fused field pass per step over the instances that take
        the fused pass; 0: every instance on a branch of its own."""
        pic_batch_set_joint(self.b, int(joint))

    def close(self):
        if getattr(self, "b", None):
            pic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
