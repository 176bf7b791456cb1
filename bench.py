"""Benchmark of the PIC/FDTD-Drude time step (one JSON line on rank 0).

A "step" is one full time step of the hot path: H update (+CPML), electron
push + Esirkepov deposit, Drude-ADE + Ampere E update (+CPML), probe sampling
and (every 64 steps) the probe-DFT flush.  Workload (default, the largest
single-GPU configuration): 768x256x256 cells, dx = 1 nm, 10 nm silver film,
1e6 electrons at 30 keV, one probe x 2001 frequencies, FP32 state with FP64
DFT accumulators.  --workload c2 is the paper-scale 384x128x128 run.

Metric: cell-updates per second (Gcell-upd/s) over the whole job; with
--gpus N (torchrun) every rank steps its own independent instance (weak
scaling, no data-path collective).

--impl reference times the FP64 CPU oracle (the deliberately plain reference
implementation) on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4096)
    ap.add_argument("--warmup", type=int, default=128)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "sweep", "adjoint"], default="c3",
                    help="sweep: 48 uneven film instances stepped through one batch graph vs one after another; "
                         "adjoint: gradient of the plasmon probe energy (192x96x96, 4000 steps) vs the plain step")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default launch settings instead of choosing them with pic_tune")
    ap.add_argument("--tuning", default=None, metavar="DEP_SMEM_BYTES,SORT_EVERY[,FIELD_BLOCK[,FIELD_PATH]]",
                    help="use these launch settings instead of running pic_tune (e.g. 8192,32,256,1)")
    ap.add_argument("--ref-seconds", type=float, default=20.0,
                    help="target CPU seconds of the oracle sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_rate(ms_local, units_per_rank, dist=None, device="cpu"):
    """(slowest rank's milliseconds, whole-job units per second): every rank
    processed units_per_rank units; the job took as long as its slowest rank
    (all-reduce MAX).  Without a process group: this process alone."""
    ms, world = float(ms_local), 1
    if dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, world = float(t.item()), dist.get_world_size()
    return ms, units_per_rank * world / (ms / 1e3)


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    v = d[k]
                    if isinstance(v, dict):
                        v = v.get("value", v.get("gbs"))
                    return float(v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(w, real_bytes):
    """Bytes each field kernel must move per launch at minimum (one read of
    every input it needs, one write of every output), counted from the
    workload geometry: per cell 9 state values (H: read E and H, write H;
    E: read H and E, write E); for E, 3 bytes of edge classes per cell of the
    planes that hold metal edges (planes of one non-metal material need
    none); per cell and absorbing-slab axis 2 psi values read and written;
    per metal edge J_p read and written."""
    N = w.ncells
    L = w.cpml_cells
    n = (w.nx, w.ny, w.nz)
    # cells inside k CPML slabs (psi read+write of 2 components per slab axis)
    inside = []
    for a in range(3):
        has = 0 in (w.bc[2 * a], w.bc[2 * a + 1])
        m = np.zeros(n[a], bool)
        if has:
            m[:L] = True
            m[n[a] - L:] = True
        inside.append(m)
    slab_cells = 0
    for a in range(3):
        other = N // n[a]
        slab_cells += int(inside[a].sum()) * other
    psi = slab_cells * 2 * 2 * real_bytes  # 2 components, read + write
    # metal edges (any of the four cells around the edge has wp > 0): J_p read + write
    wp = w.table[:, 0][w.material] > 0
    metal_edges = 0
    metal_planes = np.zeros(w.nz, bool)
    for c in range(3):
        m = wp.copy()
        for ax in ((c + 1) % 3, (c + 2) % 3):
            m = m | np.roll(m, 1, axis=2 - ax)
        metal_edges += int(m.sum())
        metal_planes |= m.any(axis=(1, 2))
    class_bytes = int(metal_planes.sum()) * w.nx * w.ny * 3
    h_bytes = N * 9 * real_bytes + psi
    e_bytes = N * 9 * real_bytes + class_bytes + psi + metal_edges * 2 * real_bytes
    # the fused pass reads E, H once and writes them once (12 values per cell),
    # with both updates' psi and the E update's classes and J_p
    f_bytes = N * 12 * real_bytes + class_bytes + 2 * psi + metal_edges * 2 * real_bytes
    return {"update_H": h_bytes, "update_E": e_bytes, "field_pass": f_bytes, "metal_edges": metal_edges,
            "slab_cells": slab_cells, "class_bytes": class_bytes}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.out = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source and on this workload; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        import hashlib
        for d in json.load(open(p))["entries"]:
            src = os.path.join(ROOT, "paper_1505_04007_gb300", "csrc", d["source"])
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            k = d["kernels"].get(kernel)
            if k is not None and d.get("source_sha") == sha and d.get("workload_key") == workload:
                return float(k["dram_bytes_per_launch_full"])
        return None
    except Exception:
        return None


def cpu_reference(w, target_s, warm=1, single=True):
    """Time the FP64 oracle on the host cores over a bounded number of full
    steps of the workload (OpenMP over cells on every core; particles serial),
    then, with `single`, one more full step on one thread.  Returns
    (Gcell-upd/s, steps, threads, seconds, single-thread Gcell-upd/s or None,
    single-thread seconds per step or None)."""
    from oracle import oracle as O
    threads = O.set_threads(len(os.sched_getaffinity(0)))
    o = O.from_workload(w)
    o.step(warm)
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    nsteps = max(1, int(target_s / max(one, 1e-3)) - 1)
    t0 = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t0
    v1 = s1 = None
    if single:
        O.set_threads(1)
        t0 = time.perf_counter()
        o.step(1)
        s1 = time.perf_counter() - t0
        v1 = w.ncells / s1 / 1e9
        O.set_threads(threads)
    o.close()
    return w.ncells * nsteps / dt / 1e9, nsteps, threads, dt, v1, s1


def batched_and_sequential(ws, warm, steps, clocks=None, tune=False):
    """Time `steps` steps (after `warm`) of the instances ws stepped through one
    pic_batch, then fresh copies of the same instances stepped alone, one after
    another, over the same steps.  With `tune`, pic_batch_tune first chooses the
    launch settings on the batch (its steps count towards the warm-up; the
    sequential copies get the same settings).  Returns (ms_batch, ms_seq,
    launches, clock record or None, tuning or None, steps before the timed
    region)."""
    import torch
    from paper_1505_04007_gb300 import pic
    sims = [pic.Simulation(w, pic.PIC_FP32) for w in ws]
    b = pic.Batch(sims)
    rep = b.tune(rounds=1) if tune else None
    before = warm + (rep["steps"] if rep else 0)
    b.step(warm)
    b.sync()
    if clocks is not None:
        clocks.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0 = sum(x.stats().kernel_launches for x in sims)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    b.sync()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks is not None else None
    launches = sum(x.stats().kernel_launches for x in sims) - k0
    # the fused passes as one joint pass per step against a branch per
    # instance: the next `steps` steps both ways, joint last
    joint = None
    if sum(x.stats().field_path for x in sims) >= 2:
        ms = {}
        for j in (0, 1):
            b.set_joint(j)
            b.step(64)  # capture under the setting, outside the timed steps
            b.sync()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(b.stream)
            b.step(steps)
            a1.record(b.stream)
            b.sync()
            ms[j] = a0.elapsed_time(a1) / steps
        joint = {"joint_ms_per_step": ms[1], "branches_ms_per_step": ms[0],
                 "steps": f"branches {before + steps + 64}..{before + 2 * steps + 64}, joint "
                          f"{before + 2 * steps + 128}..{before + 3 * steps + 128} (64 untimed steps before each)"}
    b.close()
    for x in sims:
        x.close()
    def sequential(path=None):
        ms_seq = 0.0
        for w in ws:
            x = pic.Simulation(w, pic.PIC_FP32)
            if rep:
                x.set_tuning(*rep["best"])
            if path is not None:
                t = x.tuning
                x.set_tuning(t[0], t[1], t[2], path)
            x.step(before)
            x.sync()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(x.stream)
            x.step(steps)
            a1.record(x.stream)
            x.sync()
            ms_seq += a0.elapsed_time(a1)
            x.close()
        return ms_seq

    ms_seq = sequential()
    if joint is not None:  # alone, a small grid steps faster on the split updates
        joint["sequential_split_ms_per_step"] = sequential(0) / steps
    return ms_batch, ms_seq, launches, clk, ((*rep["best"], rep["best_lanes"]) if rep else None), before, joint


def bench_sweep(args):
    """Batched stepping of the 48-instance sweep against the same instances
    stepped one after another (same GPU, same FP32 arithmetic); the same
    comparison on the eight quasi-2D grids of the Table 1 series, each far too
    small to fill the GPU."""
    import torch
    from paper_1505_04007_gb300 import workloads as W
    torch.cuda.set_device(0)
    ws = W.sweep()
    warm = max(64, args.warmup // 64 * 64)
    tune_steps = 0 if args.no_tune else (12 + 5) * 64  # pic_batch_tune, one round (5 lane candidates for 48)
    # whole 64-step blocks within the 4000 steps
    steps = max(64, min(args.steps, ws[0].nsteps - warm - tune_steps) // 64 * 64)
    cells = sum(w.ncells for w in ws)
    ms_batch, ms_seq, launches, clk, tuned, before, joint = batched_and_sequential(ws, warm, steps, ClockSampler(0),
                                                                                   tune=not args.no_tune)
    value = cells * steps / (ms_batch / 1e3) / 1e9
    seq = cells * steps / (ms_seq / 1e3) / 1e9
    t1 = W.table1(65536)
    t1_steps = 1024
    t1_cells = sum(w.ncells for w in t1)
    tb, ts, _, _, t1_tuned, t1_before, _ = batched_and_sequential(t1, 128, t1_steps, tune=not args.no_tune)
    line = {"metric": "Gcell-upd/s", "value": value, "unit": "Gcell-upd/s", "n_gpus": 1, "steps": steps,
            "warmup": warm, "ms_per_step": ms_batch / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"sweep: {len(ws)} instances, {cells / 1e6:.1f}M cells in all "
                                   f"(128..320 x 64..128 x 64..96, films 10-60 nm, 10-100 keV, gaps 5-20 nm, "
                                   f"2e4 e- each), steps {before}..{before + steps} of the 4000-step sweep timed",
                       "parallelism": ("one batch graph: per step the instances' own work on their own streams "
                                       "around one joint fused field pass over all of them (four launches)"
                                       if joint else "one batch graph (one branch per instance)"),
                       "l2": "state larger than the 129 MB L2 (no flush)",
                       "launch_settings": ({"dep_smem_bytes": tuned[0], "sort_every": tuned[1],
                                            "field_block": tuned[2], "field_path": tuned[3],
                                            "lanes": tuned[4] or "all",
                                            "chosen_by": f"pic_batch_tune, 1 round on steps 0..{tune_steps}"}
                                           if tuned else "library defaults (dep_smem_bytes 4096, sort_every 16, field_block 256)")},
            "sequential": {"value": seq, "unit": "Gcell-upd/s", "ms_per_step": ms_seq / steps,
                           "note": "fresh copies of the same instances over the same step range, each stepped "
                                   "alone (own 64-step graphs), one after another"},
            "batched_vs_sequential": value / seq,
            "joint_pass": joint,
            "small_grids": {"workload": f"Table 1 series: {len(t1)} quasi-2D films, 2048 x 2 x 82..147 cells "
                                        f"({t1_cells / 1e6:.2f}M in all), 1024 e- each, "
                                        f"steps {t1_before}..{t1_before + t1_steps}",
                            "launch_settings": t1_tuned,
                            "batched": t1_cells * t1_steps / (tb / 1e3) / 1e9,
                            "sequential": t1_cells * t1_steps / (ts / 1e3) / 1e9,
                            "unit": "Gcell-upd/s", "batched_vs_sequential": ts / tb},
            "gpu_launches": launches, "clocks": clk}
    # the field updates of all instances per batched step against the copy rate
    # (push, deposit, probe and sort bytes left out: a lower bound on the rate)
    peak, src = measured_peak()
    # fused grids (CPML on every face, nx a multiple of 4): one fused pass per step
    fb = sum(ab["field_pass"] for ab in (algorithmic_bytes(w, 4) for w in ws))
    ach = fb / (ms_batch / steps * 1e-3) / 1e9
    line["roofline"] = {"bound": "hbm", "kernel": "fused field passes of all 48 instances (one batched step)",
                        "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "peak_source": src, "traffic": None, "algorithmic_bytes_per_launch": fb,
                        "note": "per-step time of the whole batched step (particles included)"}
    print(json.dumps(line), flush=True)


def adjoint_bytes(cfg, elem):
    """Algorithmic DRAM bytes of one forward and one backward step of the
    film study: every field, adjoint and psi value read and written once per
    update (E, H, their adjoints: 9 values per cell per update; psi: 2 values
    rw per slab cell and axis), the design-edge map on the planes that hold
    design edges, and per design edge J (rw), bJ and the stored E^n, J^n
    (written forward, read backward), plus the FP64 dL/dbJ, dL/dkJ (rw)
    backward."""
    n = (cfg.nx, cfg.ny, cfg.nz)
    N = n[0] * n[1] * n[2]
    slab = sum(N * 2 * cfg.cpml_cells // n[a] for a in range(3))
    k0, k1 = cfg.design_k0, cfg.design_k1
    planes = min(cfg.nz, k1 + 1) - max(0, k0 - 1)
    edges = n[0] * n[1] * (2 * (k1 - k0 + 1) + (k1 - k0))
    common = 18 * elem * N + 8 * elem * slab + 3 * 4 * n[0] * n[1] * planes + 5 * elem * edges
    return common, common + 32 * edges


def bench_adjoint(args):
    """Forward + adjoint of the film study (192x96x96 cells, 30 nm design
    slab, 4000 steps, FP32 state) against the plain FP32 step of the same
    grid, with the FP32 gradient's error against the FP64 one."""
    import torch
    import numpy as np
    from paper_1505_04007_gb300 import adjoint as A
    from paper_1505_04007_gb300 import pic
    from paper_1505_04007_gb300 import workloads as W
    torch.cuda.set_device(0)
    wp, gamma = W.TABLE1_WP, W.TABLE1_GAMMA
    res = {}
    for prec in ("fp32", "fp64"):
        cfg = A.film_config(precision=pic.PIC_FP32 if prec == "fp32" else pic.PIC_FP64)
        st = A.Adjoint(cfg)
        mask = np.random.default_rng(1505).uniform(0.2, 0.8, st.n)
        st.forward(mask, wp, gamma)  # warm-up
        t0 = time.perf_counter()
        loss = st.forward(mask, wp, gamma)
        t1 = time.perf_counter()
        dm, dwp, dga = st.backward()
        t2 = time.perf_counter()
        res[prec] = dict(loss=loss, dm=dm, dwp=dwp, dga=dga, fwd=t1 - t0, bwd=t2 - t1, cfg=cfg)
        st.close()
    cfg = res["fp32"]["cfg"]
    cells = cfg.nx * cfg.ny * cfg.nz
    steps = cfg.nsteps
    # the plain FP32 step of the same grid (film of the design slab at m = 1, no electrons)
    w = W.Workload(name="adjoint_grid", nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, dx=cfg.dx, dy=cfg.dx, dz=cfg.dx,
                   dt=cfg.dt, nsteps=steps)
    w.cpml_alpha_max = cfg.cpml_alpha_max
    w.material = W.slab_material(cfg.nx, cfg.ny, cfg.nz, cfg.design_k0, cfg.design_k1)
    w.table = np.array([[0.0, 0.0, 1.0], [wp, gamma, 1.0]])
    w.xyz, w.u = np.zeros((0, 3)), np.zeros((0, 3))
    w.probes = np.array([list(cfg.probe)])
    w.freqs = np.array([cfg.omega0 / (2 * np.pi)])
    # (its launch settings chosen by pic_tune, as the plain bench does: on a
    # grid this small the split field updates beat the fused pass)
    sim = pic.Simulation(w, pic.PIC_FP32, particles=False)
    plain_tuning = sim.tune(rounds=1)["best"]
    sim.step(256)
    sim.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    sim.step(steps)
    e1.record(sim.stream)
    sim.sync()
    plain_s = e0.elapsed_time(e1) / 1e3
    sim.close()
    r32, r64 = res["fp32"], res["fp64"]
    line = {"metric": "Gcell-upd/s", "value": cells * steps / (r32["fwd"] + r32["bwd"]) / 1e9, "unit": "Gcell-upd/s",
            "n_gpus": 1, "steps": steps, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"adjoint: {cfg.nx}x{cfg.ny}x{cfg.nz} cells, design slab planes "
                                   f"[{cfg.design_k0}, {cfg.design_k1}) (30 nm), rigid 40 keV bunch, "
                                   f"{steps} steps, loss |F(wp/sqrt2)|^2 of Ez",
                       "note": "value counts one forward + one backward step as one cell-update; host wall clock"},
            "forward_s": r32["fwd"], "backward_s": r32["bwd"], "plain_step_s": plain_s,
            "plain_step_launch_settings": list(plain_tuning),
            "forward_plus_backward_vs_plain": (r32["fwd"] + r32["bwd"]) / plain_s,
            "fp32_vs_fp64": {"loss_rel": abs(r32["loss"] / r64["loss"] - 1),
                             "dmask_rel_l2": float(np.linalg.norm(r32["dm"] - r64["dm"]) / np.linalg.norm(r64["dm"])),
                             "dwp_rel": abs(r32["dwp"] / r64["dwp"] - 1), "dgamma_rel": abs(r32["dga"] / r64["dga"] - 1)},
            "fp64_forward_s": r64["fwd"], "fp64_backward_s": r64["bwd"]}
    # checkpoint mode: field states every 64 steps, segments recomputed in the backward run
    cfg_c = A.film_config(precision=pic.PIC_FP32)
    cfg_c.flags = 2
    st = A.Adjoint(cfg_c)
    mask = np.random.default_rng(1505).uniform(0.2, 0.8, st.n)
    st.forward(mask, wp, gamma)
    t0 = time.perf_counter()
    loss_c = st.forward(mask, wp, gamma)
    t1 = time.perf_counter()
    dm_c, _, _ = st.backward()
    t2 = time.perf_counter()
    st.close()
    line["checkpoint_mode"] = {
        "forward_s": t1 - t0, "backward_s": t2 - t1,
        "forward_plus_backward_vs_plain": (t2 - t0) / plain_s,
        "vs_stored_steps": {"loss_equal": loss_c == r32["loss"],
                            "dmask_rel_l2": float(np.linalg.norm(dm_c - r32["dm"]) / np.linalg.norm(r32["dm"]))}}
    peak, src = measured_peak()
    fb, bb = adjoint_bytes(cfg, 4)
    f_gbs = fb / (r32["fwd"] / steps) / 1e9
    b_gbs = bb / (r32["bwd"] / steps) / 1e9
    line["roofline"] = {"bound": "hbm", "kernel": "adjoint backward step (k_adj_E + k_adj_H)",
                        "achieved": b_gbs, "peak": peak, "unit": "GB/s", "frac": b_gbs / peak,
                        "peak_source": src, "traffic": None, "algorithmic_bytes_per_launch": bb,
                        "forward": {"achieved": f_gbs, "frac": f_gbs / peak, "algorithmic_bytes_per_step": fb},
                        "note": "per-step durations from the host wall clock of whole 4000-step runs"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "adjoint":
        if int(os.environ.get("RANK", "0")) == 0 and args.impl == "ours":
            bench_adjoint(args)
        return
    if args.workload == "sweep":
        if int(os.environ.get("RANK", "0")) == 0 and args.impl == "ours":
            bench_sweep(args)
        return
    rank, world, local = dist_env()
    from paper_1505_04007_gb300 import workloads as W
    mk = W.WORKLOADS[args.workload]
    w = mk()
    desc = (f"{args.workload}: {w.nx}x{w.ny}x{w.nz} cells dx={w.dx*1e9:g}nm, film planes {w.info['film_cells']}, "
            f"{w.nparticles} e- at {w.info['kev']:g} keV, {len(w.probes)} probes x {len(w.freqs)} freqs, CPML 8")

    if args.impl == "reference":
        if rank != 0:
            return
        v, nst, thr, secs, _, _ = cpu_reference(w, args.ref_seconds, single=False)
        line = {"impl": "reference", "metric": "Gcell-upd/s", "value": v, "unit": "Gcell-upd/s",
                "n_gpus": args.gpus, "steps": nst, "warmup": 1, "ms_per_step": secs / nst * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": desc, "parallelism": "none (host cores)"},
                "cpu_baseline": {"value": v, "unit": "Gcell-upd/s", "cores": thr, "kind": "oracle",
                                 "sample": f"{nst} full time steps of the workload (of the {args.steps} requested), "
                                           f"FP64 oracle, OpenMP over cells, particles serial"},
                "e2e": {"value": v, "unit": "Gcell-upd/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_1505_04007_gb300 import pic
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prec = pic.PIC_FP32 if args.precision == "fp32" else pic.PIC_FP64
    real = 4 if prec == pic.PIC_FP32 else 8
    stream = torch.cuda.Stream()
    sim = pic.Simulation(w, prec, stream=stream)
    state_mb = sim._ws.numel() / 1e6 if sim._ws is not None else float("nan")
    l2_note = ("state larger than the 129 MB L2 (no flush)" if state_mb > 129.0 else
               f"state ({state_mb:.0f} MB) fits in the 129 MB L2: an L2-resident latency figure, not an HBM rate")
    tuned = None
    if args.tuning:
        vals = [int(v) for v in args.tuning.split(",")]
        sim.set_tuning(*vals)
        dep, every, blk, fpath = sim.tuning
        tuned = {"dep_smem_bytes": dep, "sort_every": every, "field_block": blk, "field_path": fpath,
                 "chosen_by": "--tuning"}
    elif not args.no_tune:  # launch settings chosen on this workload's own steps, before the warm-up
        rep = sim.tune(rounds=2)
        tuned = {"dep_smem_bytes": rep["best"][0], "sort_every": rep["best"][1], "field_block": rep["best"][2],
                 "field_path": rep["best"][3],
                 "chosen_by": f"pic_tune, 2 rounds on steps 0..{rep['steps']} (before the warm-up)"}
    # Warm-up: at least the W steps asked for, then on to a 64-step block
    # boundary, then the timed pattern twice, each followed by the steps to
    # the next boundary (a partial-block run is captured into a graph on its
    # second use, here, not in the timed region), so the timed steps replay
    # exactly the graphs a user's repeated pic_step(K) from a block boundary
    # replays.
    s0 = sim.stats().step

    def to_boundary(extra=0):
        done = sim.stats().step
        sim.step(extra + (-(done + extra)) % 64)

    to_boundary(args.warmup)
    for _ in range(2):
        sim.step(args.steps)
        to_boundary()
    sim.sync()
    warm_run = sim.stats().step - s0

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ------------------------------------------------ timed region (device)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k0 = sim.stats().kernel_launches
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    sim.sync()
    ms, rate = job_rate(ms, w.ncells * args.steps, dist, "cuda")
    cells_total = w.ncells * args.steps * world
    value = rate / 1e9
    launches = sim.stats().kernel_launches - k0  # counted by the library (graph replays count their kernels)

    # ------------------------------ per-kernel durations (CUDA events, live)
    prof = sim.profile(min(args.steps, 1024))
    ab = algorithmic_bytes(w, real)
    peak, peak_kind = measured_peak()
    if "field_pass" in prof:  # fused path: E^{n+1} and H^{n+3/2} in one pass
        dom = "field_pass"
    else:
        dom = "update_E" if prof["update_E"] >= prof["update_H"] else "update_H"
    achieved = ab[dom] / (prof[dom] * 1e-6) / 1e9
    traffic = traffic_for(dom, args.workload)
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} copy bandwidth",
            "traffic": traffic, "algorithmic_bytes_per_launch": ab[dom],
            "achieved_basis": "algorithmic bytes per launch / live CUDA-event duration (the 60% target is "
                              "judged on this figure)",
            "kernel_us": {k: round(v, 3) for k, v in prof.items()}}
    if traffic:
        # the same duration against the DRAM bytes ncu counted (cold, serialised
        # launches; part of the reuse between kernels stays in the 129 MB L2)
        roof["dram_achieved"] = traffic / (prof[dom] * 1e-6) / 1e9
        roof["dram_frac"] = roof["dram_achieved"] / peak
    sim.close()

    # -------------------------------------------- end-to-end through the API
    e2e = None
    if not args.no_e2e:
        barrier()
        t0 = time.perf_counter()
        s2 = pic.Simulation(w, prec, stream=stream)
        tc = time.perf_counter()
        if tuned is not None:
            s2.set_tuning(tuned["dep_smem_bytes"], tuned["sort_every"], tuned["field_block"], tuned["field_path"])
        ta = time.perf_counter()
        s2.step(args.steps)
        spec = s2.probe_read()
        t1 = time.perf_counter()
        s2.close()
        ms_e2e, _ = job_rate((t1 - t0) * 1e3, w.ncells * args.steps, dist, "cuda")
        secs = ms_e2e / 1e3
        h2d = w.ncells + w.nparticles * 3 * 2 * 8 + len(w.probes) * 24 + len(w.freqs) * 8
        d2h = spec.size * 16
        e2e = {"value": cells_total / secs / 1e9, "unit": "Gcell-upd/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "pic_create (material tables, upload) + particles + probes + steps + spectrum read",
               "create_ms": (tc - t0) * 1e3, "setup_ms": (ta - t0) * 1e3, "steps_and_read_ms": (t1 - ta) * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, nst, thr, secs, v1, s1 = cpu_reference(w, args.ref_seconds)
        cpu = {"value": v, "unit": "Gcell-upd/s", "cores": thr, "kind": "oracle",
               "sample": f"{nst} full time steps of the same workload (from step 1), FP64, {secs:.1f} s on "
                         f"{thr} threads",
               "single_thread": {"value": v1, "unit": "Gcell-upd/s", "cores": 1,
                                 "sample": f"one more full step on one thread, {s1:.1f} s"}}

    if rank == 0:
        line = {"metric": "Gcell-upd/s", "value": value, "unit": "Gcell-upd/s", "n_gpus": world,
                "steps": args.steps, "warmup": warm_run, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == pic.PIC_FP32 else "f64", "data": "synthetic",
                "config": {"workload": desc, "global_batch": world, "parallelism": f"replicas x{world}",
                           "l2": l2_note,
                           "warmup_steps": f"{warm_run} untimed steps after tuning: the {args.warmup} asked for, "
                                           f"rounded up to a 64-step block boundary, then twice the {args.steps} "
                                           f"timed steps and on to the next boundary",
                           "particle_pushes_per_s": w.nparticles * args.steps * world / (ms / 1e3),
                           "launch_settings": tuned or "library defaults (dep_smem_bytes 4096, sort_every 16, "
                                                       "field_block 256)"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
