"""Batched stepping (pic_batch): several independent film instances stepped
through one captured graph must each give what the FP64 oracle gives for that
instance alone (same tolerances as the single-instance parity tests: rel-L2
<= 1e-10 for an FP64 instance, <= 2e-5 for FP32; probe spectra likewise).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04007_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ETA0 = (W.MU0 / W.EPS0) ** 0.5

# small uneven grids, a few hundred electrons each: the oracle runs them in seconds
SMALL = dict(sizes=((64, 96), (32, 48), (48, 64)), nparticles=384)


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


def rel_l2(a, b):
    nb = np.sqrt(sum((x ** 2).sum() for x in b))
    na = np.sqrt(sum(((x - y) ** 2).sum() for x, y in zip(a, b)))
    return na / nb if nb > 0 else na


def fields_of(getter):
    return [getter(c) for c in range(3)] + [ETA0 * getter(3 + c) for c in range(3)]


def check(o, s, tol):
    f = rel_l2(fields_of(s.field), fields_of(o.get_field))
    p = rel_l2([s.probe_read()], [o.probe_read()])
    assert f <= tol and p <= tol, (f, p)
    return f, p


def test_batch_fp32_matches_oracle(P):
    ws = W.sweep(n=3, seed=7, nsteps=128, **SMALL)
    sims = [P.Simulation(w, P.PIC_FP32) for w in ws]
    b = P.Batch(sims)
    b.step(128)  # two whole blocks through the batch graph
    b.sync()
    for w, s in zip(ws, sims):
        o = O.from_workload(w)
        o.step(128)
        check(o, s, 2e-5)
        assert s.stats().step == 128
    b.close()


def test_batch_mixed_precision_with_remainder(P):
    ws = W.sweep(n=2, seed=9, nsteps=80, **SMALL)
    sims = [P.Simulation(ws[0], P.PIC_FP64), P.Simulation(ws[1], P.PIC_FP32)]
    b = P.Batch(sims)
    b.step(64 + 13)  # one block through the graph, then 13 steps per instance
    b.sync()
    for w, s, tol in zip(ws, sims, (1e-10, 2e-5)):
        o = O.from_workload(w)
        o.step(77)
        check(o, s, tol)
    b.close()


def test_batch_recaptures_after_change(P):
    ws = W.sweep(n=2, seed=5, nsteps=192, **SMALL)
    sims = [P.Simulation(w, P.PIC_FP32) for w in ws]
    orcs = [O.from_workload(w) for w in ws]
    b = P.Batch(sims)
    b.step(64)
    P.pic_set_deposit(sims[1].h, False)  # invalidates the captured steps of instance 1
    orcs[1].step(64)
    orcs[1].set_deposit(False)
    orcs[0].step(64)
    b.step(128)
    b.sync()
    for o, s in zip(orcs, sims):
        o.step(128)
        check(o, s, 2e-5)
    b.close()


def sources_for(w):
    c = (w.nx // 2, w.ny // 2, w.nz // 2)
    return [(2, (c[0], c[0] + 1, c[1], c[1] + 1, c[2], c[2] + 1), 1e18, 30 * w.dt, 8 * w.dt, 0.0),
            (1, (4, 9, 3, 6, c[2] - 2, c[2] - 1), 4e17, 36 * w.dt, 9 * w.dt, 1.2e15)]  # inside the x and y slabs


def test_joint_pass_equals_separate_branches(P):
    """FP32 instances that take the fused pass step through ONE joint field
    pass per step (pic_batch_set_joint 1, the default); the same instances as
    separate branches (0) give the same fields up to FP32 rounding (the joint
    kernels are compiled separately, and the compiler may contract a product
    and a sum into one FMA differently: rel-L2 <= 1e-6 between the two), and
    both match the oracle."""
    ws = W.sweep(n=3, seed=11, nsteps=128, **SMALL)
    runs = []
    for joint in (1, 0):
        sims = [P.Simulation(w, P.PIC_FP32, particles=False) for w in ws]
        for w, s in zip(ws, sims):
            assert s.stats().field_path == 1
            for src in sources_for(w):
                P.pic_add_source(s.h, *src)
        b = P.Batch(sims)
        b.set_joint(joint)
        b.step(128)
        b.sync()
        runs.append(sims)
        b.close()
    for w, sj, sb in zip(ws, *runs):
        d = rel_l2(fields_of(sj.field), fields_of(sb.field))
        dj = rel_l2([sj.field(P.PIC_JPX + c) for c in range(3)], [sb.field(P.PIC_JPX + c) for c in range(3)])
        o = O.from_workload(w, with_particles=False)
        for src in sources_for(w):
            o.add_source(*src)
        o.step(128)
        fj, _ = check(o, sj, 2e-5)
        fb, _ = check(o, sb, 2e-5)
        assert d <= 1e-6 and dj <= 1e-6, (w.name, d, dj, fj, fb)
        assert sj.stats().step == 128 and sj.stats().device_error == 0


def test_joint_pass_beside_other_instances(P):
    """Two FP32 instances in the joint pass beside an FP64 instance and an FP32
    instance held to the split updates (their own branches), with electrons;
    then a tuning change that moves one instance out of the joint pass."""
    ws = W.sweep(n=4, seed=13, nsteps=192, **SMALL)
    sims = [P.Simulation(ws[0], P.PIC_FP32), P.Simulation(ws[1], P.PIC_FP32),
            P.Simulation(ws[2], P.PIC_FP64), P.Simulation(ws[3], P.PIC_FP32, flags=P.PIC_FLAG_SPLIT_FIELDS)]
    assert [s.stats().field_path for s in sims] == [1, 1, 0, 0]
    b = P.Batch(sims)
    b.step(128)
    t = sims[1].tuning
    sims[1].set_tuning(t[0], t[1], t[2], 0)  # instance 1 leaves the joint pass: one instance left there
    b.step(64)
    b.sync()
    for w, s, tol in zip(ws, sims, (2e-5, 2e-5, 1e-10, 2e-5)):
        o = O.from_workload(w)
        o.step(192)
        check(o, s, tol)
    b.close()


def test_joint_pass_instances_at_odd_and_even_steps(P):
    """A block of an instance starts where its probes were last set up: one
    instance enters the batch at step 37 (its probes set up then), the other
    at 0, so the joint pass reads state copy 1 of the first and copy 0 of the
    second in the same launch; both keep oracle parity on the fields."""
    ws = W.sweep(n=2, seed=17, nsteps=165, **SMALL)
    sims = [P.Simulation(w, P.PIC_FP32, probes=False) for w in ws]
    sims[0].step(37)
    for w, s in zip(ws, sims):
        s.probe_dft(w.probes, w.freqs, w.comp_mask)  # the block position restarts here
    b = P.Batch(sims)
    b.step(128)
    b.sync()
    assert [s.stats().step for s in sims] == [165, 128]
    for w, s, n in zip(ws, sims, (165, 128)):
        o = O.from_workload(w, with_probes=False)
        o.step(n)
        f = rel_l2(fields_of(s.field), fields_of(o.get_field))
        assert f <= 2e-5, (w.name, f)
        assert s.stats().device_error == 0
    b.close()


def test_joint_pass_mixed_slabs_and_faces(P):
    """Instances with 8-cell and 4-cell absorbing layers and one with
    conducting x faces share the joint pass (each item reads its own
    instance's layer thickness and tile kinds); each matches the oracle."""
    ws = W.sweep(n=3, seed=19, nsteps=128, **SMALL)
    ws[1].cpml_cells = 4
    ws[2].bc = (W.BC_PEC, W.BC_PEC) + tuple(ws[2].bc[2:])
    sims = [P.Simulation(w, P.PIC_FP32) for w in ws]
    assert [s.stats().field_path for s in sims] == [1, 1, 1]
    b = P.Batch(sims)
    b.step(128)
    b.sync()
    for w, s in zip(ws, sims):
        o = O.from_workload(w)
        o.step(128)
        check(o, s, 2e-5)
        assert s.stats().device_error == 0
    b.close()
