"""pic_save / pic_load: a run resumed from a checkpoint continues as the
uninterrupted run does (bit for bit where no atomic sums are involved, to
rounding otherwise), including buffered probe samples in the middle of a DFT
block; a checkpoint refuses a differently configured simulation."""
import os

import numpy as np
import pytest

from paper_1505_04007_gb300 import workloads as W

from _helpers import box_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


def state(s):
    return [s.field(c) for c in range(9)]


def test_resume_fields_bitwise_fp64(P, tmp_path):
    mat = np.zeros((30, 24, 40), np.uint8)
    mat[8:13] = 1
    w = box_workload(40, 24, 30, bc=(W.BC_CPML,) * 6, material=mat, table=W.drude_table())
    src = (2, (20, 21, 12, 13, 16, 17), 1e18, 30 * w.dt, 8 * w.dt, 0.0)
    a = P.Simulation(w, P.PIC_FP64, particles=False, probes=False)
    P.pic_add_source(a.h, *src)
    a.step(50)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.step(90)
    b = P.Simulation(w, P.PIC_FP64, particles=False, probes=False)
    b.load(path)
    b.step(90)
    for x, y in zip(state(a), state(b)):
        assert np.array_equal(x, y)
    assert b.stats().step == 140


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_resume_with_particles_and_probes(P, tmp_path, prec, tol):
    precision = P.PIC_FP64 if prec == "fp64" else P.PIC_FP32
    w = W.scaled(W.c1(), 64, 24, 40, 512, 0)
    a = P.Simulation(w, precision)
    a.step(37)  # mid DFT block, mid sort interval
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.step(100)
    b = P.Simulation(w, precision)  # same configuration, same particles added
    b.load(path)
    b.step(100)
    Ea, Eb = state(a)[:6], state(b)[:6]
    num = np.sqrt(sum(((x - y) ** 2).sum() for x, y in zip(Ea, Eb)))
    den = np.sqrt(sum((x ** 2).sum() for x in Ea))
    assert num <= tol * den
    Fa, Fb = a.probe_read(), b.probe_read()
    assert np.linalg.norm(Fa - Fb) <= tol * np.linalg.norm(Fa)
    xa, _, sa = a.particles()
    xb, _, sb = b.particles()
    assert np.array_equal(sa, sb)
    assert a.stats().step == b.stats().step == 137


def test_checkpoint_refuses_other_configuration(P, tmp_path):
    w = W.scaled(W.c1(), 64, 24, 40, 256, 0)
    a = P.Simulation(w, P.PIC_FP32)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    w2 = W.scaled(W.c1(), 68, 24, 40, 256, 0)
    b = P.Simulation(w2, P.PIC_FP32)
    with pytest.raises(P.PicError) as e:
        b.load(path)
    assert e.value.code == -1
    c = P.Simulation(w, P.PIC_FP64)
    with pytest.raises(P.PicError):
        c.load(path)
    with pytest.raises(P.PicError):
        a.load(os.path.join(tmp_path, "missing.bin"))
