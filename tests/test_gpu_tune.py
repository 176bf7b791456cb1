"""Launch tuning (pic_get_tuning / pic_set_tuning / pic_tune, include/pic.h):
settings that change how fast a step runs, never what it computes.

- Switching the deposit's shared-memory box, the sort interval and the
  interior field kernels' block size in the middle of a run (after a captured 64-step block, so the graph is rebuilt)
  keeps the FP64 path within 1e-10 of the FP64 oracle and the FP32 path
  within 2e-5, on a dense bunch (4096 electrons on a 64x24x40 grid), for box
  sizes that send every block to global atomics (0) or let the densest blocks
  accumulate in shared memory (16 KB), and for sort intervals from every step
  to once per block.
- pic_tune started off a block boundary steps to the boundary, times its
  twelve candidates on real steps, keeps the fastest, and the run it leaves
  behind still equals the oracle stepped the same number of steps.
- pic_batch_tune applies each candidate to every instance of a batch (one
  of them started off a block boundary), then times the lanes (instances
  chained one after another or side by side), and the runs it leaves, stepped
  further with either lane setting, equal the oracle's.
- Invalid settings are rejected and leave the current ones in place.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04007_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ETA0 = (W.MU0 / W.EPS0) ** 0.5


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_1505_04007_gb300 import pic
    pic.load()
    return pic


def dense(nsteps):
    return W.scaled(W.c1(), 64, 24, 40, 4096, nsteps)


def rel(s, o):
    num = sum(np.linalg.norm(s.field(c) * (ETA0 if c >= 3 else 1) - o.get_field(c) * (ETA0 if c >= 3 else 1)) ** 2
              for c in range(6))
    den = sum(np.linalg.norm(o.get_field(c) * (ETA0 if c >= 3 else 1)) ** 2 for c in range(6))
    return float(np.sqrt(num / den))


@pytest.fixture(scope="module")
def oracle200():
    w = dense(200)
    o = O.from_workload(w)
    o.step(200)
    return w, o


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
@pytest.mark.parametrize("dep,every,block,path", [(0, 8, 128, 0), (16384, 1, 512, 1), (2048, 32, 256, 0),
                                                  (8192, 64, 512, 1), (8192, 32, 128, 1), (8192, 64, 128, 1),
                                                  (8192, 64, 512, 0)])  # tuned bench settings among them
def test_tuning_changes_keep_parity(P, oracle200, prec, tol, dep, every, block, path):
    w, o = oracle200
    s = P.Simulation(w, P.PIC_FP64 if prec == "fp64" else P.PIC_FP32)
    fused = prec == "fp32"  # the dense slice takes the fused pass in FP32
    assert s.tuning == (4096, 16, 256, 1 if fused else 0)
    s.step(64)  # one captured block under the default settings
    s.set_tuning(dep, every, block, path)  # the field path switched in the middle of the run too
    assert s.tuning == (dep, every, block, path if fused else 0)
    assert s.stats().field_path == (path if fused else 0)
    s.step(136)
    s.sync()
    assert rel(s, o) <= tol
    Fo, Fg = o.probe_read(), s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= tol * np.linalg.norm(Fo)
    xo, _, so = o.particles()
    xg, _, sg = s.particles()
    if prec == "fp64":
        assert np.array_equal(sg, so)
        assert np.abs(xg - xo).max() <= 1e-12 * w.dx
    s.close()


def test_tune_off_a_block_boundary_keeps_parity(P):
    s = P.Simulation(dense(0), P.PIC_FP64)
    s.step(70)
    rep = s.tune(rounds=1)
    n = 70 + rep["steps"]
    assert rep["steps"] == (64 - 70 % 64) + 12 * 64
    assert s.stats().step == n
    cands = [c for c, _ in rep["candidates"]]
    assert len(cands) == 12 and rep["best"] in cands and s.tuning == rep["best"]
    assert [c[0] for c in cands[:5]] == [0, 2048, 4096, 8192, 16384]
    assert [c[1] for c in cands[5:9]] == [8, 16, 32, 64]
    assert [c[2] for c in cands[9:]] == [128, 256, 512]
    assert all(us > 0 for _, us in rep["candidates"])
    assert all(c[3] == 0 for c in cands)  # FP64: no fused pass to choose
    box_pass, sort_pass, block_pass = rep["candidates"][:5], rep["candidates"][5:9], rep["candidates"][9:]
    assert rep["best"][0] == min(box_pass, key=lambda cu: cu[1])[0][0]
    assert rep["best"][1] == min(sort_pass, key=lambda cu: cu[1])[0][1]
    assert rep["best"] == min(block_pass, key=lambda cu: cu[1])[0]
    s.step(30)
    s.sync()
    o = O.from_workload(dense(0))
    o.step(n + 30)
    assert rel(s, o) <= 1e-10
    Fo, Fg = o.probe_read(), s.probe_read()
    assert np.linalg.norm(Fg - Fo) <= 1e-10 * np.linalg.norm(Fo)
    s.close()


def test_tune_chooses_the_field_path_fp32(P):
    s = P.Simulation(dense(0), P.PIC_FP32)
    rep = s.tune(rounds=1)
    cands = [c for c, _ in rep["candidates"]]
    assert len(cands) == 14 and rep["steps"] == 14 * 64
    assert [c[3] for c in cands[12:]] == [1, 0] and cands[12][:3] == cands[13][:3]
    assert rep["best"] == min(rep["candidates"][12:], key=lambda cu: cu[1])[0]
    assert s.tuning == rep["best"] and s.stats().field_path == rep["best"][3]
    s.step(50)
    o = O.from_workload(dense(0))
    o.step(14 * 64 + 50)
    assert rel(s, o) <= 2e-5
    s.close()


def test_batch_tune_keeps_parity(P):
    ws = [dense(0), W.scaled(W.c1(), 48, 24, 40, 1024, 0)]
    sims = [P.Simulation(ws[0], P.PIC_FP64), P.Simulation(ws[1], P.PIC_FP64)]
    sims[1].step(10)  # off a block boundary
    b = P.Batch(sims)
    rep = b.tune(rounds=1)
    # twelve launch-setting candidates, then the lanes below the instance count: one chain, or all side by side
    assert rep["steps"] == 14 * 64 and len(rep["candidates"]) == 14
    assert rep["lanes"][12:] == [1, 0] and rep["best_lanes"] in (1, 0)
    assert all(x.tuning == rep["best"] for x in sims)
    b.set_lanes(1)  # the two instances one after another inside the batch graph
    b.step(64)
    b.set_lanes(0)
    b.step(64)
    b.sync()
    n = [x.stats().step for x in sims]
    assert n == [14 * 64 + 128, 64 + 14 * 64 + 128]
    for w, x, k in zip(ws, sims, n):
        o = O.from_workload(w)
        o.step(k)
        assert rel(x, o) <= 1e-10
        Fo, Fg = o.probe_read(), x.probe_read()
        assert np.linalg.norm(Fg - Fo) <= 1e-10 * np.linalg.norm(Fo)
    b.close()
    for x in sims:
        x.close()


@pytest.mark.parametrize("dep,every,block,path", [(1000, 16, 256, 1), (32768, 16, 256, 1), (-16, 16, 256, 1),
                                                  (4096, 3, 256, 1), (4096, 128, 256, 1), (4096, 0, 256, 1),
                                                  (4096, 16, 100, 1), (4096, 16, 1024, 1), (4096, 16, 256, 2),
                                                  (4096, 16, 256, -1)])
def test_invalid_tuning_rejected(P, dep, every, block, path):
    s = P.Simulation(dense(0), P.PIC_FP32)
    s.set_tuning(8192, 32, 512, 0)
    with pytest.raises(P.PicError):
        s.set_tuning(dep, every, block, path)
    assert s.tuning == (8192, 32, 512, 0)
    s.close()
