"""The 256-source, 4096-cell launch shape (the 256^3 dipping-layer workload's on-line stage):
16^3 cells with walls (uneven K_i from 45 to 90), m_i from 3 to 6, random SPD coefficients,
every precision and every available schedule, against the oracle on three sampled sources.

Sources are independent columns of the state, so the oracle stepping three of them is an exact
check of those columns of the 256-source run.  Bars: FP64 1e-10; FP32 (CUDA cores) 1e-3; FP32
from split-BF16 tensor-core products 1e-3; plain BF16 products 5e-2.
"""
import numpy as np
import pytest

import synth
from oracle import online

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

PICK = [0, 100, 255]
TAU, NST, F_PEAK = 0.05, 40, 4.0


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.fixture(scope="module")
def case(P):
    topo, co, src, rcv = synth.many_source_case()
    w = synth.ricker(np.arange(NST) * TAU, F_PEAK)
    sub = [(f, PICK.index(j), v) for (f, j, v) in src if j in PICK]
    gt = online.dense_io(topo, sub, len(PICK), "src")
    qt = online.dense_io(topo, rcv, 128, "rcv")
    ref = online.rom_leapfrog(topo, co, gt, qt, w, TAU, NST)
    R = P.Rom.import_(topo, co)
    R.set_io(256, src, 128, rcv)
    return dict(topo=topo, R=R, w=w, ref=ref)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(P, case, prec, sched=None):
    sim = P.Sim(case["R"], prec, TAU)
    if sched is not None:
        sim.set_schedule(sched)
    wd = torch.tensor(case["w"], device="cuda")
    tr = torch.zeros((NST, 128, 256), device="cuda", dtype=torch.float64 if prec == P.FP64 else torch.float32)
    sim.step(NST, wd, tr)
    torch.cuda.synchronize()
    sim.info()
    return tr.cpu().numpy().astype(np.float64)[:, :, PICK], sim


def test_shape(case):
    K = case["topo"].cell_K()
    assert case["topo"].n_cells == 4096 and K.min() == 45 and K.max() == 90
    assert set(np.unique(case["topo"].cell_m)) == {3, 4, 5, 6}
    assert np.linalg.norm(case["ref"]) > 1e-3


def test_fp64_and_fp32_schedules(P, case):
    out, _ = _run(P, case, P.FP64)
    assert _rel(out, case["ref"]) <= 1e-10
    sim = P.Sim(case["R"], P.FP32, TAU)
    _, avail = sim.schedule()
    base = None
    for k in range(P.SCHED_COUNT):
        if not avail[k]:
            continue
        out, _ = _run(P, case, P.FP32, k)
        assert _rel(out, case["ref"]) <= 1e-3, k
        if base is None:
            base = out
        assert np.array_equal(out, base), k


@pytest.mark.parametrize("prec_tol", [(2, 1e-3), (3, 5e-2)])
def test_tensor_core(P, case, prec_tol):
    prec, tol = prec_tol
    out, sim = _run(P, case, prec)
    assert sim.info()[3] == NST
    assert _rel(out, case["ref"]) <= tol
    for k in (P.SCHED_GRAPH_SPLIT, P.SCHED_PERSIST, P.SCHED_PERSIST_STREAM):
        other, _ = _run(P, case, prec, k)
        assert np.array_equal(other, out), k
