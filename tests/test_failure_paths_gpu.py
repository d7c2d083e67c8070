"""Failure detection on the GPU without faulting it: a deliberately missing neighbour at the
persistent kernel's grid barrier, and a matrix copy barrier of the split tensor-core kernels
that expects bytes which never arrive, and the same for the wide streamed cell kernel's chunk
barriers.  Each bounded wait runs out (1 s / 100 ms), the kernel
records TIMEOUT in the sim's error word and returns; the host reads MSS_ERR_TIMEOUT, clears the
word, and the same context then steps normally and bit-identically to an undisturbed run.
"""
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TIMEOUT = 7


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _sim(P, prec, n_src=16, factor_last=False):
    topo = synth.box_topology((3, 2, 2), modes=5, m=[2, 3, 4] * 4, io_cells=[(0, 2), (7, 3)], seed=2,
                              ragged_modes=True)
    co = synth.random_coefficients(topo, seed=2)
    src, rcv = synth.random_io(topo, n_src, 4, seed=2)
    R = P.Rom.import_(topo, co)
    R.set_io(n_src, src, 4, rcv)
    return P.Sim(R, prec, 0.08, factor_last=factor_last)


def _run(P, sim, nst, prec, n_src=16):
    w = torch.tensor(synth.ricker(np.arange(nst) * 0.08, 0.6), device="cuda")
    tr = torch.zeros((nst, 4, n_src), device="cuda", dtype=torch.float32)
    sim.step(nst, w, tr)
    torch.cuda.synchronize()
    return tr


@pytest.mark.parametrize("prec,sched,knob,value", [
    ("fp32", "persist", "grid", 1),
    ("fp32_tc", "split", "tc", 16),
    ("fp32_factored", "stream", "tc", 16),     # the wide TMA-streamed cell kernel's chunk barriers
    ("tf32_tc", "graph", "tc", 16),            # the wide tensor-core kernel's copy barriers
])
def test_bounded_wait_reports_timeout_and_context_recovers(P, prec, sched, knob, value):
    fac = prec == "fp32_factored"
    pr = {"fp32": P.FP32, "fp32_tc": P.FP32_TC, "fp32_factored": P.FP32, "tf32_tc": P.TF32_TC}[prec]
    sc = {"persist": P.SCHED_PERSIST, "split": P.SCHED_GRAPH_SPLIT, "stream": P.SCHED_GRAPH_STREAM,
          "graph": P.SCHED_GRAPH}[sched]
    kb = {"grid": P.DEBUG_GRID_EXTRA_ARRIVALS, "tc": P.DEBUG_TC_EXTRA_TX}[knob]
    ref_sim = _sim(P, pr, factor_last=fac)
    ref_sim.set_schedule(sc)
    ref = _run(P, ref_sim, 60, pr).cpu().numpy()
    ref_sim.info()
    sim = _sim(P, pr, factor_last=fac)
    sim.set_schedule(sc)
    sim.debug(kb, value)
    t0 = time.perf_counter()
    _run(P, sim, 4, pr)
    elapsed = time.perf_counter() - t0
    with pytest.raises(P.MssError) as e:
        sim.info()
    assert e.value.status == TIMEOUT
    assert elapsed < 30.0
    # recover: clear the error word, restore the hook, restart from a clean state
    sim.clear_error()
    sim.debug(kb, 0)
    sim.reset()
    out = _run(P, sim, 60, pr).cpu().numpy()
    sim.info()
    assert np.array_equal(out, ref)
