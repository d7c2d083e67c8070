"""Step schedules on the GPU: graph-captured kernels (plain, TMA-streamed or split cell phase) and
the persistent time-block kernel, against the oracle and against each other, plus the autotuner.

Every schedule runs the same per-item arithmetic in the same order (cell rows accumulate over
the coefficient rows j = 0..K-1), so FP32 and FP64 traces are compared bit for bit across
schedules, and with the oracle at the precision's bar (1e-10 FP64, 1e-3 FP32).
"""
import numpy as np
import pytest

import synth
from oracle import online

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

FP64_TOL = 1e-10
FP32_TOL = 1e-3


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(shape=(3, 2, 2), modes=5, m=(2, 3, 4, 1), n_src=16, n_rcv=4, seed=0, io=((0, 2), (7, 3))):
    nc = int(np.prod(shape))
    ms = [m[i % len(m)] for i in range(nc)]
    topo = synth.box_topology(shape, modes=modes, m=ms, io_cells=list(io), seed=seed, ragged_modes=True)
    co = synth.random_coefficients(topo, seed=seed)
    src, rcv = synth.random_io(topo, n_src, n_rcv, seed=seed)
    return topo, co, src, rcv


def _corners(topo, seed=0, n_groups=10):
    """Corner groups shaped like the method's: member rows are distinct rows of an orthonormal
    face basis (K_f = M_f + 6 nodes per face), weights positive with unit sum."""
    rng = np.random.default_rng(seed)
    bases = [np.linalg.qr(rng.standard_normal((int(M) + 6, int(M))))[0] for M in topo.face_M]
    free = [list(rng.permutation(b.shape[0])) for b in bases]
    groups = []
    for _ in range(n_groups):
        k = int(rng.integers(2, 5))
        fs = [int(f) for f in rng.choice(topo.n_faces, size=k, replace=False) if free[f]]
        wt = rng.uniform(0.2, 1.0, len(fs))
        wt /= wt.sum()
        groups.append([(f, bases[f][free[f].pop()], float(x)) for f, x in zip(fs, wt)])
    return [g for g in groups if len(g) >= 2]


def _sim(P, topo, co, src, rcv, n_src, n_rcv, tau, prec, corners=None):
    R = P.Rom.import_(topo, co)
    R.set_io(n_src, src, n_rcv, rcv)
    if corners:
        R.set_corners(corners)
    return P.Sim(R, prec, tau, corner_correction=bool(corners))


def _run(P, sim, w, nst, n_src, n_rcv, prec, use_graph=True):
    wd = torch.tensor(np.asarray(w, np.float64), device="cuda")
    dt = torch.float64 if prec == P.FP64 else torch.float32
    tr = torch.zeros((nst, n_rcv, n_src), device="cuda", dtype=dt)
    sim.step(nst, wd, tr, use_graph=use_graph)
    torch.cuda.synchronize()
    sim.info()
    return tr.cpu().numpy().astype(np.float64)


def _oracle(topo, co, src, rcv, n_src, n_rcv, w, tau, nst, corners=None):
    gt = online.dense_io(topo, src, n_src, "src")
    qt = online.dense_io(topo, rcv, n_rcv, "rcv")
    cr = [[(f, np.asarray(row), wt) for (f, row, wt) in g] for g in corners] if corners else None
    return online.rom_leapfrog(topo, co, gt, qt, w, tau, nst, corners=cr)


@pytest.mark.parametrize("n_src", [16, 37, 5])
@pytest.mark.parametrize("corners", [False, True])
def test_schedules_match_oracle_and_each_other(P, n_src, corners):
    topo, co, src, rcv = _case(n_src=n_src, seed=3 + n_src)
    cg = _corners(topo, seed=n_src) if corners else None
    tau, nst = 0.08, 120
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, n_src, 4, w, tau, nst, cg)
    for prec, tol in ((P.FP64, FP64_TOL), (P.FP32, FP32_TOL)):
        outs = {}
        sim = _sim(P, topo, co, src, rcv, n_src, 4, tau, prec, cg)
        _, avail = sim.schedule()
        assert avail[P.SCHED_GRAPH] and avail[P.SCHED_PERSIST] and avail[P.SCHED_GRAPH_SPLIT]
        assert bool(avail[P.SCHED_GRAPH_STREAM]) == (prec == P.FP32 and n_src >= 16)
        for k in range(P.SCHED_COUNT):
            if not avail[k]:
                continue
            sim.reset()
            sim.set_schedule(k)
            outs[k] = _run(P, sim, w, nst, n_src, 4, prec)
            assert _rel(outs[k], ref) <= tol, (prec, k, _rel(outs[k], ref))
        for k, o in outs.items():
            assert np.array_equal(o, outs[P.SCHED_GRAPH]), (prec, k, _rel(o, outs[P.SCHED_GRAPH]))


def test_persistent_spans_several_time_blocks(P):
    """1100 steps = three persistent launches (512 + 512 + 76); equal to the graph schedule."""
    topo, co, src, rcv = _case(shape=(2, 2, 2), n_src=16, seed=9)
    tau, nst = 0.05, 1100
    w = synth.ricker(np.arange(nst) * tau, 0.3)
    sim = _sim(P, topo, co, src, rcv, 16, 4, tau, P.FP32)
    outs = []
    for k in (P.SCHED_GRAPH, P.SCHED_PERSIST, P.SCHED_PERSIST_STREAM):
        sim.reset()
        sim.set_schedule(k)
        outs.append(_run(P, sim, w, nst, 16, 4, P.FP32))
    assert np.abs(outs[0]).max() > 0
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_autotune_keeps_state_and_picks_fastest(P):
    topo, co, src, rcv = _case(shape=(4, 3, 2), modes=8, n_src=32, seed=12)
    tau, nst = 0.06, 200
    w = synth.ricker(np.arange(nst) * tau, 0.5)
    sim = _sim(P, topo, co, src, rcv, 32, 4, tau, P.FP32)
    full = _run(P, sim, w, nst, 32, 4, P.FP32)
    sim.reset()
    a = _run(P, sim, w[:90], 90, 32, 4, P.FP32)
    _, avail = sim.schedule()              # availability at the sim's initial tile
    chosen, ms = sim.autotune(16)
    cur, avail_after = sim.schedule()
    assert cur == chosen and avail_after[chosen]
    times = {k: ms[k] for k in range(P.SCHED_COUNT) if avail[k]}
    assert all(t > 0 for t in times.values()) and all(ms[k] == -1 for k in range(P.SCHED_COUNT) if not avail[k])
    assert chosen == min(times, key=times.get)
    assert sim.tile()[0] in (8, 16)
    assert sim.info()[3] == 90
    b = _run(P, sim, w[90:], nst - 90, 32, 4, P.FP32)
    assert np.array_equal(np.concatenate([a, b]), full)
    # the tile variants do not change any source's arithmetic
    for k in (P.SCHED_GRAPH, P.SCHED_GRAPH_SPLIT, P.SCHED_PERSIST):
        for st in (16, 8, 4):
            sim.reset()
            sim.set_schedule(k)
            sim.set_tile(source_tile=st)
            assert sim.tile()[0] == st
            assert np.array_equal(_run(P, sim, w, nst, 32, 4, P.FP32), full), (k, st)


def test_streamed_kernel_full_launch_shape(P):
    """512 cells, 15 modes per interior face, m = 4, 64 one-sided I/O faces, 16 sources: the 3D
    layered workload's launch shape on the streamed schedules; the oracle steps 2 sources."""
    io = [(c, 2) for c in range(448, 512)]
    topo = synth.box_topology((8, 8, 8), modes=15, m=4, io_cells=io, seed=21)
    co = synth.random_coefficients(topo, seed=21, spread=2.0)
    src, rcv = synth.random_io(topo, 16, 8, seed=21, density=0.02)
    tau, nst = 0.05, 40
    w = synth.ricker(np.arange(nst) * tau, 1.0)
    pick = [0, 13]
    sub = [(f, pick.index(j), v) for (f, j, v) in src if j in pick]
    ref = _oracle(topo, co, sub, rcv, 2, 8, w, tau, nst)
    sim = _sim(P, topo, co, src, rcv, 16, 8, tau, P.FP32)
    base = None
    for k in (P.SCHED_GRAPH, P.SCHED_GRAPH_STREAM, P.SCHED_PERSIST_STREAM, P.SCHED_GRAPH_SPLIT):
        sim.reset()
        sim.set_schedule(k)
        out = _run(P, sim, w, nst, 16, 8, P.FP32)
        assert _rel(out[:, :, pick], ref) <= FP32_TOL
        if base is None:
            base = out
        assert np.array_equal(out, base), k


@pytest.mark.parametrize("n_src", [16, 37, 200])
def test_tensor_core_fused_and_split_agree(P, n_src):
    """The split tensor-core kernels (one product per CTA, N up to 128 sources), their pipelined
    resident-grid form and the warp-specialised persistent kernel give the fused kernel's traces
    bit for bit, within the precision's bar of the oracle."""
    topo, co, src, rcv = _case(n_src=n_src, seed=30 + n_src)
    tau, nst = 0.08, 100
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, n_src, 4, w, tau, nst)
    for prec, tol in ((P.FP32_TC, 1e-3), (P.BF16_TC, 5e-2)):
        sim = _sim(P, topo, co, src, rcv, n_src, 4, tau, prec)
        _, avail = sim.schedule()
        assert avail[P.SCHED_GRAPH] and avail[P.SCHED_GRAPH_SPLIT] and avail[P.SCHED_PERSIST]
        assert avail[P.SCHED_PERSIST_STREAM] and not avail[P.SCHED_GRAPH_STREAM]
        outs = []
        for k in (P.SCHED_GRAPH, P.SCHED_GRAPH_SPLIT, P.SCHED_PERSIST, P.SCHED_PERSIST_STREAM):
            sim.reset()
            sim.set_schedule(k)
            outs.append(_run(P, sim, w, nst, n_src, 4, prec))
            assert _rel(outs[-1], ref) <= tol, (prec, k)
        for o in outs[1:]:
            assert np.array_equal(outs[0], o), (prec, _rel(o, outs[0]))


def test_tensor_core_tiles(P):
    """Split tensor-core products with 16..128 sources per CTA, against the oracle; every tile
    within the bar, and the autotuner's pick among them."""
    n_src = 150
    topo, co, src, rcv = _case(n_src=n_src, seed=77)
    tau, nst = 0.08, 80
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, n_src, 4, w, tau, nst)
    sim = _sim(P, topo, co, src, rcv, n_src, 4, tau, P.FP32_TC)
    outs = {}
    for nt in (16, 32, 64, 128):
        sim.reset()
        sim.set_schedule(P.SCHED_GRAPH_SPLIT)
        sim.set_tile(tc_sources=nt)
        assert sim.tile()[1] == nt
        outs[nt] = _run(P, sim, w, nst, n_src, 4, P.FP32_TC)
        assert _rel(outs[nt], ref) <= 1e-3, nt
    for nt in (32, 64, 128):
        assert _rel(outs[nt], outs[16]) <= 1e-6, nt
    chosen, ms = sim.autotune(8)
    assert sim.tile()[1] in (16, 32, 64, 128) and ms[chosen] > 0
