"""On-line stepping on the GPU (through the C ABI) against the oracle's ROM leapfrog.

Bars: FP64 traces within 1e-10 relative L2 of the oracle; FP32 within 1e-3, the stated bound
for the reduced-precision path.  (FP32 rounding, 6e-8, is amplified by the cancellation in
U^{k+1} - U^k between neighbouring hidden layers of real ROMs -- |U| / |U^{k+1} - U^k| of order
10..100 -- and accumulates over the steps; measured 2e-5 on random coefficient sets and
~5e-4 on ROMs of the 2D layered workload over 300 steps.)
Cases cover ragged cells (uneven K and m), one-sided faces, several source tiles with a
ragged tail, corner correction, graph vs eager launch, resume, the host-buffer entry point,
oracle-built ROMs, and the 512-cell / 16-source launch configuration on sampled sources.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom

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


def _lib_run(P, topo, co, src, rcv, n_src, n_rcv, w, tau, nst, prec, corners=None, use_graph=True):
    R = P.Rom.import_(topo, co)
    R.set_io(n_src, src, n_rcv, rcv)
    if corners:
        R.set_corners(corners)
    sim = P.Sim(R, prec, tau, corner_correction=bool(corners))
    wd = torch.tensor(np.asarray(w, np.float64), device="cuda")
    dt = torch.float64 if prec == P.FP64 else torch.float32
    tr = torch.zeros((nst, n_rcv, n_src), device="cuda", dtype=dt)
    sim.step(nst, wd, tr, use_graph=use_graph)
    torch.cuda.synchronize()
    sim.info()                    # raises if a bounded device wait gave up
    return tr.cpu().numpy().astype(np.float64), sim


def _random_case(shape=(3, 2, 2), modes=5, m=(2, 3, 4), n_src=3, n_rcv=4, seed=0, io=((0, 2), (7, 3))):
    nc = int(np.prod(shape))
    ms = [m[i % len(m)] for i in range(nc)]
    topo = synth.box_topology(shape, modes=modes, m=ms, io_cells=list(io), seed=seed, ragged_modes=True)
    co = synth.random_coefficients(topo, seed=seed)
    src, rcv = synth.random_io(topo, n_src, n_rcv, seed=seed)
    return topo, co, src, rcv


def _oracle(topo, co, src, rcv, n_src, n_rcv, w, tau, nst, corners=None):
    gt = online.dense_io(topo, src, n_src, "src")
    qt = online.dense_io(topo, rcv, n_rcv, "rcv")
    cr = None
    if corners:
        cr = [[(f, np.asarray(row), wt) for (f, row, wt) in g] for g in corners]
    return online.rom_leapfrog(topo, co, gt, qt, w, tau, nst, corners=cr)


@pytest.mark.parametrize("n_src", [1, 3, 16, 37])
def test_fp64_parity_ragged(P, n_src):
    topo, co, src, rcv = _random_case(n_src=n_src, seed=n_src)
    tau, nst = 0.08, 150
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, n_src, 4, w, tau, nst)
    assert np.max(np.abs(ref)) < 1e6                      # stable step
    out, _ = _lib_run(P, topo, co, src, rcv, n_src, 4, w, tau, nst, P.FP64)
    assert _rel(out, ref) <= FP64_TOL
    out32, _ = _lib_run(P, topo, co, src, rcv, n_src, 4, w, tau, nst, P.FP32)
    assert _rel(out32, ref) <= FP32_TOL


def _random_corners(topo, seed=0, n_groups=10):
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


def test_corner_correction_parity(P):
    topo, co, src, rcv = _random_case(n_src=5, seed=3)
    corners = _random_corners(topo, seed=3)
    tau, nst = 0.08, 120
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, 5, 4, w, tau, nst, corners=corners)
    out, sim = _lib_run(P, topo, co, src, rcv, 5, 4, w, tau, nst, P.FP64, corners=corners)
    assert sim.info()[6] == 3
    assert _rel(out, ref) <= FP64_TOL
    plain = _oracle(topo, co, src, rcv, 5, 4, w, tau, nst)
    assert _rel(plain, ref) > 1e-6                      # the correction does change the result


def test_graph_eager_and_resume_bitwise(P):
    topo, co, src, rcv = _random_case(n_src=16, seed=5)
    tau, nst = 0.08, 80
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    for prec in (P.FP64, P.FP32):
        a, _ = _lib_run(P, topo, co, src, rcv, 16, 4, w, tau, nst, prec, use_graph=True)
        b, _ = _lib_run(P, topo, co, src, rcv, 16, 4, w, tau, nst, prec, use_graph=False)
        assert np.array_equal(a, b)
        # resume: first half, save, new sim, load, second half
        R = P.Rom.import_(topo, co)
        R.set_io(16, src, 4, rcv)
        s1 = P.Sim(R, prec, tau)
        dt = torch.float64 if prec == P.FP64 else torch.float32
        wd = torch.tensor(w, device="cuda")
        t1 = torch.zeros((nst // 2, 4, 16), device="cuda", dtype=dt)
        s1.step(nst // 2, wd, t1)
        now, old, k = s1.save_state()
        assert k == nst // 2
        s2 = P.Sim(R, prec, tau)
        s2.load_state(now, old, k)
        t2 = torch.zeros((nst - nst // 2, 4, 16), device="cuda", dtype=dt)
        s2.step(nst - nst // 2, wd[nst // 2:], t2)
        torch.cuda.synchronize()
        c = np.concatenate([t1.cpu().numpy(), t2.cpu().numpy()]).astype(np.float64)
        assert np.array_equal(a, c)


def test_run_host_matches_device_path(P):
    topo, co, src, rcv = _random_case(n_src=7, seed=9)
    tau, nst = 0.08, 60
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    a, sim = _lib_run(P, topo, co, src, rcv, 7, 4, w, tau, nst, P.FP64)
    b = sim.run_host(w)
    assert np.array_equal(a, b)


def _oracle_rom_case(n=32, cell=8, M=4, m=3):
    wl = synth.workload_2d_layers(n, cell, m=m, n_modes=M, n_steps=300)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = list(map(tuple, wl.src_nodes)) + list(map(tuple, wl.rcv_nodes))
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    lam = fine.lambda_max(op.A, op.B)
    tau = wl.cfl_fraction * fine.tau_critical(lam)
    R = rom.build_rom(part, m, M, -rom.omega_max(wl.f_max) ** 2)
    gp, qp = part.prime_vectors(wl.src_nodes), part.prime_vectors(wl.rcv_nodes)
    gt = rom.project_io(part, R.bases, gp)
    qt = rom.project_io(part, R.bases, qp)
    src = [(f, j, gt[f][:, j]) for f in range(len(gt)) for j in range(gt[f].shape[1]) if np.any(gt[f][:, j])]
    rcv = [(f, j, qt[f][:, j]) for f in range(len(qt)) for j in range(qt[f].shape[1]) if np.any(qt[f][:, j])]
    w = synth.ricker(np.arange(wl.n_steps) * tau, wl.f_peak)
    corners = online.corner_rows(part.corner_groups(), R.bases)
    return wl, R, src, rcv, w, tau, corners


def test_oracle_built_rom_parity(P):
    wl, R, src, rcv, w, tau, corners = _oracle_rom_case()
    ns, nr, nst = len(wl.src_nodes), len(wl.rcv_nodes), wl.n_steps
    for cor in (None, corners):
        ref = _oracle(R.topology, R.coeffs, src, rcv, ns, nr, w, tau, nst,
                      corners=None if cor is None else [[(f, row, wt) for (f, row, wt) in g] for g in cor])
        out, _ = _lib_run(P, R.topology, R.coeffs, src, rcv, ns, nr, w, tau, nst, P.FP64,
                          corners=None if cor is None else [[(f, row, wt) for (f, row, wt) in g] for g in cor])
        assert _rel(out, ref) <= FP64_TOL
        out32, _ = _lib_run(P, R.topology, R.coeffs, src, rcv, ns, nr, w, tau, nst, P.FP32,
                            corners=None if cor is None else [[(f, row, wt) for (f, row, wt) in g] for g in cor])
        assert _rel(out32, ref) <= FP32_TOL


def test_full_size_launch_sampled_sources(P):
    """512 cells (8^3 box), 15 modes per interior face, m = 4, 64 one-sided I/O faces,
    16 sources -- the 3D layered workload's launch shape; the oracle steps 2 of the sources."""
    io = [(c, 2) for c in range(448, 512)]
    topo = synth.box_topology((8, 8, 8), modes=15, m=4, io_cells=io, seed=21)
    co = synth.random_coefficients(topo, seed=21, spread=2.0)
    src, rcv = synth.random_io(topo, 16, 8, seed=21, density=0.02)
    tau, nst = 0.05, 40
    w = synth.ricker(np.arange(nst) * tau, 1.0)
    out64, _ = _lib_run(P, topo, co, src, rcv, 16, 8, w, tau, nst, P.FP64)
    out32, _ = _lib_run(P, topo, co, src, rcv, 16, 8, w, tau, nst, P.FP32)
    pick = [0, 13]
    sub = [(f, pick.index(j), v) for (f, j, v) in src if j in pick]
    ref = _oracle(topo, co, sub, rcv, 2, 8, w, tau, nst)
    assert _rel(out64[:, :, pick], ref) <= FP64_TOL
    assert _rel(out32[:, :, pick], ref) <= FP32_TOL


@pytest.mark.parametrize("prec_tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("n_src", [3, 4, 8])
def test_fine_grid_gpu_parity(P, prec_tol, n_src):
    """Scalar kernel (3 sources) and the vector kernel over sources (4 and 8: multiples of the
    16-byte vector width in both precisions)."""
    prec, tol = prec_tol
    n = (10, 12, 14)
    g = synth.Grid(n=n, h=1.0 / 14, bc=(("D", "N"), ("D", "D"), ("N", "D")))
    rng = np.random.default_rng(4)
    s, r = rng.uniform(0.5, 3, n), rng.uniform(0.5, 2.5, n)
    op = fine.FineOperator(g, s, r)
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    srcn = [(10, 3, 4), (5, 6, 7), (2, 2, 9), (7, 10, 2), (3, 9, 12), (9, 1, 1), (6, 6, 6), (1, 11, 5)][:n_src]
    rcvn = [(10, 8, 8), (4, 4, 4), (7, 1, 13), (10, 3, 4)]
    nst = 200
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    G = np.zeros((op.N, n_src))
    Q = np.zeros((4, op.N))
    for j, p in enumerate(srcn):
        G[op.node_unknown(p), j] = 1
    for j, p in enumerate(rcvn):
        Q[j, op.node_unknown(p)] = 1
    ref = fine.fine_leapfrog(op.A, op.B, G, Q, w, tau, nst)
    L = P.Operator(g, s, r)
    fs = P.FineSim(L, prec, tau, srcn, rcvn)
    wd = torch.tensor(w, device="cuda")
    tr = torch.zeros((nst, 4, n_src), device="cuda", dtype=torch.float64 if prec == 0 else torch.float32)
    fs.step(nst, wd, tr)
    torch.cuda.synchronize()
    assert _rel(tr.cpu().numpy().astype(np.float64), ref) <= tol


# ---------------------------------------------------------------- tensor-core cell products
TC_TOL = {2: 1e-3, 3: 5e-2}   # FP32_TC (split BF16, three products) / BF16_TC (one product)


@pytest.mark.parametrize("n_src", [1, 16, 37, 64])
def test_tensor_core_parity_ragged(P, n_src):
    topo, co, src, rcv = _random_case(n_src=n_src, seed=40 + n_src)
    tau, nst = 0.08, 150
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, n_src, 4, w, tau, nst)
    errs = {}
    for prec in (P.FP32_TC, P.BF16_TC):
        out, _ = _lib_run(P, topo, co, src, rcv, n_src, 4, w, tau, nst, prec)
        errs[prec] = _rel(out, ref)
        assert errs[prec] <= TC_TOL[prec], (prec, errs[prec])
    assert errs[P.FP32_TC] < errs[P.BF16_TC]


TF32_TOL = 1e-3   # TF32_TC: split TF32 (three products), FP32-class


def _worst_receiver(a, b):
    return max(float(np.linalg.norm(a[:, r] - b[:, r]) / np.linalg.norm(b[:, r]))
               for r in range(b.shape[1]) if np.linalg.norm(b[:, r]) > 1e-12 * np.linalg.norm(b))


@pytest.mark.parametrize("n_src", [1, 16, 37])
def test_tf32_tensor_core_parity_ragged(P, n_src):
    """The wide tensor-core kernel (MSS_TF32_TC) on small ragged cells (m = 2..4, uneven K, one
    M tile): 1 and 37 sources exercise a partial 16-source tile, 37 three tiles per cell."""
    topo, co, src, rcv = _random_case(n_src=n_src, seed=60 + n_src)
    tau, nst = 0.08, 150
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = _oracle(topo, co, src, rcv, n_src, 4, w, tau, nst)
    out, sim = _lib_run(P, topo, co, src, rcv, n_src, 4, w, tau, nst, P.TF32_TC)
    assert sim.schedule()[1].tolist() == [1, 0, 0, 0, 0]
    assert _rel(out, ref) <= TF32_TOL
    assert _worst_receiver(out, ref) <= TF32_TOL


@pytest.mark.parametrize("modes,ms", [(24, (2, 5)), (45, (3, 4, 5)), (64, (2, 3, 4, 5))])
def test_tf32_tensor_core_multi_tile(P, modes, ms):
    """K_i up to 144, 270 and 384 (two and three M tiles of 128 rows, the last one short; the
    triangular factor's blocks skipped off its triangle) on a 3 x 3 x 3 box, random coefficients,
    16 sources, against the FP64 oracle."""
    topo = synth.box_topology((3, 3, 3), modes=modes, m=[ms[i % len(ms)] for i in range(27)],
                              io_cells=[(0, 2), (26, 3)], seed=modes, ragged_modes=False)
    assert max(topo.cell_K()) == 6 * modes
    co = synth.random_coefficients(topo, seed=modes)
    src, rcv = synth.random_io(topo, 16, 6, seed=modes)
    tau, nst = 0.05, 120
    w = synth.ricker(np.arange(nst) * tau, 0.8)
    ref = _oracle(topo, co, src, rcv, 16, 6, w, tau, nst)
    assert np.linalg.norm(ref) > 0
    out, _ = _lib_run(P, topo, co, src, rcv, 16, 6, w, tau, nst, P.TF32_TC)
    assert _rel(out, ref) <= TF32_TOL
    assert _worst_receiver(out, ref) <= TF32_TOL


def test_tensor_core_uneven_cells_256_sources(P):
    """512 cells with 3..6 S-fraction layers and 8..16 modes per face, 256 sources (the
    many-source launch shape); the oracle steps sources 0, 77 and 255."""
    rng = np.random.default_rng(5)
    ms = rng.integers(3, 7, 512)
    io = [(c, 2) for c in range(448, 512)]
    topo = synth.box_topology((8, 8, 8), modes=16, m=ms, io_cells=io, seed=23, ragged_modes=True)
    co = synth.random_coefficients(topo, seed=23, spread=2.0)
    src, rcv = synth.random_io(topo, 256, 6, seed=23, density=0.01)
    tau, nst = 0.05, 30
    w = synth.ricker(np.arange(nst) * tau, 1.0)
    pick = [0, 77, 255]
    sub = [(f, pick.index(j), v) for (f, j, v) in src if j in pick]
    ref = _oracle(topo, co, sub, rcv, 3, 6, w, tau, nst)
    out, sim = _lib_run(P, topo, co, src, rcv, 256, 6, w, tau, nst, P.FP32_TC)
    assert sim.info()[3] == nst
    assert _rel(out[:, :, pick], ref) <= TC_TOL[2]
    out32, _ = _lib_run(P, topo, co, src, rcv, 256, 6, w, tau, nst, P.FP32)
    assert _rel(out32[:, :, pick], ref) <= FP32_TOL
