"""Receivers inside cells through the Galerkin lift (Remark MFEM), built and stepped on the GPU.

mss_partition_set_lift_nodes marks nodes strictly inside cells; the GPU off-line builder computes
their lift weights w_k = G_k^{-T} Q_k^T V^T e_n, and the on-line receiver blocks read
sum_k w_k . U^k off the face and hidden-layer state.  Checks:
* exact case (2-cell strip, S = I, m K~ = N_i): the lifted traces equal the fine leapfrog's traces at
  those nodes (the oracle's own pin, ``tests/test_oracle_lift.py``, holds the lift to 1e-10; here the
  GPU builder's CG at 1e-13 sets the bar, 1e-7);
* compressed case (3D layered medium, DCT faces): GPU traces against the oracle's lifted traces
  on the oracle's coefficients for the same bases, FP64 within 1e-7 and FP32 within 1e-3.
"""
import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _gpu_traces(P, grid, s, r, cell, io, lift, src, rcv, m, n_modes, shift, tau, w, prec):
    L = P.Operator(grid, s, r)
    LP = P.Partition(L, cell, io)
    LP.set_lift_nodes(np.asarray(lift, np.int32))
    LR = P.Rom.build(LP, m, n_modes, shift, cg_tol=1e-13)
    LR.set_io_nodes(LP, np.asarray(src, np.int32), np.asarray(rcv, np.int32))
    sim = P.Sim(LR, prec, tau)
    dt = torch.float64 if prec == P.FP64 else torch.float32
    tr = torch.zeros((len(w), len(rcv), len(src)), device="cuda", dtype=dt)
    sim.step(len(w), torch.tensor(w, device="cuda"), tr)
    torch.cuda.synchronize()
    return tr.cpu().numpy().astype(np.float64)


def test_lifted_receivers_exact_strip(P):
    c, ny = 4, 6
    g = synth.Grid(n=(ny, 2 * c), h=1.0 / (2 * c), bc=(("D", "D"), ("D", "D")))
    rng = np.random.default_rng(78)
    s, r = rng.uniform(0.5, 3.0, (ny, 2 * c)), rng.uniform(0.5, 2.5, (ny, 2 * c))
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (ny, c))
    K = len(part.faces[0].nodes)
    m = len(part.build_cell(0).nodes) // K
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    src, inner = [(2, c)], [(2, 1), (4, 3), (3, 6), (1, 5)]
    nst = 250
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    G = np.zeros((op.N, 1))
    G[op.node_unknown(src[0]), 0] = 1.0
    Q = np.zeros((len(inner), op.N))
    for j, p in enumerate(inner):
        Q[j, op.node_unknown(p)] = 1.0
    ref = fine.fine_leapfrog(op.A, op.B, G, Q, w, tau, nst)
    out = _gpu_traces(P, g, s, r, (ny, c), [], inner, src, inner, m, 10 ** 6, -0.02 * lam, tau, w, P.FP64)
    assert np.linalg.norm(out - ref) <= 1e-7 * np.linalg.norm(ref)
    for j in range(len(inner)):
        assert np.linalg.norm(out[:, j] - ref[:, j]) <= 1e-6 * np.linalg.norm(ref[:, j])


def test_lifted_receivers_match_oracle_3d(P):
    wl = synth.workload_3d_layers(32, 16, m=3, n_modes=6, n_src=2, n_steps=400, band="cell")
    inner = [(24, 8, 8), (20, 5, 20), (9, 24, 27), (28, 21, 11)]        # strictly inside cells
    io = [tuple(int(x) for x in p) for p in wl.src_nodes]
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    s = -rom.omega_max(wl.f_max) ** 2
    R = rom.build_rom(part, wl.m, wl.n_modes, s, keep=True)
    lifted = []
    for p in inner:
        u = op.node_unknown(p)
        prime = int(part.plain_prime[u])
        for cl in part.cells:
            nodes = list(part.build_cell(cl.id).nodes)
            if prime in nodes:
                assert nodes.index(prime) >= cl.K
                lifted.append((cl.id, rom.receiver_lift(R.cells[cl.id], [nodes.index(prime)])[0]))
                break
    assert len(lifted) == len(inner)
    lam = fine.lambda_max(op.A, op.B)
    tau = wl.cfl_fraction * fine.tau_critical(lam)
    w = synth.ricker(np.arange(wl.n_steps) * tau, wl.f_peak)
    gt = rom.project_io(part, R.bases, part.prime_vectors(wl.src_nodes))
    qt = [np.zeros((0, b.shape[1])) for b in R.bases]
    ref = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, wl.n_steps, lifted=lifted)
    assert np.all(np.linalg.norm(ref, axis=(0, 2)) > 0)
    for prec, tol in ((P.FP64, 1e-7), (P.FP32, 1e-3)):
        out = _gpu_traces(P, wl.grid, wl.sigma, wl.rho, wl.cell, io, inner, wl.src_nodes, inner, wl.m, wl.n_modes,
                          s, tau, w, prec)
        assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref), prec
    # a receiver inside a cell that is not a lift node is refused
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, np.asarray(io, np.int32))
    LR = P.Rom.build(LP, wl.m, wl.n_modes, s)
    with pytest.raises(P.MssError):
        LR.set_io_nodes(LP, wl.src_nodes, np.asarray(inner[:1], np.int32))
    with pytest.raises(P.MssError):
        LP.set_lift_nodes(np.asarray([[16, 8, 8]], np.int32))      # on a skeleton plane
