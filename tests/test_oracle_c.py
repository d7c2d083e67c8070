"""The oracle's plain C leapfrog loops (the host-core timing path) against the NumPy oracle.

Both restate the same steps (Algorithm alg1red stage 2 for the ROM, the fine-grid leapfrog of
Section 1), so they agree to rounding: traces within 1e-12 relative L2 on ragged topologies
(uneven K_i and m_i, I/O faces) and on an assembled 2D grid.
"""
import numpy as np
import pytest

import synth
from oracle import c_leapfrog, fine, online


@pytest.mark.parametrize("shape,modes,m,n_src", [((3, 2, 2), 5, (2, 3, 4), 3), ((2, 2), 3, (1, 2, 3), 1),
                                                 ((2, 2, 2), 4, (3,), 16)])
def test_rom_leapfrog_matches_numpy(shape, modes, m, n_src):
    nc = int(np.prod(shape))
    ms = [m[i % len(m)] for i in range(nc)]
    io = [(0, 2), (nc - 1, 3)] if len(shape) == 3 else [(0, 2)]
    topo = synth.box_topology(shape, modes=modes, m=ms, io_cells=io, seed=3, ragged_modes=True)
    co = synth.random_coefficients(topo, seed=3)
    src, rcv = synth.random_io(topo, n_src, 4, seed=3)
    gt = online.dense_io(topo, src, n_src, "src")
    qt = online.dense_io(topo, rcv, 4, "rcv")
    tau, nst = 0.07, 150
    w = synth.ricker(np.arange(nst) * tau, 0.6)
    ref = online.rom_leapfrog(topo, co, gt, qt, w, tau, nst)
    out = c_leapfrog.rom_leapfrog(topo, co, gt, qt, w, tau, nst)
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)


def test_fine_leapfrog_matches_numpy():
    wl = synth.workload_2d_layers(24, 8, m=2, n_modes=3, n_steps=300)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    N = op.A.shape[0]
    g = np.zeros((N, 2))
    g[op.node_unknown((12, 12)), 0] = 1.0
    g[op.node_unknown((5, 17)), 1] = 1.0
    q = np.zeros((3, N))
    for j, p in enumerate([(23, 4), (23, 12), (10, 3)]):
        q[j, op.node_unknown(p)] = 1.0
    tau = 0.5 * fine.tau_critical(fine.lambda_max(op.A, op.B))
    w = synth.ricker(np.arange(wl.n_steps) * tau, wl.f_peak)
    ref = fine.fine_leapfrog(op.A, op.B, g, q, w, tau, wl.n_steps)
    out = c_leapfrog.fine_leapfrog(op.A, op.B, g, q, w, tau, wl.n_steps)
    assert np.linalg.norm(ref) > 0
    assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
