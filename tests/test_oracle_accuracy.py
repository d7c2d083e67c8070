"""Accuracy of the method itself: the oracle's multiscale ROM against the oracle's fine grid.

The paper prints no error values (they exist only in its missing figures), so nothing here is a
parity pin.  What Section 7 does state is the operating point -- coarse cells about one minimum
wavelength across, m = 4 layers -- and that the error falls exponentially as the number of
boundary functions per face grows (with plateaus).  This test runs the 3D layered recipe at that
operating point (32^3 voxels, eight 16^3 cells, surface sources and receivers on I/O faces,
Appendix D corner correction) and checks that the receiver error against the fine-grid leapfrog
on the original graph falls as face modes are added, reaching the 1e-3 relative-L2 level at 28
modes per face.
"""
import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom


@pytest.fixture(scope="module")
def case():
    wl = synth.workload_3d_layers(32, 16, m=4, n_modes=6, n_src=2, n_steps=1500, band="cell")
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    tau = 0.5 * fine.tau_critical(fine.lambda_max(op.A, op.B))
    w = synth.ricker(np.arange(wl.n_steps) * tau, wl.f_peak)
    N = op.A.shape[0]
    g = np.zeros((N, len(wl.src_nodes)))
    q = np.zeros((len(wl.rcv_nodes), N))
    for j, p in enumerate(wl.src_nodes):
        g[op.node_unknown(tuple(p)), j] = 1.0
    for j, p in enumerate(wl.rcv_nodes):
        q[j, op.node_unknown(tuple(p))] = 1.0
    ref = fine.fine_leapfrog(op.A.tocsr(), op.B, g, q, w, tau, wl.n_steps)
    return wl, part, tau, w, ref


def _rom_error(case, n_modes):
    wl, part, tau, w, ref = case
    s = -rom.omega_max(wl.f_max) ** 2
    R = rom.build_rom(part, wl.m, n_modes, s)
    gt = rom.project_io(part, R.bases, part.prime_vectors(wl.src_nodes))
    qt = [x.T for x in rom.project_io(part, R.bases, part.prime_vectors(wl.rcv_nodes))]
    corners = online.corner_rows(part.corner_groups(), R.bases)
    tr = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, wl.n_steps, corners=corners)
    return float(np.linalg.norm(tr - ref) / np.linalg.norm(ref))


def test_band_puts_one_minimum_wavelength_in_a_cell(case):
    wl = case[0]
    c_min = float(np.sqrt(np.min(wl.sigma / wl.rho)))
    assert abs(c_min / wl.f_max - wl.cell[0] * wl.grid.h) < 1e-9


def test_receiver_error_falls_with_face_modes(case):
    errs = [_rom_error(case, nm) for nm in (6, 15, 28)]
    # measured: 1.6e-2, 1.4e-3, 4.9e-4
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] < 5e-2
    assert errs[2] <= 1e-3
