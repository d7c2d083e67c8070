"""Cells with no Dirichlet node: the constant mode and the near-singular last coefficient.

A cell that touches no Dirichlet wall has zero row sums in its split operator (Eq. splitN_c),
so the constant vector is a null vector of A_i.  It is also the dominant eigenvector of
K = (A_i + sB_i)^{-1}B_i, so the rational Krylov space (Eq. npks) nearly contains it.  The
projected pencil A^m then has an eigenvalue close to zero, and the S-fraction's last coefficient
Gamma^m is nearly singular.  That explains the small SPD margins and the FP32 sensitivity of
such cells.  Checked on a 3 x 3 x 3 partition: two cells float, the centre one and the one under
the Neumann top.
"""
import numpy as np
import pytest

import synth
from oracle import fine, partition, rom


@pytest.mark.parametrize("band", ["nyquist", "cell"])
def test_floating_cells_nearly_hold_the_constant_mode(band):
    wl = synth.workload_3d_layers(24, 8, m=3, n_modes=4, n_src=2, n_steps=10, band=band)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    bases = [rom.face_basis(f, 4) for f in part.faces]
    s = -rom.omega_max(wl.f_max) ** 2
    top, ratio, floating = {}, {}, []
    for cid in range(len(part.cells)):
        cell = part.build_cell(cid)
        scale = abs(cell.A).max()
        if np.abs(np.asarray(cell.A.sum(axis=1)).ravel()).max() <= 1e-12 * scale:
            floating.append(cid)
        cr = rom.build_cell_rom(part, cid, bases, 3, s, keep=True)
        ev = np.linalg.eigvalsh(cr.Am)
        assert ev[-1] < 0.0                                  # the ROM pencil stays negative definite
        top[cid] = ev[-1] / abs(ev[0])
        g = np.linalg.eigvalsh(cr.gamma[-1])
        ratio[cid] = g[0] / g[-1]
        if cid in floating:
            # Rayleigh quotient of the constant vector's B-projection onto V: the largest eigenvalue
            # of A^m lies at or above it, and it is A_i's form on the part of 1 that V misses
            V, Bd = cr.V, cell.B
            one = np.ones(V.shape[0]) / np.sqrt(Bd.sum())
            p = V @ (V.T @ (Bd * one))
            r = one - p
            rq = (p @ (cell.A @ p)) / (p @ (Bd * p))
            assert np.isclose(p @ (cell.A @ p), r @ (cell.A @ r), rtol=1e-6, atol=1e-12 * scale)
            assert ev[-1] >= rq * (1 + 1e-9)
    assert sorted(floating) == [13, 22]
    walls = [c for c in top if c not in floating]
    assert max(abs(top[c]) for c in floating) < min(abs(top[c]) for c in walls)
    assert max(ratio[c] for c in floating) < min(ratio[c] for c in walls)
