"""The per-cell layer-count rule of the dipping-layer workload (reading R22), in the oracle.

The rule picks the smallest m whose ROM transfer function is within a tolerance of the largest
m's at damped test frequencies.  It relies on nested Krylov spaces: the ROM of m layers is the
leading block of the ROM of more layers.  That is checked against a separate build.  The
rule's answer must then be the smallest admissible m, and must not fall as the tolerance
tightens.
"""
import numpy as np
import pytest

import synth
from oracle import fine, partition, rom


@pytest.fixture(scope="module")
def case():
    wl = synth.workload_3d_dipping(32, 16, m=4, n_modes=6, n_steps=10)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes[:2]) + list(wl.rcv_nodes[:2])]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    bases = [rom.face_basis(f, wl.n_modes) for f in part.faces]
    w = rom.omega_max(wl.f_max)
    return part, bases, -w * w, w


def test_krylov_spaces_are_nested(case):
    part, bases, s, _ = case
    cell = part.build_cell(0)
    C = rom.cell_input_matrix(part, 0, bases)
    K = C.shape[1]
    _, A5, S5 = rom.krylov_rom(cell.A, cell.B, C, 5, s)
    _, A3, S3 = rom.krylov_rom(cell.A, cell.B, C, 3, s)
    assert np.linalg.norm(A5[:3 * K, :3 * K] - A3) <= 1e-10 * np.linalg.norm(A3)
    assert np.linalg.norm(S5[:3 * K] - S3) <= 1e-12 * np.linalg.norm(S3)


def test_rule_returns_the_smallest_admissible_m(case):
    part, bases, s, w = case
    for cid in range(len(part.cells)):
        prev = 0
        for tol in (1e-2, 1e-4, 1e-7):
            m, err, errs = rom.layer_count_rule(part, cid, bases, s, w, (2, 6), tol)
            assert err <= tol and errs[m] == err
            assert all(errs[k] > tol for k in range(2, m))
            assert errs[6] == 0.0
            assert m >= prev
            prev = m
