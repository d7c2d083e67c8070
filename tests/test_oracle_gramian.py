"""The paper's own boundary basis in the oracle: the frequency-limited Gramian of Eq. trgr.

Pinned by a closed form.  In a uniform 2D box with Dirichlet walls, the 5-point graph Laplacian
has the textbook sine eigenvectors and eigenvalues.  The Gramian of every interior face is then
a finite sum of outer products of sampled sines, written here without any eigensolver.  The
oracle's route (eigensolver, normalisation in the B inner product, selection of the modes
below the band limit, restriction to the face nodes) has to reproduce it.  The top
eigenvectors form the basis.  A dense and a shift-invert eigensolver give the same propagative
subspace.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fine, partition, rom


def _uniform_box(n, cell, rho=1.0, sigma=1.0):
    grid = synth.Grid(n=(n, n), h=1.0 / n, bc=(("D", "D"), ("D", "D")))
    s = np.full((n, n), sigma)
    r = np.full((n, n), rho)
    op = fine.FineOperator(grid, s, r)
    return grid, op, partition.Partition(op, s, r, (cell, cell))


def _closed_form(grid, op, sigma, rho, lam_max):
    """Sine eigenpairs of -B^{-1}A = (sigma/rho) L5 / h^2, B-normalised (z^T B z = 1)."""
    n = grid.n[0]
    h = grid.h
    flat = np.nonzero(op.index >= 0)[0]              # unknowns follow the node order
    y, x = np.unravel_index(flat, grid.node_shape)
    cols = []
    for a in range(1, n):
        for b in range(1, n):
            lam = (sigma / rho) * (4 * math.sin(a * math.pi / (2 * n)) ** 2
                                   + 4 * math.sin(b * math.pi / (2 * n)) ** 2) / h ** 2
            if lam <= lam_max:
                # sum_i sin^2(a pi i / n) = n / 2 per axis, mass rho h^2 per node: c = 2 / sqrt(rho)
                cols.append(2.0 / math.sqrt(rho) * np.sin(a * math.pi * x / n) * np.sin(b * math.pi * y / n))
    return np.stack(cols, axis=1)


def _band_between_levels(n, h, ratio, level):
    lv = sorted({round(ratio * (4 * math.sin(a * math.pi / (2 * n)) ** 2 + 4 * math.sin(b * math.pi / (2 * n)) ** 2)
                       / h ** 2, 9) for a in range(1, n) for b in range(1, n)})
    return 0.5 * (lv[level] + lv[level + 1])


@pytest.mark.parametrize("rho,sigma", [(1.0, 1.0), (2.0, 3.0)])
def test_gramian_of_uniform_box_is_the_sine_mode_sum(rho, sigma):
    n, cell = 12, 4
    grid, op, part = _uniform_box(n, cell, rho, sigma)
    lam_max = _band_between_levels(n, grid.h, sigma / rho, 9)
    Zc = _closed_form(grid, op, sigma, rho, lam_max)
    modes = rom.propagative_modes(op.A, op.B, lam_max)
    assert modes[1].shape[1] == Zc.shape[1]
    G = rom.face_gramians(part, modes)
    S = rom.gramian_bases(part, lam_max, 3, modes=modes)
    assert len(part.faces) == 12
    for f, Gf, Sf in zip(part.faces, G, S):
        idx = np.asarray(f.parents)
        Gc = Zc[idx] @ Zc[idx].T
        assert np.allclose(Gf, Gc, rtol=0, atol=1e-12 * np.abs(Gc).max())
        # the basis spans the top of the spectrum: its Rayleigh quotients are the 3 largest eigenvalues
        ev = np.sort(np.linalg.eigvalsh(Gc))[::-1][:3]
        assert np.allclose(np.sort(np.linalg.eigvalsh(Sf.T @ Gc @ Sf))[::-1], ev, rtol=1e-10, atol=1e-12 * ev[0])
        assert np.allclose(Sf.T @ Sf, np.eye(3), atol=1e-12)


def test_dense_and_shift_invert_eigensolvers_agree():
    wl = synth.workload_2d_layers(24, 8, m=2, n_modes=3, n_steps=10)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    lam_max = (2 * math.pi * wl.f_max) ** 2
    ld, Zd = rom.propagative_modes(op.A, op.B, lam_max)
    ls, Zs = rom.propagative_modes(op.A, op.B, lam_max, dense_limit=10)
    assert ld.size == ls.size and ld.size > 4
    assert np.allclose(ld, ls, rtol=1e-10)
    # same B-orthogonal projector onto the propagative subspace (eigenvector signs are free)
    assert np.allclose(Zd @ Zd.T, Zs @ Zs.T, atol=1e-9 * np.abs(Zd @ Zd.T).max())
    assert np.allclose(Zd.T @ (op.B[:, None] * Zd), np.eye(ld.size), atol=1e-10)


def _gramian_pin_error(modes_fn=None):
    """Largest relative deviation of the oracle's face Gramians from the closed form (rho = 2)."""
    n, cell, rho, sigma = 12, 4, 2.0, 3.0
    grid, op, part = _uniform_box(n, cell, rho, sigma)
    lam_max = _band_between_levels(n, grid.h, sigma / rho, 9)
    Zc = _closed_form(grid, op, sigma, rho, lam_max)
    modes = (modes_fn or rom.propagative_modes)(op.A, op.B, lam_max)
    G = rom.face_gramians(part, modes)
    err = 0.0
    for f, Gf in zip(part.faces, G):
        idx = np.asarray(f.parents)
        Gc = Zc[idx] @ Zc[idx].T
        err = max(err, np.abs(Gf - Gc).max() / np.abs(Gc).max())
    return err


def test_gramian_pin_catches_planted_mistakes():
    assert _gramian_pin_error() < 1e-12

    def euclidean_modes(A, Bd, lam_max):
        # eigenvectors normalised in the Euclidean instead of the B inner product
        lam, Z = rom.propagative_modes(A, Bd, lam_max)
        return lam, Z / np.linalg.norm(Z, axis=0)

    def generalised_sign(A, Bd, lam_max):
        # eigenvalues of B^{-1}A instead of -B^{-1}A (reading R16 ignored): every mode passes
        import scipy.linalg as sla
        lam, Z = sla.eigh(A.toarray(), np.diag(Bd))
        keep = lam <= lam_max
        return lam[keep], Z[:, keep]

    def one_mode_short(A, Bd, lam_max):
        lam, Z = rom.propagative_modes(A, Bd, lam_max)
        return lam[:-1], Z[:, :-1]

    assert _gramian_pin_error(euclidean_modes) > 1e-3
    assert _gramian_pin_error(one_mode_short) > 1e-3
    assert _gramian_pin_error(generalised_sign) > 1e-3
