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
from oracle import fine, freq, partition, rom


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


# --------------------------------------------------------------------------- reading R24
def test_psd_cholesky_on_known_matrices():
    """The floored factor: exact on SPD matrices, L L^T = M to rounding on a semidefinite one,
    and a clear refusal of an indefinite one."""
    rng = np.random.default_rng(24)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.geomspace(1.0, 1e-3, 12)
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    L, fl = rom.psd_cholesky(M)
    assert fl == 0 and np.allclose(L, np.linalg.cholesky(M), rtol=0, atol=1e-14)
    lam0 = lam.copy()
    lam0[-1] = 0.0                                            # exactly singular: one null vector
    M0 = (Q * lam0) @ Q.T
    M0 = 0.5 * (M0 + M0.T)
    L0, _ = rom.psd_cholesky(M0)
    assert np.allclose(L0, np.tril(L0), atol=0)
    assert np.max(np.abs(L0 @ L0.T - M0)) <= 1e-12
    lamn = lam.copy()
    lamn[-1] = -1e-4                                          # indefinite beyond rounding
    Mn = (Q * lamn) @ Q.T
    with pytest.raises(rom.RomError):
        rom.psd_cholesky(0.5 * (Mn + Mn.T))


@pytest.fixture(scope="module")
def deep_floating_cell():
    """The 24^3 one-cell-band medium at m = 7: the centre cell's last coefficient fails a plain
    Cholesky factorisation (its smallest eigenvalue is at the level of rounding)."""
    wl = synth.workload_3d_layers(24, 8, m=7, n_modes=4, n_src=2, n_steps=10, band="cell")
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    bases = [rom.face_basis(f, 4) for f in part.faces]
    s = -rom.omega_max(wl.f_max) ** 2
    cid = 13
    cell = part.build_cell(cid)
    C = rom.cell_input_matrix(part, cid, bases)
    _, Am, Sm = rom.krylov_rom(cell.A, cell.B, C, 7, s)
    al, be = rom.block_lanczos(Am, Sm, 7)
    return cell, C, Am, Sm, al, be, s


def test_semidefinite_last_coefficient_is_accepted_and_keeps_the_rom(deep_floating_cell):
    cell, C, Am, Sm, al, be, s = deep_floating_cell
    # the unmodified recursion (Eq. GammaTrans): the last coefficient has no plain Cholesky factor
    G = be[0].T.copy()
    Gp = np.zeros_like(G)
    for k in range(7):
        Gi = np.linalg.inv(G)
        Gk = -Gi.T @ al[k] @ Gi - Gp
        Gk = 0.5 * (Gk + Gk.T)
        if k < 6:
            G = np.linalg.solve(G.T @ Gk, be[k + 1].T)
        Gp = Gk
    with pytest.raises(np.linalg.LinAlgError):
        np.linalg.cholesky(Gp)
    gam, gh = rom.gamma_trans(al, be)
    last = gam[-1]
    ev = np.linalg.eigvalsh(last)
    assert ev[0] >= -1e-14 * ev[-1]                          # exactly semidefinite as L L^T
    assert np.max(np.abs(last - Gp)) <= 1e-7 * np.max(np.abs(Gp))
    for k in range(6):
        np.linalg.cholesky(gam[k])                           # the others stay SPD
    # the accepted coefficients are still this cell's ROM: the S-fraction transfer function
    # equals the projected pencil's (Eqs. GammaU1st-tfgamma) and the cell's at the shift
    for z in (s, 0.5 * s, 3.0 * s):
        ref = freq.rom_tf(Am, Sm, z)
        assert np.linalg.norm(freq.sfraction_tf(gam, gh, z) - ref) <= 1e-7 * np.linalg.norm(ref)
    exact = freq.cell_tf(cell.A, cell.B, C, s)
    assert np.linalg.norm(freq.sfraction_tf(gam, gh, s) - exact) <= 1e-7 * np.linalg.norm(exact)


def test_indefinite_last_coefficient_is_refused(deep_floating_cell):
    """A planted mistake: shifting the last Lanczos block alpha_m by a positive multiple of the
    identity makes Gamma^m indefinite, far beyond rounding."""
    _, _, _, _, al, be, _ = deep_floating_cell
    bad = [a.copy() for a in al]
    bad[-1] = bad[-1] + 0.1 * np.max(np.abs(bad[-1])) * np.eye(bad[-1].shape[0])
    with pytest.raises(rom.RomError):
        rom.gamma_trans(al[:-1] + [bad[-1]], be)
