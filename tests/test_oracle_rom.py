"""Pins of the oracle's ROM construction (Sections 4-6, Appendix C) and coupled system.

Against: the 1D closed form (Remark sfint: the S-fraction of a 1D string is the
FD scheme with primary/dual steps 1/Gamma^k, 1/Gamma-hat^k); brute force on tiny
grids (no compression, m K = N_i => the MS-ROM reproduces the fine grid exactly,
in time and in frequency); moment matching at the shift and the exact Markov
parameter (Eq. npks, Remark Sinsubspace); the S-fraction equals the ROM transfer
function (Eqs. GammaU1st-tfgamma); Stieltjes / SPD properties (Lemma lemStil,
Eq. S-fraction); uniqueness of the S-fraction (Section 5); the Galerkin CFL
inequality (Remark MFEM); Appendix D exactness at S = I.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fine, freq, online, partition, rom


def _media(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 3.0, n), rng.uniform(0.5, 2.5, n)


def test_face_basis_is_neumann_eigenbasis():
    """DCT-II columns are orthonormal eigenvectors of the reflecting 1D Laplacian tridiag(1,-2,1), ends -1."""
    for n in (1, 5, 9):
        P = rom.dct_modes(n)
        assert np.allclose(P.T @ P, np.eye(n), atol=1e-14)
        L = -2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
        L[0, 0] = L[-1, -1] = -1 if n > 1 else 0
        for a in range(n):
            lam = -4 * math.sin(math.pi * a / (2 * n)) ** 2
            assert np.allclose(L @ P[:, a], lam * P[:, a], atol=1e-13)
    order = rom.face_mode_order((3, 5))[:6]
    assert order[0] == (0, 0)
    keys = [a * a * 25 + b * b * 9 for a, b in order]
    assert keys == sorted(keys)


def test_sfraction_1d_closed_form():
    """Remark sfint / Example 1D: K~=1, m = N_i -> Gamma^k = sigma_v / h, Gamma-hat^k = 1 / b_k."""
    wl = synth.workload_1d(16, 8)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell)
    bases = [rom.face_basis(f, 1) for f in part.faces]
    h = wl.grid.h
    for cid, order in ((0, range(7, -1, -1)), (1, range(8, 16))):
        c = part.build_cell(cid)
        cr = rom.build_cell_rom(part, cid, bases, m=len(c.nodes), s=-5.0)
        # layer k of cell 0 sits at node 9-k (voxel 8-k below it), of cell 1 at node 7+k
        vox = list(order)
        for k in range(8):
            v = vox[k]
            assert abs(cr.gamma[k][0, 0] - wl.sigma[v] / h) < 1e-10 * wl.sigma[v] / h
            if k == 0:
                b = wl.rho[v] * h / 2
            else:
                vprev = vox[k - 1]
                b = (wl.rho[v] + wl.rho[vprev]) * h / 2
            assert abs(cr.gamma_hat[k][0, 0] - 1 / b) < 1e-10 / b


def _two_cell(n3d=False):
    if not n3d:
        c, ny = 4, 6
        g = synth.Grid(n=(ny, 2 * c), h=1.0 / (2 * c), bc=(("D", "D"), ("D", "D")))
        s, r = _media((ny, 2 * c), 0)
        part_cell = (ny, c)
        src, rcv = [(2, c)], [(4, c), (1, c), (3, c)]
    else:
        c = 3
        g = synth.Grid(n=(c, c, 2 * c), h=1.0 / (2 * c), bc=(("D", "D"), ("D", "D"), ("D", "D")))
        s, r = _media((c, c, 2 * c), 1)
        part_cell = (c, c, c)
        src, rcv = [(1, 1, c)], [(2, 2, c), (1, 2, c)]
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, part_cell)
    return op, part, c, src, rcv


@pytest.mark.parametrize("n3d", [False, True])
def test_two_cell_bruteforce_time_domain(n3d):
    """S = I, m K~ = N_i: the ROM leapfrog reproduces the fine leapfrog (a linear change of variables)."""
    op, part, c, src, rcv = _two_cell(n3d)
    K = len(part.faces[0].nodes)
    N0 = len(part.build_cell(0).nodes)
    assert N0 % K == 0
    m = N0 // K
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    R = rom.build_rom(part, m, n_modes=10 ** 6, s=-0.02 * lam)
    gp, qp = part.prime_vectors(src), part.prime_vectors(rcv)
    gt = rom.project_io(part, R.bases, gp)
    qt = [x.T for x in rom.project_io(part, R.bases, qp)]
    nst = 250
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    tr = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, nst)
    g = np.zeros((op.N, 1))
    g[op.node_unknown(src[0])] = 1
    q = np.zeros((len(rcv), op.N))
    for j, p in enumerate(rcv):
        q[j, op.node_unknown(p)] = 1
    ref = fine.fine_leapfrog(op.A, op.B, g, q, w, tau, nst)
    assert np.linalg.norm(tr - ref) <= 1e-10 * np.linalg.norm(ref)


def test_two_cell_bruteforce_frequency_domain():
    """Algorithm alg2red in the exact case equals the fine skeleton response at Laplace points."""
    op, part, c, src, rcv = _two_cell(False)
    K = len(part.faces[0].nodes)
    m = len(part.build_cell(0).nodes) // K
    lam = fine.lambda_max(op.A, op.B)
    R = rom.build_rom(part, m, n_modes=10 ** 6, s=-0.02 * lam)
    gp = part.prime_vectors(src)
    gt = rom.project_io(part, R.bases, gp)
    for z in (-0.1 * lam, -1.0, 0.3 * lam + 0.2j * lam):
        ut = freq.coupled_rom_solve(R.topology, R.coeffs, gt, z)
        u = spla.spsolve((op.A + z * sp.diags(op.B)).tocsc(), gp.astype(complex))
        uf = u[part.faces[0].nodes]
        assert np.linalg.norm(R.bases[0] @ ut[0][:, 0] - uf) <= 1e-10 * np.linalg.norm(uf)


def _layered_cell(n=(10, 10, 10), cell=(5, 5, 5), seed=4):
    g = synth.Grid(n=n, h=1.0 / n[-1], bc=(("D", "N"), ("D", "D"), ("D", "D")))
    s, r = _media(n, seed)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, cell, io_nodes=[(n[0], 2, 3)])
    return op, part


def test_moment_matching_and_markov_parameter():
    """The ROM matches C^T K^j (A+sB)^{-1} C, j = 0..2m-3, and the Markov parameter C^T B^{-1} C."""
    op, part = _layered_cell()
    lam = fine.lambda_max(op.A, op.B)
    s = -0.05 * lam
    bases = [rom.face_basis(f, 4) for f in part.faces]
    for cid in (0, 5):
        c = part.build_cell(cid)
        m = 3
        cr = rom.build_cell_rom(part, cid, bases, m, s, keep=True)
        A, Bd, C = c.A.tocsc(), c.B, cr.C
        lu = spla.splu((A + s * sp.diags(Bd)).tocsc())
        X = lu.solve(C)
        Am, Sm = cr.Am, cr.Sm
        Rinv = np.linalg.inv(Am + s * np.eye(Am.shape[0]))
        Y = Rinv @ Sm
        for j in range(2 * m - 2):
            mu = C.T @ X
            mur = Sm.T @ Y
            assert np.linalg.norm(mur - mu) <= 1e-9 * np.linalg.norm(mu)
            X = lu.solve(Bd[:, None] * X)
            Y = Rinv @ Y
        markov = C.T @ (C / Bd[:, None])
        assert np.linalg.norm(Sm.T @ Sm - markov) <= 1e-11 * np.linalg.norm(markov)
        assert np.linalg.norm(cr.gamma_hat[0] - markov) <= 1e-9 * np.linalg.norm(markov)
        # block-diagonal over faces (Remark Sinsubspace)
        o = 0
        for f in c.faces:
            M = bases[f].shape[1]
            off = cr.gamma_hat[0][o:o + M].copy()
            off[:, o:o + M] = 0
            assert np.max(np.abs(off)) <= 1e-10 * np.max(np.abs(cr.gamma_hat[0]))
            o += M
        # moments differ beyond the matched ones (the pin is not vacuous)
        mu = C.T @ X
        assert np.linalg.norm(Sm.T @ Y - mu) > 1e-8 * np.linalg.norm(mu)


def test_sfraction_equals_rom_and_is_stieltjes():
    op, part = _layered_cell()
    lam = fine.lambda_max(op.A, op.B)
    s = -0.05 * lam
    bases = [rom.face_basis(f, 4) for f in part.faces]
    for cid in (1, 7):
        cr = rom.build_cell_rom(part, cid, bases, 4, s, keep=True)
        ev = np.linalg.eigvalsh(cr.Am)
        assert ev[-1] < 0
        assert ev[0] >= -1.0000001 * lam * 1.0                   # Galerkin: inside the cell spectrum bound
        for G in cr.gamma + cr.gamma_hat:
            assert np.allclose(G, G.T)
            assert np.linalg.eigvalsh(G)[0] > 0
        for z in (s, 0.1 * s, 10 * s, 0.4 * lam + 0.1j * lam, -2.0 + 5.0j):
            Fr = freq.rom_tf(cr.Am, cr.Sm, z)
            Fs = freq.sfraction_tf(cr.gamma, cr.gamma_hat, z)
            assert np.linalg.norm(Fs - Fr) <= 1e-10 * np.linalg.norm(Fr)
        # Stieltjes sign structure: on the negative axis F~ is symmetric negative definite
        # (poles at z = -theta >= 0); for Im z > 0, -Im F~ is positive definite.
        F = freq.rom_tf(cr.Am, cr.Sm, -3.0)
        assert np.allclose(F, F.T) and np.linalg.eigvalsh(F)[-1] < 0
        Fc = freq.rom_tf(cr.Am, cr.Sm, 1.0 + 2.0j)
        assert np.linalg.eigvalsh(-(Fc - Fc.conj().T) / 2j)[0] > 0


def test_sfraction_is_unique_under_lanczos_rotation():
    """Section 5: the S-fraction of a given F~ is unique -- an orthogonal change of the ROM basis
    (which changes Q, alpha, beta) leaves Gamma, Gamma-hat unchanged."""
    op, part = _layered_cell()
    lam = fine.lambda_max(op.A, op.B)
    bases = [rom.face_basis(f, 3) for f in part.faces]
    cr = rom.build_cell_rom(part, 2, bases, 3, -0.05 * lam, keep=True)
    O, _ = np.linalg.qr(np.random.default_rng(3).standard_normal(cr.Am.shape))
    al, be = rom.block_lanczos(O.T @ cr.Am @ O, O.T @ cr.Sm, 3)
    g2, h2 = rom.gamma_trans(al, be)
    for a, b in zip(cr.gamma + cr.gamma_hat, g2 + h2):
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(a)


def test_rom_convergence_in_m():
    """Pade accuracy improves with m at Laplace points away from the shift (trend, Section 4.2)."""
    op, part = _layered_cell((12, 12, 12), (6, 6, 6))
    lam = fine.lambda_max(op.A, op.B)
    s = -0.02 * lam
    bases = [rom.face_basis(f, 3) for f in part.faces]
    c = part.build_cell(0)
    errs = []
    for m in (1, 2, 3, 4):
        cr = rom.build_cell_rom(part, 0, bases, m, s, keep=True)
        e = 0
        for z in (0.3 * s, 3 * s):
            Ft = freq.cell_tf(c.A, c.B, cr.C, z)
            e = max(e, np.linalg.norm(freq.rom_tf(cr.Am, cr.Sm, z) - Ft) / np.linalg.norm(Ft))
        errs.append(e)
    assert all(errs[i + 1] < 0.5 * errs[i] for i in range(3))
    assert errs[-1] < 1e-4


def test_deflation_and_size_errors():
    op, part = _layered_cell((6, 6, 6), (3, 3, 3))
    bases = [rom.face_basis(f, 100) for f in part.faces]
    with pytest.raises(rom.RomError):
        rom.build_cell_rom(part, 0, bases, 20, -10.0)


def test_rom_stable_spectrum_and_energy():
    """Proposition prop1stil: the coupled ROM pencil is non-negative (stable); the source-free
    ROM leapfrog conserves its discrete energy (Remark MFEM).  Remark Sinsubspace allows the
    mass diagonalisation to tighten the CFL limit, so only a loose bound is asserted."""
    n = (12, 12)
    g = synth.Grid(n=n, h=1.0 / 12, bc=(("D", "D"), ("D", "D")))
    s, r = _media(n, 9)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (6, 6), io_nodes=[(9, 3)])
    Ap, Bp = part.modified_operator()
    lam_f = fine.lambda_max(Ap, Bp)
    R = rom.build_rom(part, 3, 4, -0.05 * lam_f)
    Kg, Mg, _ = freq.rom_pencil(R.topology, R.coeffs)
    import scipy.linalg as sla
    lam_r = sla.eigh(Kg, Mg, eigvals_only=True)
    assert lam_r[0] > -1e-9 * lam_r[-1]
    assert lam_r[-1] <= 1.5 * lam_f
    tau = 0.9 * 2 / math.sqrt(lam_r[-1])
    st = synth.random_state(R.topology, 2, seed=1)
    zero_g = [np.zeros((int(M), 2)) for M in R.topology.face_M]
    zero_q = [np.zeros((1, int(M))) for M in R.topology.face_M]
    e0 = online.rom_energy(R.topology, R.coeffs, st[0], st[1], tau)
    _, fin = online.rom_leapfrog(R.topology, R.coeffs, zero_g, zero_q, np.zeros(400), tau, 400,
                                 state=st, return_state=True)
    e1 = online.rom_energy(R.topology, R.coeffs, fin[0], fin[1], tau)
    assert abs(e1 - e0) <= 1e-10 * abs(e0)


def test_appendix_d_correction_exact_at_fine_level():
    """With S = I the Appendix D averaging turns the corner-removed leapfrog into the original one."""
    n = (12, 12)
    g = synth.Grid(n=n, h=1.0 / 12, bc=(("D", "D"), ("D", "D")))
    s, r = _media(n, 12)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (4, 4))
    Ap, Bp = part.modified_operator()
    groups = [[(part.faces[f].nodes[rr], wt) for (f, rr, wt) in grp] for grp in part.corner_groups()]
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    nst = 300
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    src = [(4, 4), (5, 7)]
    rcv = [(8, 8), (2, 9), (4, 8)]
    gp, qp = part.prime_vectors(src), part.prime_vectors(rcv)
    G = np.zeros((op.N, 2))
    Q = np.zeros((3, op.N))
    for j, p in enumerate(src):
        G[op.node_unknown(p), j] = 1
    for j, p in enumerate(rcv):
        Q[j, op.node_unknown(p)] = 1
    ref = fine.fine_leapfrog(op.A, op.B, G, Q, w, tau, nst)
    out = fine.fine_leapfrog(Ap, Bp, gp, qp.T, w, tau, nst, groups=groups)
    assert np.linalg.norm(out - ref) <= 1e-11 * np.linalg.norm(ref)
    raw = fine.fine_leapfrog(Ap, Bp, gp, qp.T, w, tau, nst)
    assert np.linalg.norm(raw - ref) > 1e-4 * np.linalg.norm(ref)
