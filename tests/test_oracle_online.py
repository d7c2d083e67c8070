"""Pins of the oracle's on-line stepping and sensitivity of the pins to planted mistakes.

* Energy conservation of the source-free leapfrog on random SPD coefficient sets
  (any topology; Remark MFEM: the Stieltjes ROM is conservative).
* Superposition over sources and agreement with the frequency-domain system
  (the leapfrog of the coupled pencil M x_tt = -K x, step by step).
* Planted mistakes (made in a copy of the oracle's functions, on the CPU):
  each plausible error -- the GammaTrans recursion as printed, a flipped source
  sign, a dropped B in the Krylov operator, a transposed flux -- must fail a pin.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import fine, freq, online, partition, rom


def _random_rom(seed=0, ragged=True):
    topo = synth.box_topology((3, 2, 2), modes=5, m=[2, 3, 4] * 4, io_cells=[(0, 2), (7, 3)],
                              seed=seed, ragged_modes=ragged)
    co = synth.random_coefficients(topo, seed=seed)
    return topo, co


def test_energy_random_coefficients():
    topo, co = _random_rom(1)
    Kg, Mg, _ = freq.rom_pencil(topo, co)
    lam = sla.eigh(Kg, Mg, eigvals_only=True)[-1]
    tau = 0.95 * 2 / math.sqrt(lam)
    st = synth.random_state(topo, 3, seed=2)
    zg = [np.zeros((int(M), 3)) for M in topo.face_M]
    zq = [np.zeros((1, int(M))) for M in topo.face_M]
    e0 = online.rom_energy(topo, co, st[0], st[1], tau)
    _, fin = online.rom_leapfrog(topo, co, zg, zq, np.zeros(500), tau, 500, state=st, return_state=True)
    e1 = online.rom_energy(topo, co, fin[0], fin[1], tau)
    assert abs(e1 - e0) <= 1e-10 * abs(e0)


def test_leapfrog_equals_global_pencil_recursion():
    """Stepping cell by cell equals x^{n+1} = 2x^n - x^{n-1} + tau^2 M^{-1}(-K x^n - G w_n)."""
    topo, co = _random_rom(3)
    Kg, Mg, foff = freq.rom_pencil(topo, co)
    lam = sla.eigh(Kg, Mg, eigvals_only=True)[-1]
    tau = 0.5 * 2 / math.sqrt(lam)
    src, rcv = synth.random_io(topo, 2, 3, seed=4)
    gt = online.dense_io(topo, src, 2, "src")
    qt = online.dense_io(topo, rcv, 3, "rcv")
    nst = 120
    w = synth.ricker(np.arange(nst) * tau, 0.04 / tau)
    tr = online.rom_leapfrog(topo, co, gt, qt, w, tau, nst)
    n = Kg.shape[0]
    G = np.zeros((n, 2))
    Q = np.zeros((3, n))
    for f in range(topo.n_faces):
        G[foff[f]:foff[f + 1]] = gt[f]
        Q[:, foff[f]:foff[f + 1]] = qt[f]
    Mi = np.linalg.inv(Mg)
    x = np.zeros((n, 2))
    xo = np.zeros((n, 2))
    ref = np.zeros_like(tr)
    for k in range(nst):
        ref[k] = Q @ x
        x, xo = 2 * x - xo + tau * tau * Mi @ (-Kg @ x - G * w[k]), x
    assert np.linalg.norm(tr - ref) <= 1e-11 * np.linalg.norm(ref)
    # superposition: sources run one at a time add up
    tr0 = online.rom_leapfrog(topo, co, [g[:, :1] for g in gt], qt, w, tau, nst)
    tr1 = online.rom_leapfrog(topo, co, [g[:, 1:] for g in gt], qt, w, tau, nst)
    assert np.linalg.norm(np.concatenate([tr0, tr1], axis=2) - tr) <= 1e-13 * np.linalg.norm(tr)


# ---------------------------------------------------------------- planted mistakes
def _exact_case():
    c, ny = 4, 6
    g = synth.Grid(n=(ny, 2 * c), h=1.0 / (2 * c), bc=(("D", "D"), ("D", "D")))
    rng = np.random.default_rng(0)
    s, r = rng.uniform(0.5, 3.0, (ny, 2 * c)), rng.uniform(0.5, 2.5, (ny, 2 * c))
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (ny, c))
    return op, part, c


def _bruteforce_error(gamma_trans=None, krylov=None, flip_source=False):
    op, part, c = _exact_case()
    m = len(part.build_cell(0).nodes) // len(part.faces[0].nodes)
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    saved = (rom.gamma_trans, rom.krylov_rom)
    try:
        if gamma_trans:
            rom.gamma_trans = gamma_trans
        if krylov:
            rom.krylov_rom = krylov
        R = rom.build_rom(part, m, 10 ** 6, -0.02 * lam)
    except (rom.RomError, np.linalg.LinAlgError):
        return np.inf
    finally:
        rom.gamma_trans, rom.krylov_rom = saved
    src, rcv = [(2, c)], [(4, c), (1, c)]
    gp, qp = part.prime_vectors(src), part.prime_vectors(rcv)
    gt = rom.project_io(part, R.bases, gp)
    if flip_source:
        gt = [-x for x in gt]
    qt = [x.T for x in rom.project_io(part, R.bases, qp)]
    nst = 200
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    tr = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, nst)
    ref = fine.fine_leapfrog(op.A, op.B, gp, qp.T, w, tau, nst)
    err = np.linalg.norm(tr - ref) / np.linalg.norm(ref)
    return err if np.isfinite(err) else np.inf


def test_pins_catch_planted_mistakes():
    assert _bruteforce_error() < 1e-10

    def printed_gamma_trans(alphas, betas):
        # Eq. GammaTrans exactly as printed: G_1 = beta_1, Gamma^k = -G_k^T alpha_k G_k^{-1} - Gamma^{k-1},
        # G_{k+1} = (G_k^T Gamma^k)^{-1} beta_{k+1}
        G = betas[0].copy()
        Gp = np.zeros_like(G)
        gam, gh = [], []
        for k in range(len(alphas)):
            gh.append(G @ G.T)
            Gk = -G.T @ alphas[k] @ np.linalg.inv(G) - Gp
            gam.append(Gk)
            if k + 1 < len(alphas):
                G = np.linalg.solve(G.T @ Gk, betas[k + 1])
            Gp = Gk
        return gam, gh

    def krylov_without_b(A, Bd, C, m, s):
        # (A+sB)^{-1} applied without B between the powers and zero-power block C (Eq. npks literally)
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        lu = spla.splu((A + s * sp.diags(Bd)).tocsc())
        X = C.copy()
        blocks = []
        for j in range(m):
            if j > 0:
                X = lu.solve(blocks[-1])
            blocks.append(rom._b_orthonormalize(X, Bd, blocks, 1.0))
        V = np.hstack(blocks)
        return V, V.T @ (A @ V), V.T @ C

    assert _bruteforce_error(gamma_trans=printed_gamma_trans) > 1e-3
    assert _bruteforce_error(flip_source=True) > 1e-3
    # with m K = N the subspace is the whole space either way: the literal Krylov form is still
    # exact here, and its mistake (non-exact Markov parameter) shows in the moment/Markov pin instead
    op, part, c = _exact_case()
    bases = [rom.face_basis(f, 2) for f in part.faces]
    cell = part.build_cell(0)
    C = rom.cell_input_matrix(part, 0, bases)
    V, Am, Sm = krylov_without_b(cell.A, cell.B, C, 2, -5.0)
    markov = C.T @ (C / cell.B[:, None])
    assert np.linalg.norm(Sm.T @ Sm - markov) > 1e-6 * np.linalg.norm(markov)
