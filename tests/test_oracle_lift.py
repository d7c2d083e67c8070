"""Pin of the oracle's interior receivers (``rom.receiver_lift`` with ``online.rom_leapfrog(lifted=...)``).

The ROM is a Galerkin method (Remark MFEM): a cell's fine-grid state is approximated by V x, x the
projected state.  The lift reads a fine node inside a cell off the S-fraction state as
sum_k w_k^T U^k, w_k = G_k^{-T} Q_k^T V^T e_n (Lanczos blocks Q_k of Eq. NtDtri, G_k of Eq.
GammaTrans).  Brute force fixes it: without compression (S = I) and with m K~ = N_i the basis V spans
the whole cell, so the lifted trace must equal the fine leapfrog's trace at that node to rounding
(2-cell strips in 2D and 3D, nodes strictly inside either cell).  Planted mistakes (on the CPU) fail
it: G_k G_k^T in place of the identity, the S-fraction variables read as Lanczos coordinates, and
weights shifted by one layer.
"""
import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom


def _strip(n3d: bool):
    if n3d:
        c = 3
        g = synth.Grid(n=(c, c, 2 * c), h=1.0 / (2 * c), bc=(("D", "D"), ("D", "D"), ("D", "D")))
        shape, cell = (c, c, 2 * c), (c, c, c)
        src = [(1, 1, c)]
        inner = [(1, 1, 1), (2, 1, 2), (1, 2, 4)]     # two in cell 0, one in cell 1
    else:
        c, ny = 4, 6
        g = synth.Grid(n=(ny, 2 * c), h=1.0 / (2 * c), bc=(("D", "D"), ("D", "D")))
        shape, cell = (ny, 2 * c), (ny, c)
        src = [(2, c)]
        inner = [(2, 1), (4, 3), (3, 6)]
    rng = np.random.default_rng(77 + int(n3d))
    s, r = rng.uniform(0.5, 3.0, shape), rng.uniform(0.5, 2.5, shape)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, cell)
    return op, part, src, inner


def _lifted(part, R, inner):
    out = []
    for p in inner:
        u = part.op.node_unknown(p)
        prime = int(part.plain_prime[u])
        for c in part.cells:
            nodes = list(part.build_cell(c.id).nodes)
            if prime in nodes and c.id in R.cells:
                w = rom.receiver_lift(R.cells[c.id], [nodes.index(prime)])[0]
                out.append((c.id, w))
                break
        else:
            raise AssertionError("node %s not inside a cell" % (p,))
    return out


def _run(n3d, tamper=None):
    op, part, src, inner = _strip(n3d)
    K = len(part.faces[0].nodes)
    N0 = len(part.build_cell(0).nodes)
    assert N0 % K == 0
    m = N0 // K
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    R = rom.build_rom(part, m, n_modes=10 ** 6, s=-0.02 * lam, keep=True)
    for cr in R.cells.values():
        assert np.linalg.matrix_rank(cr.V) == cr.V.shape[0] == cr.V.shape[1]
    lifted = _lifted(part, R, inner)
    if tamper is not None:
        lifted = tamper(R, lifted)
    gp = part.prime_vectors(src)
    gt = rom.project_io(part, R.bases, gp)
    qt = [np.zeros((0, b.shape[1])) for b in R.bases]
    nst = 250
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    tr = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, nst, lifted=lifted)
    G = np.zeros((op.N, 1))
    G[op.node_unknown(src[0]), 0] = 1.0
    Q = np.zeros((len(inner), op.N))
    for j, p in enumerate(inner):
        Q[j, op.node_unknown(p)] = 1.0
    ref = fine.fine_leapfrog(op.A, op.B, G, Q, w, tau, nst)
    assert np.all(np.linalg.norm(ref, axis=(0, 2)) > 0)
    return float(np.linalg.norm(tr - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("n3d", [False, True])
def test_lifted_interior_receivers_reproduce_fine_grid(n3d):
    assert _run(n3d) <= 1e-10


def _gk_factors(R, cid):
    cr = R.cells[cid]
    al, be = rom.block_lanczos(cr.Am, cr.Sm, len(cr.gamma))
    return rom.gamma_trans(al, be, return_g=True)[2]


def _transposed_g(R, lifted):
    """Planted: the Lanczos coordinates taken as z_k = G_k^T U^k instead of G_k^{-1} U^k."""
    out = []
    for cid, w in lifted:
        Gs = _gk_factors(R, cid)
        out.append((cid, np.array([Gs[k] @ (Gs[k].T @ w[k]) for k in range(len(w))])))
    return out


def _unscaled(R, lifted):
    """Planted: the S-fraction variables read as Lanczos coordinates (no G_k)."""
    out = []
    for cid, w in lifted:
        Gs = _gk_factors(R, cid)
        out.append((cid, np.array([Gs[k].T @ w[k] for k in range(len(w))])))
    return out


def _layer_shift(R, lifted):
    """Planted: every layer's weights applied one layer deeper."""
    out = []
    for cid, w in lifted:
        w2 = np.zeros_like(w)
        w2[1:] = w[:-1]
        out.append((cid, w2))
    return out


@pytest.mark.parametrize("plant", [_transposed_g, _unscaled, _layer_shift])
def test_planted_lift_mistakes_fail(plant):
    assert _run(False, tamper=plant) > 1e-4
