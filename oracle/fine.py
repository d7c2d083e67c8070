"""Fine-grid semi-discrete problem A u - B u_tt = g w(t)  (Section 1, Eq. wave_fll).

Conservative node-based discretisation of div(sigma grad u) - rho u_tt:
nodes sit at voxel corners; voxel v with stiffness sigma_v and density rho_v
adds, for every edge (k, l) of the voxel, the term
    -(sigma_v h^(d-2) / 2^(d-1)) (e_k - e_l)(e_k - e_l)^T       to A,
and rho_v h^d / 2^d to the mass b_k of each of its 2^d corner nodes.
A is then a symmetric non-positive graph Laplacian and B a positive diagonal
(Section 1: "A is the graph-Laplacian operator and elements of B are masses of
the grid cells").  Dirichlet walls remove their nodes; Neumann walls keep them.

Reading: the paper fixes only the type of the operator; this voxel-assembled
form is the standard conservative discretisation and reproduces, for a uniform
medium, the textbook 5/7-point stencil scaled by sigma/rho.
"""
from __future__ import annotations

import itertools
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp


def voxel_block_terms(sigma: np.ndarray, rho: np.ndarray, h: float):
    """Edge weights and node masses contributed by a block of voxels.

    Returns (edges, mass): ``edges[a]`` holds the weight of every edge along array
    axis ``a`` of the block's node grid (shape: voxel count along ``a``, node count
    along the other axes); ``mass`` has the node-grid shape.
    """
    d = sigma.ndim
    wfac = h ** (d - 2) / 2 ** (d - 1)
    mfac = h ** d / 2 ** d
    nshape = tuple(s + 1 for s in sigma.shape)
    mass = np.zeros(nshape)
    for off in itertools.product((0, 1), repeat=d):
        sl = tuple(slice(o, o + s) for o, s in zip(off, sigma.shape))
        mass[sl] += rho * mfac
    edges = []
    for a in range(d):
        shape = list(nshape)
        shape[a] = sigma.shape[a]
        e = np.zeros(shape)
        others = [b for b in range(d) if b != a]
        for off in itertools.product((0, 1), repeat=d - 1):
            sl = [slice(None)] * d
            for b, o in zip(others, off):
                sl[b] = slice(o, o + sigma.shape[b])
            e[tuple(sl)] += sigma * wfac
        edges.append(e)
    return edges, mass


def kept_mask(grid) -> np.ndarray:
    """Nodes that survive the Dirichlet walls."""
    keep = np.ones(grid.node_shape, dtype=bool)
    for a, (lo, hi) in enumerate(grid.bc):
        sl = [slice(None)] * grid.dim
        if lo == "D":
            sl[a] = 0
            keep[tuple(sl)] = False
        if hi == "D":
            sl[a] = grid.n[a]
            keep[tuple(sl)] = False
    return keep


class FineOperator:
    """A (CSR, unknowns x unknowns) and diag(B) of the fine grid.

    ``index`` maps a full-grid node (C order over the node grid, x fastest) to
    its unknown number, -1 for removed nodes; unknowns follow the node order.
    """

    def __init__(self, grid, sigma: np.ndarray, rho: np.ndarray):
        self.grid = grid
        self.keep = kept_mask(grid)
        flat = self.keep.ravel()
        self.index = np.full(flat.size, -1, dtype=np.int64)
        self.index[flat] = np.arange(int(flat.sum()))
        self.N = int(flat.sum())
        edges, mass = voxel_block_terms(sigma, rho, grid.h)
        self.B = mass.ravel()[flat].copy()
        ids = np.arange(flat.size).reshape(grid.node_shape)
        rows, cols, vals = [], [], []
        diag = np.zeros(self.N)
        for a, e in enumerate(edges):
            sl0 = [slice(None)] * grid.dim
            sl1 = [slice(None)] * grid.dim
            sl0[a] = slice(0, grid.n[a])
            sl1[a] = slice(1, grid.n[a] + 1)
            p = self.index[ids[tuple(sl0)].ravel()]
            q = self.index[ids[tuple(sl1)].ravel()]
            w = e.ravel()
            both = (p >= 0) & (q >= 0)
            rows += [p[both], q[both]]
            cols += [q[both], p[both]]
            vals += [w[both], w[both]]
            np.add.at(diag, p[p >= 0], -w[p >= 0])
            np.add.at(diag, q[q >= 0], -w[q >= 0])
        rows.append(np.arange(self.N))
        cols.append(np.arange(self.N))
        vals.append(diag)
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.N, self.N))
        self.A.sum_duplicates()

    def node_unknown(self, node) -> int:
        """Unknown number of a node given by its array-order coordinates."""
        flat = int(np.ravel_multi_index(tuple(int(c) for c in node), self.grid.node_shape))
        return int(self.index[flat])


def lambda_max(A: sp.spmatrix, B: np.ndarray) -> float:
    """Largest eigenvalue of -B^{-1} A (dense for small, ARPACK otherwise)."""
    n = A.shape[0]
    bi = 1.0 / np.sqrt(B)
    M = sp.diags(bi) @ (-A) @ sp.diags(bi)
    if n <= 2000:
        return float(np.linalg.eigvalsh(M.toarray())[-1])
    import scipy.sparse.linalg as sla
    return float(sla.eigsh(M.tocsc(), k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0])


def tau_critical(lam_max: float) -> float:
    """Leapfrog stability limit 2 / sqrt(lambda_max) of u_tt = -L u."""
    return 2.0 / np.sqrt(lam_max)


def fine_leapfrog(A: sp.spmatrix, B: np.ndarray, g: np.ndarray, q: np.ndarray, w: np.ndarray,
                  tau: float, n_steps: int, u0=None, um1=None, groups=None) -> np.ndarray:
    """Explicit leapfrog of A u - B u_tt = g w(t):
        u^{n+1} = 2 u^n - u^{n-1} + tau^2 B^{-1} (A u^n - g w(t_n)),
    u^0 = u^{-1} = 0 unless given.  g: (N, S) sources, q: (R, N) receivers.
    Returns traces r[n] = q u^n, n = 0..n_steps-1, shape (n_steps, R, S).
    ``groups`` (corner-set removed graphs only): lists of (prime node, b_l / b_k); every
    new level gets each group's hanging values replaced by their mass-weighted mean
    (Appendix D with S = I).
    """
    N, S = g.shape
    u = np.zeros((N, S)) if u0 is None else np.array(u0, dtype=np.float64)
    uo = np.zeros((N, S)) if um1 is None else np.array(um1, dtype=np.float64)
    binv = (1.0 / B)[:, None]
    out = np.zeros((n_steps, q.shape[0], S))
    for n in range(n_steps):
        out[n] = q @ u
        un = 2.0 * u - uo + tau * tau * binv * (A @ u - g * w[n])
        if groups:
            for grp in groups:
                mean = sum(wt * un[l] for l, wt in grp)
                for l, _ in grp:
                    un[l] = mean
        uo, u = u, un
    return out


def fine_energy(A, B, u_new, u_old, tau: float) -> float:
    """Conserved leapfrog energy 1/2 |(u^{n+1}-u^n)/tau|_B^2 - 1/2 (u^{n+1})^T A u^n (source-free)."""
    du = (u_new - u_old) / tau
    return float(0.5 * np.sum(B[:, None] * du * du) - 0.5 * np.sum(u_new * (A @ u_old)))
