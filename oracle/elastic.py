"""Anisotropic (VTI) elastic fine-grid operator, the first step of the elastic workload.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

The paper's elastic experiment (Section 7) solves u_i,tt = sigma_ij,j with sigma_ij =
C_ijkl (u_k,l + u_l,k) / 2 and a second-order discretisation, and states that the method
applies to any symmetric non-positive pencil (A, B) of the form A u - B u_tt = g w(t)
(Section 1).  Here the pencil is assembled as follows:

* A = -K, with K the stiffness of trilinear (Q1) finite elements on the voxel grid.  It is
  integrated exactly for constant C per voxel by 2 x 2 x 2 Gauss points.
* B is the lumped (row-sum) mass: rho h^3 / 8 per voxel corner and displacement component.
* The unknowns are 3 per kept node, numbered node-major (node, then component x, y, z in
  array-axis order).  Dirichlet walls remove their nodes, as in the scalar operator.

The medium is vertically transversely isotropic (VTI), with the symmetry axis along array axis
0 (z).  Its 6 x 6 Voigt stiffness comes from Thomsen's parameters (Thomsen 1986):
    C33 = rho Vp^2,  C44 = rho Vs^2,  C11 = C33 (1 + 2 eps),  C66 = C44 (1 + 2 gamma),
    (C13 + C44)^2 = (C33 - C44) (C33 (1 + 2 delta) - C44),  C12 = C11 - 2 C66.
Voigt order (xx, yy, zz, yz, xz, xy) in physical axes x, y, z.  Array axes map to them as
[z][y][x]: axis 0 is z, axis 2 is x.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

from .fine import kept_mask

# physical axis (x, y, z) of each array axis (0, 1, 2)
PHYS_OF_ARRAY = (2, 1, 0)
VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def vti_stiffness(vp: float, vs: float, eps: float, delta: float, rho: float, gamma: float = 0.0) -> np.ndarray:
    """6 x 6 Voigt stiffness of a VTI medium from Thomsen's parameters (axis z)."""
    if not (0.0 < vs < vp and rho > 0.0 and 1.0 + 2.0 * delta > (vs / vp) ** 2):
        raise ValueError("Thomsen parameters out of range (need 0 < Vs < Vp, rho > 0, 1 + 2 delta > (Vs/Vp)^2)")
    c33 = rho * vp * vp
    c44 = rho * vs * vs
    c11 = c33 * (1.0 + 2.0 * eps)
    c66 = c44 * (1.0 + 2.0 * gamma)
    c13 = math.sqrt((c33 - c44) * (c33 * (1.0 + 2.0 * delta) - c44)) - c44
    c12 = c11 - 2.0 * c66
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = c11
    C[2, 2] = c33
    C[0, 1] = C[1, 0] = c12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = c13
    C[3, 3] = C[4, 4] = c44
    C[5, 5] = c66
    return C


def tensor_from_voigt(C: np.ndarray) -> np.ndarray:
    """C_ijkl (3 x 3 x 3 x 3) from the 6 x 6 Voigt matrix."""
    idx = {}
    for a, (i, j) in enumerate(VOIGT):
        idx[(i, j)] = idx[(j, i)] = a
    T = np.zeros((3, 3, 3, 3))
    for i, j, k, l in itertools.product(range(3), repeat=4):
        T[i, j, k, l] = C[idx[(i, j)], idx[(k, l)]]
    return T


def christoffel(C: np.ndarray, n: np.ndarray, rho: float) -> np.ndarray:
    """Christoffel matrix G_ik = C_ijkl n_j n_l / rho; its eigenvalues are squared phase velocities."""
    T = tensor_from_voigt(C)
    return np.einsum("ijkl,j,l->ik", T, n, n) / rho


def _corner_gradients(h: float):
    """(Gauss weight, G) for the 8 Gauss points of a voxel of edge h: G[c, q] = d N_c / d x_q at the
    point, corner c in C order over the array axes, q a physical axis."""
    g = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))
    corners = list(itertools.product((0, 1), repeat=3))
    out = []
    for xi in itertools.product(g, repeat=3):                 # array-axis coordinates in [0, 1]
        G = np.zeros((8, 3))
        for c, cc in enumerate(corners):
            f = [xi[a] if cc[a] else 1.0 - xi[a] for a in range(3)]
            for a in range(3):
                d = (1.0 if cc[a] else -1.0) / h
                G[c, PHYS_OF_ARRAY[a]] = d * f[(a + 1) % 3] * f[(a + 2) % 3]
        out.append((h ** 3 / 8.0, G))
    return out


def voxel_stiffness(C: np.ndarray, h: float) -> np.ndarray:
    """Q1 element stiffness (24 x 24) of a voxel with constant Voigt stiffness C: dof 3 c + p is
    component p (physical axis) at corner c; K_e = integral of C_pqrs dN_c/dx_q dN_d/dx_s."""
    T = tensor_from_voigt(C)
    K = np.zeros((8, 3, 8, 3))
    for wgt, G in _corner_gradients(h):
        K += wgt * np.einsum("pqrs,cq,ds->cpdr", T, G, G)
    return K.reshape(24, 24)


class ElasticOperator:
    """A (CSR, -K) and diag(B) of the 3D VTI elastic grid; 3 unknowns per kept node, node-major.

    ``C`` is the per-voxel Voigt stiffness, shape (n0, n1, n2, 6, 6), and ``rho`` the per-voxel
    density.  ``index`` maps a full-grid node (C order) to its kept-node number, -1 for removed
    nodes; unknown 3 k + p is component p (physical x, y, z) of kept node k.
    """

    def __init__(self, grid, C: np.ndarray, rho: np.ndarray):
        if grid.dim != 3:
            raise ValueError("the elastic operator is 3D")
        self.grid = grid
        self.keep = kept_mask(grid)
        flat = self.keep.ravel()
        self.index = np.full(flat.size, -1, dtype=np.int64)
        self.index[flat] = np.arange(int(flat.sum()))
        self.nodes = int(flat.sum())
        self.N = 3 * self.nodes
        h = grid.h
        n0, n1, n2 = grid.n
        E = np.zeros((6, 6, 24, 24))                   # K_e is linear in the 36 Voigt entries
        for a in range(6):
            for b in range(6):
                U = np.zeros((6, 6))
                U[a, b] = 1.0
                E[a, b] = voxel_stiffness(U, h)
        Ke = np.einsum("vab,abij->vij", C.reshape(-1, 6, 6), E)
        ids = np.arange(flat.size).reshape(grid.node_shape)
        vox = np.stack(np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij"), -1).reshape(-1, 3)
        corner_nodes = []
        for cc in itertools.product((0, 1), repeat=3):
            p = vox + np.array(cc)
            corner_nodes.append(self.index[ids[p[:, 0], p[:, 1], p[:, 2]]])
        cn = np.stack(corner_nodes, axis=1)                                   # (voxels, 8) kept node or -1
        dof = (3 * cn[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
        dof[np.repeat(cn, 3, axis=1) < 0] = -1
        rows = np.repeat(dof[:, :, None], 24, axis=2)
        cols = np.repeat(dof[:, None, :], 24, axis=1)
        ok = (rows >= 0) & (cols >= 0)
        K = sp.csr_matrix((Ke[ok], (rows[ok], cols[ok])), shape=(self.N, self.N))
        K.sum_duplicates()
        self.A = (-K).tocsr()
        mass = np.zeros(grid.node_shape)
        r = rho * h ** 3 / 8.0
        for cc in itertools.product((0, 1), repeat=3):
            mass[cc[0]:cc[0] + n0, cc[1]:cc[1] + n1, cc[2]:cc[2] + n2] += r
        self.B = np.repeat(mass.ravel()[flat], 3)

    def unknown(self, node, component: int) -> int:
        """Unknown number of a displacement component (0 = x, 1 = y, 2 = z) at an array-order node."""
        flat = int(np.ravel_multi_index(tuple(int(c) for c in node), self.grid.node_shape))
        k = int(self.index[flat])
        return -1 if k < 0 else 3 * k + component
