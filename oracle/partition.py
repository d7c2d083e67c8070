"""Coarse cells, operator splitting and corner-set removal.

Section 2 (Eq. part, Eq. splitN_c, Examples 1d_example, 2dom_ex, multidom_ex):
the fine grid is cut into box cells of voxels; cell i receives the terms of its
own voxels, A_i = sum_{v in cell i} A_v and likewise B_i, so that
A + w^2 B = sum_i P_i (A_i + w^2 B_i) P_i^T holds exactly (voxel ownership
reproduces the halving rules of Example multidom_ex on the skeleton).

Section 3 (Eq. nocorners, Example cs_multidom_ex) and Appendix B: a node that
lies on more than one face Gamma_ij is replaced by one hanging node per face.
Reading used here (the paper's example doubles masses and couplings, which
breaks zero row sums of the neighbouring rows): every cell splits its own share
of the node's row -- each edge weight, each Dirichlet loss, the mass -- equally
among its faces that contain the node; an edge between two such nodes goes to
the faces holding both.  The hanging rows then equal the paper's example rows
up to a common factor 1/2 (same B'^{-1} A' rows), A' stays symmetric,
non-positive, with zero row sums, and sum_f b_{k_f} = b_k, which is the mass
balance Appendix D relies on.

I/O faces (reading of Eq. gsupport): sources/receivers that fall inside a cell
(not on the skeleton) become an extra one-sided face of that cell whose nodes
are those I/O nodes (kept uncompressed).
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Sequence, Tuple

import numpy as np
import scipy.sparse as sp

from .fine import FineOperator, voxel_block_terms


class Face:
    """A face Gamma_ij (kind 'int', two cells) or an I/O face (kind 'io', one cell)."""

    def __init__(self, fid: int, kind: str, cells: List[int]):
        self.id = fid
        self.kind = kind
        self.cells = cells
        self.axis = -1
        self.shape: Tuple[int, ...] = ()
        self.nodes: List[int] = []       # prime node ids, face order
        self.parents: List[int] = []     # original unknown of each face node


class Cell:
    """Coarse cell: its faces (ascending id) and, lazily, its split matrices."""

    def __init__(self, cid: int, coords: Tuple[int, ...]):
        self.id = cid
        self.coords = coords
        self.faces: List[int] = []
        self.nodes: np.ndarray = np.zeros(0, dtype=np.int64)   # prime ids: boundary (face order) then interior
        self.K = 0                                               # boundary node count
        self.A = None                                            # sparse, local numbering
        self.B = None


class Partition:
    """Box partition of a fine grid with corner set removed and I/O faces added."""

    def __init__(self, op: FineOperator, sigma: np.ndarray, rho: np.ndarray, cell: Sequence[int],
                 io_nodes: Sequence[Sequence[int]] = ()):
        g = op.grid
        self.op, self.grid, self.sigma, self.rho = op, g, sigma, rho
        self.d = g.dim
        self.cell_size = tuple(int(c) for c in cell)
        for a in range(self.d):
            if g.n[a] % self.cell_size[a] != 0 or self.cell_size[a] < 2:
                raise ValueError("cell size must divide the grid and be >= 2")
        self.n_cells = tuple(g.n[a] // self.cell_size[a] for a in range(self.d))
        cstr = [int(np.prod(self.n_cells[a + 1:])) for a in range(self.d)]
        self.cells = [Cell(i, c) for i, c in enumerate(np.ndindex(*self.n_cells))]
        nshape = g.node_shape
        keep = op.keep

        # ---- interior faces: axis-major, then cell in C order
        self.faces: List[Face] = []
        node_faces: Dict[int, List[int]] = {}
        for a in range(self.d):
            for C in np.ndindex(*self.n_cells):
                if C[a] + 1 >= self.n_cells[a]:
                    continue
                c0 = sum(i * s for i, s in zip(C, cstr))
                f = Face(len(self.faces), "int", [c0, c0 + cstr[a]])
                f.axis = a
                ranges = []
                for b in range(self.d):
                    if b == a:
                        ranges.append([self.cell_size[a] * (C[a] + 1)])
                    else:
                        lo, hi = self.cell_size[b] * C[b], self.cell_size[b] * (C[b] + 1)
                        ranges.append([p for p in range(lo, hi + 1) if self._axis_kept(b, p)])
                f.shape = tuple(len(ranges[b]) for b in range(self.d) if b != a)
                for p in itertools.product(*ranges):
                    flat = int(np.ravel_multi_index(p, nshape))
                    assert keep.ravel()[flat]
                    f.parents.append(int(op.index[flat]))
                    node_faces.setdefault(int(op.index[flat]), []).append(f.id)
                self.faces.append(f)
        self.n_int_faces = len(self.faces)

        # ---- I/O nodes inside a cell -> one I/O face per cell
        io_per_cell: Dict[int, List[int]] = {}
        for p in io_nodes:
            u = op.node_unknown(p)
            if u < 0:
                raise ValueError("I/O node on a Dirichlet wall")
            if u in node_faces:
                continue
            cid = self._cell_of_inner_node(p, cstr)
            io_per_cell.setdefault(cid, [])
            if u not in io_per_cell[cid]:
                io_per_cell[cid].append(u)
        for cid in sorted(io_per_cell):
            f = Face(len(self.faces), "io", [cid])
            f.parents = sorted(io_per_cell[cid])
            f.shape = (len(f.parents),)
            for u in f.parents:
                node_faces[u] = [f.id]
            self.faces.append(f)
        for f in self.faces:
            for c in f.cells:
                self.cells[c].faces.append(f.id)

        # ---- prime numbering: plain nodes (original order), then hanging nodes
        self.node_faces = node_faces
        corner = sorted(u for u, fs in node_faces.items() if len(fs) > 1)
        self.corner_set = corner
        is_corner = np.zeros(op.N, dtype=bool)
        is_corner[corner] = True
        self.plain_prime = np.full(op.N, -1, dtype=np.int64)
        plain = np.nonzero(~is_corner)[0]
        self.plain_prime[plain] = np.arange(plain.size)
        self.hanging: Dict[Tuple[int, int], int] = {}
        nxt = plain.size
        parents = list(plain)
        for u in corner:
            for f in sorted(node_faces[u]):
                self.hanging[(u, f)] = nxt
                parents.append(u)
                nxt += 1
        self.Np = nxt
        self.prime_parent = np.array(parents, dtype=np.int64)
        for f in self.faces:
            f.nodes = [self._prime(u, f.id) for u in f.parents]
        self._is_corner = is_corner
        self._global = None

    # ------------------------------------------------------------------ helpers
    def _axis_kept(self, a: int, p: int) -> bool:
        lo, hi = self.grid.bc[a]
        return not ((p == 0 and lo == "D") or (p == self.grid.n[a] and hi == "D"))

    def _cell_of_inner_node(self, p, cstr) -> int:
        C = []
        for a in range(self.d):
            c = min(int(p[a]) // self.cell_size[a], self.n_cells[a] - 1)
            C.append(c)
        return sum(i * s for i, s in zip(C, cstr))

    def _prime(self, u: int, f: int) -> int:
        if self._is_corner_u(u):
            return self.hanging[(u, f)]
        return int(self.plain_prime[u])

    def _is_corner_u(self, u: int) -> bool:
        return len(self.node_faces.get(u, ())) > 1

    def face_of_cell_holding(self, cid: int, u: int) -> List[int]:
        """Faces of cell ``cid`` that contain original node ``u`` (F_c(u))."""
        return sorted(f for f in self.node_faces.get(u, ()) if cid in self.faces[f].cells)

    # ------------------------------------------------------------------ raw split (before corner removal)
    def raw_cell_operator(self, cid: int):
        """(A_i, diag B_i, original unknowns) of cell i by voxel ownership, corner set kept (Eq. splitN_c)."""
        op, g = self.op, self.grid
        C = self.cells[cid].coords
        lo = [self.cell_size[a] * C[a] for a in range(self.d)]
        vsl = tuple(slice(lo[a], lo[a] + self.cell_size[a]) for a in range(self.d))
        edges, mass = voxel_block_terms(self.sigma[vsl], self.rho[vsl], g.h)
        bshape = tuple(s + 1 for s in self.cell_size)
        loc = np.full(bshape, -1, dtype=np.int64)
        for q in np.ndindex(*bshape):
            p = tuple(lo[a] + q[a] for a in range(self.d))
            loc[q] = op.index[int(np.ravel_multi_index(p, g.node_shape))]
        nodes = np.array(sorted(int(u) for u in loc.ravel() if u >= 0), dtype=np.int64)
        pos = {int(u): i for i, u in enumerate(nodes)}
        n = len(nodes)
        A = np.zeros((n, n))
        for a in range(self.d):
            for q in np.ndindex(*edges[a].shape):
                q2 = list(q)
                q2[a] += 1
                u, v = int(loc[q]), int(loc[tuple(q2)])
                w = float(edges[a][q])
                if u >= 0:
                    A[pos[u], pos[u]] -= w
                if v >= 0:
                    A[pos[v], pos[v]] -= w
                if u >= 0 and v >= 0:
                    A[pos[u], pos[v]] += w
                    A[pos[v], pos[u]] += w
        B = np.zeros(n)
        for q in np.ndindex(*bshape):
            if loc[q] >= 0:
                B[pos[int(loc[q])]] += mass[q]
        return A, B, nodes

    # ------------------------------------------------------------------ cell matrices (Eq. splitN_c)
    def build_cell(self, cid: int) -> Cell:
        c = self.cells[cid]
        if c.A is not None:
            return c
        op, g = self.op, self.grid
        C = c.coords
        lo = [self.cell_size[a] * C[a] for a in range(self.d)]
        vsl = tuple(slice(lo[a], lo[a] + self.cell_size[a]) for a in range(self.d))
        edges, mass = voxel_block_terms(self.sigma[vsl], self.rho[vsl], g.h)
        bshape = tuple(s + 1 for s in self.cell_size)
        # original unknown of each local node of the box (-1 removed)
        loc = np.full(bshape, -1, dtype=np.int64)
        for q in np.ndindex(*bshape):
            p = tuple(lo[a] + q[a] for a in range(self.d))
            loc[q] = op.index[int(np.ravel_multi_index(p, g.node_shape))]

        def copies(u: int) -> List[int]:
            if self._is_corner_u(u):
                return [self.hanging[(u, f)] for f in self.face_of_cell_holding(cid, u)]
            return [int(self.plain_prime[u])]

        rows, cols, vals = [], [], []
        diag: Dict[int, float] = {}
        bvec: Dict[int, float] = {}

        def add_edge(a_, b_, w):
            rows.extend([a_, b_, a_, b_])
            cols.extend([b_, a_, a_, b_])
            vals.extend([w, w, -w, -w])

        for a in range(self.d):
            e = edges[a]
            for q in np.ndindex(*e.shape):
                q2 = list(q)
                q2[a] += 1
                u, v = int(loc[q]), int(loc[tuple(q2)])
                w = float(e[q])
                if u < 0 and v < 0:
                    continue
                if u >= 0 and v >= 0:
                    cu, cv = self._is_corner_u(u), self._is_corner_u(v)
                    if cu and cv:
                        common = sorted(set(self.face_of_cell_holding(cid, u)) &
                                        set(self.face_of_cell_holding(cid, v)))
                        if not common:
                            raise ValueError("edge between corner nodes of different faces")
                        pairs = [(self.hanging[(u, f)], self.hanging[(v, f)]) for f in common]
                    elif cu:
                        pairs = [(h, int(self.plain_prime[v])) for h in copies(u)]
                    elif cv:
                        pairs = [(int(self.plain_prime[u]), h) for h in copies(v)]
                    else:
                        pairs = [(int(self.plain_prime[u]), int(self.plain_prime[v]))]
                    for (x, y) in pairs:
                        add_edge(x, y, w / len(pairs))
                else:
                    k = u if u >= 0 else v
                    cs = copies(k)
                    for x in cs:
                        diag[x] = diag.get(x, 0.0) - w / len(cs)
        for q in np.ndindex(*bshape):
            u = int(loc[q])
            if u < 0:
                continue
            cs = copies(u)
            for x in cs:
                bvec[x] = bvec.get(x, 0.0) + float(mass[q]) / len(cs)
        # local ordering: boundary nodes face by face, then interior nodes ascending
        bnd: List[int] = []
        for f in c.faces:
            bnd.extend(self.faces[f].nodes)
        allp = set(bvec.keys())
        interior = sorted(allp - set(bnd))
        order = bnd + interior
        if len(set(order)) != len(order) or set(order) != allp:
            raise AssertionError("cell boundary/interior split is inconsistent")
        pos = {p: i for i, p in enumerate(order)}
        n = len(order)
        rr = [pos[x] for x in rows] + [pos[x] for x in diag]
        cc = [pos[x] for x in cols] + [pos[x] for x in diag]
        vv = vals + list(diag.values())
        c.A = sp.csr_matrix((vv, (rr, cc)), shape=(n, n))
        c.A.sum_duplicates()
        c.B = np.array([bvec[p] for p in order])
        c.nodes = np.array(order, dtype=np.int64)
        c.K = len(bnd)
        return c

    # ------------------------------------------------------------------ global modified operator
    def modified_operator(self):
        """A' = sum_i P_i A_i P_i^T and diag(B') on the prime nodes (corner set removed)."""
        if self._global is None:
            rows, cols, vals = [], [], []
            B = np.zeros(self.Np)
            for c in self.cells:
                self.build_cell(c.id)
                coo = c.A.tocoo()
                rows.append(c.nodes[coo.row])
                cols.append(c.nodes[coo.col])
                vals.append(coo.data)
                np.add.at(B, c.nodes, c.B)
            A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(self.Np, self.Np))
            A.sum_duplicates()
            self._global = (A, B)
        return self._global

    def copy_matrix(self) -> sp.csr_matrix:
        """E: original unknowns -> prime nodes, (E u)_{k_f} = u_k (Appendix B)."""
        return sp.csr_matrix((np.ones(self.Np), (np.arange(self.Np), self.prime_parent)),
                             shape=(self.Np, self.op.N))

    def cell_node_mass(self, cid: int, u: int) -> float:
        """Mass b^c_k of original node u contributed by the voxels of cell cid (Eq. splitN_c)."""
        g = self.grid
        C = self.cells[cid].coords
        p = np.unravel_index(int(np.nonzero(self.op.index == u)[0][0]), g.node_shape)
        tot = 0.0
        for off in itertools.product((-1, 0), repeat=self.d):
            v = tuple(int(p[a]) + off[a] for a in range(self.d))
            if any(v[a] < self.cell_size[a] * C[a] or v[a] >= self.cell_size[a] * (C[a] + 1)
                   for a in range(self.d)):
                continue
            tot += float(self.rho[v]) * g.h ** self.d / 2 ** self.d
        return tot

    def hanging_mass(self, u: int, f: int) -> float:
        """b'_{k_f}: every cell of face f holding k gives b^c_k / |F_c(k)|."""
        tot = 0.0
        for c in self.faces[f].cells:
            fs = self.face_of_cell_holding(c, u)
            if f in fs:
                tot += self.cell_node_mass(c, u) / len(fs)
        return tot

    def distribute(self, node) -> Dict[int, float]:
        """Weights of an original node on its prime copies: b_{k_f} / b_k (1 for a plain node)."""
        u = self.op.node_unknown(node)
        if u < 0:
            raise ValueError("node removed by a Dirichlet wall")
        if not self._is_corner_u(u):
            return {int(self.plain_prime[u]): 1.0}
        fs = sorted(self.node_faces[u])
        ms = [self.hanging_mass(u, f) for f in fs]
        tot = sum(ms)
        return {self.hanging[(u, f)]: float(mf / tot) for f, mf in zip(fs, ms)}

    def prime_vectors(self, nodes: Sequence[Sequence[int]], weights=None) -> np.ndarray:
        """Columns g' (prime-node space) of point sources/receivers at ``nodes``."""
        out = np.zeros((self.Np, len(nodes)))
        for j, p in enumerate(nodes):
            wj = 1.0 if weights is None else float(weights[j])
            for h, val in self.distribute(p).items():
                out[h, j] += wj * val
        return out

    # ------------------------------------------------------------------ Appendix D data
    def corner_groups(self):
        """For every corner-set node k: [(face, row of k_f in the face, b_{k_f} / b_k)] (Appendix D)."""
        out = []
        for u in self.corner_set:
            fs = sorted(self.node_faces[u])
            ms = [self.hanging_mass(u, f) for f in fs]
            tot = sum(ms)
            grp = []
            for f, mf in zip(fs, ms):
                r = self.faces[f].nodes.index(self.hanging[(u, f)])
                grp.append((f, r, mf / tot))
            out.append(grp)
        return out
