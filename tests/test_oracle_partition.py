"""Pins of the oracle's operator splitting and corner-set removal.

Against: the split coefficients the paper prints (Examples 1d_example, 2dom_ex,
multidom_ex, cs_multidom_ex; fixtures in tests/golden/paper_examples.json),
the splitting identity Eq. splitN_c, diagonal dominance (Proposition prop2),
and the algebra of the hanging-node construction (copy map E with
E^T A' E = A, E^T B' = B; hanging copies per node: 4 on a 2D corner, 4 on a 3D
edge, 12 on a 3D vertex).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import fine, partition

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))


def _uniform(n, bc, h):
    g = synth.Grid(n=tuple(n), h=h, bc=tuple(bc))
    s = np.ones(n)
    return g, s, s.copy()


def _row_dict(A, nodes, u, shape):
    """Row of node u of a (cell) matrix as {offset: value} in array-axis offsets."""
    pos = {int(x): i for i, x in enumerate(nodes)}
    i = pos[u]
    out = {}
    pu = np.array(np.unravel_index(u, shape))
    for j, x in enumerate(nodes):
        if A[i, j] != 0 and j != i:
            px = np.array(np.unravel_index(int(x), shape))
            out[",".join(str(int(v)) for v in (px - pu))] = A[i, j]
    return out, A[i, i]


def _full_index(op):
    inv = np.full(op.N, -1, dtype=np.int64)
    inv[op.index[op.index >= 0]] = np.nonzero(op.index >= 0)[0]
    return inv


def test_example_1d_split():
    """Example 1d_example: two cells of a uniform 1D grid, beta = 1/2."""
    n, h = 8, 0.125
    g, s, r = _uniform((n,), (("D", "D"),), h)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (4,))
    full = _full_index(op)
    gold = GOLD["example_1d_split"]
    sk = op.node_unknown((4,))
    for cid, key in ((0, "A1_row_skeleton"), (1, "A2_row_skeleton")):
        A, B, nodes = part.raw_cell_operator(cid)
        fn = full[nodes]
        row, diag = _row_dict(A / h * h * h, fn, int(full[sk]), g.node_shape)
        exp = {k: v for k, v in gold[key].items() if k != "0"}
        assert set(row) == set(exp)
        for k in exp:
            assert abs(row[k] - exp[k]) < 1e-12
        assert abs(diag - gold[key]["0"]) < 1e-12
        pos = list(nodes).index(sk)
        assert abs(B[pos] / h - gold["B_skeleton"]) < 1e-15
        assert np.allclose(np.delete(B, pos) / h, gold["B_interior"])


def test_example_2dom_split():
    """Example 2dom_ex: two cells in a 2D box, tangential weights and masses halved on Gamma."""
    ny, nx, h = 6, 8, 0.125
    g, s, r = _uniform((ny, nx), (("D", "D"), ("D", "D")), h)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (ny, 4))
    full = _full_index(op)
    gold = GOLD["example_2dom_split"]
    A, B, nodes = part.raw_cell_operator(0)
    fn = full[nodes]
    for q in range(2, ny - 1):
        u = op.node_unknown((q, 4))
        row, diag = _row_dict(A / h ** 2 * h * h, fn, int(full[u]), g.node_shape)
        exp = {k: v for k, v in gold["A1_row_skeleton"].items() if k != "0,0"}
        assert row.keys() == exp.keys()
        for k in exp:
            assert abs(row[k] - exp[k]) < 1e-12
        assert abs(diag - gold["A1_row_skeleton"]["0,0"]) < 1e-12
        assert abs(B[list(nodes).index(u)] / h ** 2 - gold["B_skeleton"]) < 1e-15


@pytest.mark.parametrize("name,pos", [("low_x_side", (5, 4)), ("high_x_side", (5, 8)),
                                       ("low_y_side", (4, 6)), ("high_y_side", (8, 6)),
                                       ("low_low_corner", (4, 4))])
def test_example_multidom_rows(name, pos):
    """Example multidom_ex skeleton rows of cell (1, 1) on a 3x3 grid of 4x4-voxel cells."""
    n, h = 12, 1.0 / 12
    g, s, r = _uniform((n, n), (("D", "D"), ("D", "D")), h)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (4, 4))
    full = _full_index(op)
    cid = 1 * 3 + 1
    A, B, nodes = part.raw_cell_operator(cid)
    exp = GOLD["example_multidom_rules"]["rows"][name]
    u = op.node_unknown(pos)
    row, diag = _row_dict(A, full[nodes], int(full[u]), g.node_shape)
    assert row.keys() == exp["couplings"].keys()
    for k, v in exp["couplings"].items():
        assert abs(row[k] - v) < 1e-12
    assert abs(diag - exp["diag"]) < 1e-12
    assert abs(B[list(nodes).index(u)] / h ** 2 - exp["mass"]) < 1e-15


def _media(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 3.0, n), rng.uniform(0.5, 2.5, n)


@pytest.mark.parametrize("n,cell,bc", [((12, 12), (4, 4), (("D", "D"), ("D", "D"))),
                                       ((8, 12), (4, 3), (("D", "N"), ("N", "D"))),
                                       ((8, 6, 6), (4, 3, 3), (("D", "N"), ("D", "D"), ("N", "D")))])
def test_splitting_identity_and_dominance(n, cell, bc):
    """Eq. splitN_c: sum_i P_i A_i P_i^T = A and sum_i P_i B_i P_i^T = B; Proposition prop2."""
    g = synth.Grid(n=n, h=0.1, bc=bc)
    s, r = _media(n, 7)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, cell)
    A = np.zeros((op.N, op.N))
    B = np.zeros(op.N)
    for c in part.cells:
        Ac, Bc, nodes = part.raw_cell_operator(c.id)
        A[np.ix_(nodes, nodes)] += Ac
        B[nodes] += Bc
        off = Ac - np.diag(np.diag(Ac))
        assert np.all(np.abs(np.diag(Ac)) >= np.abs(off).sum(axis=1) - 1e-13)
        assert np.all(np.diag(Ac) < 0) and np.all(off >= 0)
        assert np.all(Bc > 0)
    Ad = op.A.toarray()
    assert np.max(np.abs(A - Ad)) <= 1e-14 * np.max(np.abs(Ad))
    assert np.max(np.abs(B - op.B)) <= 1e-15 * np.max(op.B)


def test_corner_example_rows():
    """Example cs_multidom_ex: hanging-node rows equal the printed ones up to a common factor,
    i.e. the rows of B'^{-1} A' coincide (uniform medium, 2x2 cells)."""
    n, h = 8, 1.0 / 8
    g, s, r = _uniform((n, n), (("D", "D"), ("D", "D")), h)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, (4, 4))
    Ap, Bp = part.modified_operator()
    Ap = Ap.toarray()
    k = op.node_unknown((4, 4))
    assert part.corner_set == [k]
    gold = GOLD["example_corner_removal"]
    # face of each hanging copy: the faces are segments above/below (x = 4) and left/right (y = 4)
    seen = set()
    for f in sorted(part.node_faces[k]):
        face = part.faces[f]
        hp = part.hanging[(k, f)]
        others = [op.node_unknown(p) for p in [(5, 4), (3, 4), (4, 5), (4, 3)]]
        # direction of the face: the plain neighbour that shares the face
        plain_on_face = [u for u in others if part.plain_prime[u] in face.nodes]
        assert len(plain_on_face) == 1
        nb = np.array(np.unravel_index(int(np.nonzero(op.index == plain_on_face[0])[0][0]), g.node_shape))
        d = tuple(int(v) for v in (nb - np.array([4, 4])))
        name = {(1, 0): "hanging_up", (-1, 0): "hanging_down", (0, 1): "hanging_right", (0, -1): "hanging_left"}[d]
        seen.add(name)
        exp = gold[name]
        row = {}
        for j in np.nonzero(Ap[hp])[0]:
            if j == hp:
                continue
            pj = np.array(np.unravel_index(int(np.nonzero(op.index == part.prime_parent[j])[0][0]), g.node_shape))
            row[",".join(str(int(v)) for v in (pj - np.array([4, 4])))] = Ap[hp, j] / Bp[hp]
        expr = {kk: v / exp["mass"] * h ** -2 for kk, v in exp["couplings"].items()}
        assert row.keys() == expr.keys()
        for kk in expr:
            assert abs(row[kk] - expr[kk]) < 1e-9 * abs(expr[kk])
        assert abs(Ap[hp, hp] / Bp[hp] - exp["diag"] / exp["mass"] * h ** -2) < 1e-9 * h ** -2
    assert len(seen) == 4


@pytest.mark.parametrize("n,cell,bc,io", [
    ((12, 12), (4, 4), (("D", "D"), ("D", "D")), [(6, 6), (4, 4), (10, 2)]),
    ((8, 8, 8), (4, 4, 4), (("D", "N"), ("D", "D"), ("D", "D")), [(8, 2, 6), (4, 4, 4)]),
    ((6, 9, 6), (3, 3, 3), (("N", "N"), ("N", "D"), ("D", "N")), [])])
def test_corner_removal_algebra(n, cell, bc, io):
    """E^T A' E = A, E^T B' = B, A' symmetric non-positive with zero row sums where A has them."""
    g = synth.Grid(n=n, h=0.1, bc=bc)
    s, r = _media(n, 11)
    op = fine.FineOperator(g, s, r)
    part = partition.Partition(op, s, r, cell, io_nodes=io)
    Ap, Bp = part.modified_operator()
    E = part.copy_matrix()
    Ad = op.A.toarray()
    assert np.max(np.abs((E.T @ Ap @ E).toarray() - Ad)) <= 1e-14 * np.max(np.abs(Ad))
    assert np.max(np.abs(E.T @ Bp - op.B)) <= 1e-15 * np.max(op.B)
    Apd = Ap.toarray()
    assert np.array_equal(Apd, Apd.T)
    assert np.linalg.eigvalsh(Apd)[-1] <= 1e-12 * np.max(np.abs(Apd))
    rs = np.abs(Ad.sum(axis=1)) < 1e-12 * np.abs(np.diag(Ad))
    rsp = np.abs(Apd.sum(axis=1)) < 1e-12 * np.abs(np.diag(Apd))
    assert np.all(rsp[np.isin(part.prime_parent, np.nonzero(rs)[0])])
    # every face node belongs to exactly one face after removal (Eq. nocorners)
    owner = {}
    for f in part.faces:
        for x in f.nodes:
            assert x not in owner
            owner[x] = f.id
    # copies per corner-set node: 4 (2D corner / 3D edge) or 12 (3D vertex) away from walls
    counts = sorted(set(len(part.node_faces[u]) for u in part.corner_set))
    if len(n) == 2:
        assert set(counts) <= {2, 4}
    else:
        assert 4 in counts
        if all(nc >= 3 for nc in part.n_cells):
            assert 12 in counts


def test_io_faces():
    """Interior I/O nodes ride on a one-sided face of their cell; skeleton I/O nodes do not."""
    n = (12, 12)
    g = synth.Grid(n=n, h=0.1, bc=(("D", "D"), ("D", "D")))
    s, r = _media(n, 2)
    op = fine.FineOperator(g, s, r)
    io = [(6, 6), (11, 2), (11, 6), (4, 5), (2, 2)]
    part = partition.Partition(op, s, r, (4, 4), io_nodes=io)
    iof = [f for f in part.faces if f.kind == "io"]
    cells = sorted(f.cells[0] for f in iof)
    # (6,6) interior of cell (1,1); (11,2) in cell (2,0); (11,6) in cell (2,1); (2,2) in cell (0,0)
    assert cells == [0, 4, 6, 7]
    assert all(len(f.cells) == 1 for f in iof)
    u45 = op.node_unknown((4, 5))
    assert all(u45 not in f.parents for f in iof)
    gv = part.prime_vectors([(4, 4)])
    hs = np.nonzero(gv[:, 0])[0]
    assert len(hs) == 4 and abs(gv[:, 0].sum() - 1.0) < 1e-15
