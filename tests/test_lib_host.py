"""Native library on the CPU: it loads, exports every entry point of include/mss.h, and its
host-side stage-1 logic (assembly, partition, corner removal, face bases, I/O projection,
ROM import checks) matches the oracle.  No GPU call is made here.
"""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _header_symbols():
    txt = open(os.path.join(ROOT, "include", "mss.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mss_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(P):
    import ctypes
    L = ctypes.CDLL(P.LIB_PATH)
    syms = _header_symbols()
    assert len(syms) >= 30
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    assert set(syms) == set(P.EXPORTED)
    assert P.lib().mss_version().decode().startswith("mss")


CASES = [((12, 12), (4, 4), (("D", "D"), ("D", "D")), [(6, 6), (4, 4), (10, 2)]),
         ((8, 8, 8), (4, 4, 4), (("D", "N"), ("D", "D"), ("D", "D")), [(8, 2, 6), (4, 4, 4)]),
         ((6, 9, 6), (3, 3, 3), (("N", "N"), ("N", "D"), ("D", "N")), []),
         ((16,), (4,), (("D", "N"),), [(9,)])]


@pytest.mark.parametrize("n,cell,bc,io", CASES)
def test_assembly_and_partition_match_oracle(P, n, cell, bc, io):
    from oracle import fine, partition
    g = synth.Grid(n=n, h=0.1, bc=bc)
    rng = np.random.default_rng(11)
    s, r = rng.uniform(0.5, 3, n), rng.uniform(0.5, 2.5, n)
    op = fine.FineOperator(g, s, r)
    L = P.Operator(g, s, r)
    rp, col, val, b = L.export()
    A = sp.csr_matrix((val, col, rp), shape=(L.N, L.N))
    assert L.N == op.N
    assert abs(A - op.A).max() <= 1e-14 * abs(op.A).max()
    assert np.max(np.abs(b - op.B)) <= 1e-15 * op.B.max()
    part = partition.Partition(op, s, r, cell, io_nodes=io)
    LP = P.Partition(L, cell, io)
    info = LP.info()
    assert info[0] == len(part.cells) and info[1] == len(part.faces) and info[2] == part.n_int_faces
    assert info[3] == part.Np and info[4] == len(part.corner_set)
    kind, cells, shape, ptr, nodes, par = LP.faces()
    for f, F in enumerate(part.faces):
        assert kind[f] == (1 if F.kind == "io" else 0)
        assert list(cells[f][:len(F.cells)]) == F.cells
        assert list(nodes[ptr[f]:ptr[f + 1]]) == F.nodes
        assert list(par[ptr[f]:ptr[f + 1]]) == F.parents
        if F.kind == "int":
            assert tuple(shape[f][:len(F.shape)]) == tuple(F.shape)
    for c in part.cells:
        oc = part.build_cell(c.id)
        lc = LP.cell(c.id)
        assert list(lc["faces"]) == oc.faces
        assert list(lc["nodes"]) == list(oc.nodes) and lc["K"] == oc.K
        Ac = sp.csr_matrix((lc["val"], lc["col"], lc["rowptr"]), shape=(len(lc["nodes"]),) * 2)
        assert abs(Ac - oc.A).max() <= 1e-14 * abs(oc.A).max()
        assert np.max(np.abs(lc["B"] - oc.B)) <= 1e-15 * oc.B.max()
    lam = fine.lambda_max(op.A, op.B)
    assert abs(L.lambda_max(1e-10) - lam) <= 1e-6 * lam


def test_rom_import_validation(P):
    topo = synth.box_topology((2, 2), modes=3, m=2)
    co = synth.random_coefficients(topo, seed=1)
    R = P.Rom.import_(topo, co)
    info = R.info()
    assert info[0] == 4 and info[1] == topo.n_faces
    cm, cfp, cf, fM, fc, g, gh, fm = R.export()
    assert np.allclose(g, np.concatenate([x.ravel() for cg in co.gamma for x in cg]), rtol=0, atol=0)
    bad = synth.random_coefficients(topo, seed=1)
    bad.gamma_hat[1][1] = -bad.gamma_hat[1][1]
    with pytest.raises(P.MssError) as e:
        P.Rom.import_(topo, bad)
    assert e.value.status == 5
    topo2 = synth.box_topology((2, 2), modes=3, m=2)
    topo2.cell_faces[0] = topo2.cell_faces[0][:1]
    with pytest.raises(P.MssError) as e:
        P.Rom.import_(topo2, co)
    assert e.value.status == 1
    with pytest.raises(P.MssError):
        R.set_io(0, [], 1, [])           # n_src must be >= 1
    with pytest.raises(P.MssError):
        P.Sim(R, P.FP64, 0.1)            # no I/O yet: refused before any device work


def test_operator_errors(P):
    g = synth.Grid(n=(4, 4), h=0.1, bc=(("D", "D"), ("D", "D")))
    s = np.ones((4, 4))
    s[1, 2] = -1.0
    with pytest.raises(P.MssError) as e:
        P.Operator(g, s, np.ones((4, 4)))
    assert e.value.status == 2
    L = P.Operator(g, np.ones((4, 4)), np.ones((4, 4)))
    with pytest.raises(P.MssError):
        P.Partition(L, (3, 3))           # does not divide
    with pytest.raises(P.MssError):
        P.Partition(L, (2, 2), [(0, 2)])  # I/O node on a Dirichlet wall
