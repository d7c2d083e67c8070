"""The library's elastic assembly (mss_assemble_elastic) against the oracle's VTI pencil, on the CPU.

The oracle's operator (``oracle/elastic.py``) is pinned by Thomsen's relations, the patch test,
rigid-motion null spaces and energy conservation (``tests/test_oracle_elastic.py``).  The
library's C++ assembly must give the same pencil: the same unknown numbering (3 per kept node,
node-major), the same A entry by entry and the same lumped mass, on a layered VTI medium with
mixed Dirichlet / Neumann walls and a random anisotropic medium.  It is also checked on its own
terms: A symmetric, rigid motions in the null space of a free block, lambda_max of -B^{-1}A against
a dense eigensolver.  Consumers that take one unknown per node refuse it.
"""
import numpy as np
import pytest

import synth
from oracle import elastic as el

RHO = 2.2
VP, VS, EPS, DELTA, GAMMA = 3.2, 1.6, 0.15, 0.07, 0.1


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _layered(n):
    C = np.zeros(tuple(n) + (6, 6))
    rho = np.zeros(tuple(n))
    for i in range(n[0]):
        f = 1.0 + 0.4 * i / max(1, n[0] - 1)
        C[i] = el.vti_stiffness(VP * f, VS * f, EPS, DELTA, RHO * f, GAMMA)
        rho[i] = RHO * f
    return C, rho


def _random_aniso(n, seed):
    rng = np.random.default_rng(seed)
    C = np.zeros(tuple(n) + (6, 6))
    for idx in np.ndindex(*n):
        M = rng.standard_normal((6, 6))
        C[idx] = M @ M.T + 6.0 * np.eye(6)
    return C, rng.uniform(0.8, 2.5, n)


def _dense(P_op):
    rp, col, val, b = P_op.export()
    A = np.zeros((P_op.N, P_op.N))
    for r in range(P_op.N):
        A[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    return A, b, rp, col


@pytest.mark.parametrize("medium", ["layered", "random"])
def test_elastic_assembly_matches_oracle(P, medium):
    n = (3, 4, 2)
    g = synth.Grid(n=n, h=0.3, bc=(("D", "N"), ("N", "D"), ("N", "N")))
    C, rho = _layered(n) if medium == "layered" else _random_aniso(n, 5)
    ref = el.ElasticOperator(g, C, rho)
    L = P.Operator.elastic(g, C, rho)
    assert L.N == ref.N
    A, b, rp, col = _dense(L)
    Aref = ref.A.toarray()
    assert np.linalg.norm(A - Aref) <= 1e-13 * np.linalg.norm(Aref)
    assert np.allclose(b, ref.B, rtol=1e-14, atol=0)
    assert np.array_equal(A, A.T) or np.linalg.norm(A - A.T) <= 1e-14 * np.linalg.norm(A)
    for r in range(L.N):                       # columns ascending, the diagonal present
        c = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c) > 0) and r in c
    for node in [(0, 0, 0), (1, 2, 1), (3, 4, 2), (2, 0, 2)]:
        assert L.node(node) == ref.unknown(node, 0)


def test_free_block_rigid_motions_and_lambda_max(P):
    n = (2, 3, 2)
    h = 0.5
    g = synth.Grid(n=n, h=h, bc=(("N", "N"), ("N", "N"), ("N", "N")))
    C, rho = _layered(n)
    L = P.Operator.elastic(g, C, rho)
    A, b, _, _ = _dense(L)
    # node coordinates in physical axes (x, y, z) = array axes (2, 1, 0), node-major unknowns
    pts = np.array([[i2 * h, i1 * h, i0 * h] for i0, i1, i2 in np.ndindex(n[0] + 1, n[1] + 1, n[2] + 1)])
    motions = [np.tile(e, len(pts)) for e in np.eye(3)]
    for axis in range(3):                      # infinitesimal rotations: u = w x r
        w = np.eye(3)[axis]
        motions.append(np.cross(np.tile(w, (len(pts), 1)), pts).ravel())
    for u in motions:
        assert np.linalg.norm(A @ u) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(u)
    lam = np.linalg.eigvalsh(-A / np.sqrt(np.outer(b, b)))
    assert abs(L.lambda_max(1e-12) - lam[-1]) <= 1e-8 * lam[-1]
    assert lam[0] > -1e-10 * lam[-1]            # -A positive semidefinite


def test_elastic_operator_refusals(P):
    n = (2, 2, 2)
    g = synth.Grid(n=n, h=0.5, bc=(("D", "D"), ("D", "D"), ("D", "D")))
    C, rho = _layered(n)
    bad = C.copy()
    bad[0, 0, 0, 0, 1] += 1.0                  # not symmetric
    with pytest.raises(P.MssError):
        P.Operator.elastic(g, bad, rho)
    neg = C.copy()
    neg[1, 1, 1] = -np.eye(6)                  # not positive definite
    with pytest.raises(P.MssError):
        P.Operator.elastic(g, neg, rho)
    with pytest.raises(P.MssError):
        P.Operator.elastic(synth.Grid(n=(4, 4), h=0.5, bc=(("D", "D"), ("D", "D"))), C[0], rho[0])
    L = P.Operator.elastic(g, C, rho)
    with pytest.raises(P.MssError):            # one unknown per node: the partition refuses it
        P.Partition(L, (1, 1, 1), np.zeros((0, 3), np.int32))


def test_patch_test_linear_fields(P):
    """A linear displacement u = E x carries exactly the strain energy of its uniform strain:
    -u^T A u = V e^T C e, e the Voigt strain (xx, yy, zz, 2yz, 2xz, 2xy) of sym(E), V the block's
    volume, on a free block with a different anisotropic stiffness in every voxel (the element
    integration is exact for constant C per voxel, so the sum over voxels is exact too)."""
    n = (2, 2, 3)
    h = 0.4
    g = synth.Grid(n=n, h=h, bc=(("N", "N"), ("N", "N"), ("N", "N")))
    C, rho = _random_aniso(n, 11)
    L = P.Operator.elastic(g, C, rho)
    A, _, _, _ = _dense(L)
    pts = np.array([[i2 * h, i1 * h, i0 * h] for i0, i1, i2 in np.ndindex(n[0] + 1, n[1] + 1, n[2] + 1)])
    rng = np.random.default_rng(3)
    for _ in range(4):
        E = rng.standard_normal((3, 3))
        u = (pts @ E.T).ravel()
        eps = 0.5 * (E + E.T)
        e = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[1, 2], 2 * eps[0, 2], 2 * eps[0, 1]])
        exact = sum(h ** 3 * e @ C[idx] @ e for idx in np.ndindex(*n))
        assert abs(-u @ A @ u - exact) <= 1e-11 * abs(exact)
