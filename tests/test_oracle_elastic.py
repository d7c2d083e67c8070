"""Pins of the oracle's VTI elastic operator (Q1 finite elements, lumped mass).

* Thomsen's relations: the phase velocities of the Voigt matrix (Christoffel eigenvalues) along
  the symmetry axis and across it, and delta recovered by Thomsen's definition.
* Patch test: a linear displacement field carries exactly the strain energy of its uniform
  strain, and rigid motions carry none.  This is element by element, and for the assembled
  operator of a free (all-Neumann) block.
* The pencil is symmetric and non-positive, negative definite with Dirichlet walls, and its
  lumped mass integrates rho.  The fine-grid leapfrog conserves its discrete energy on it.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import elastic as el
from oracle import fine

RHO = 2.2
VP, VS, EPS, DELTA, GAMMA = 3.2, 1.6, 0.15, 0.07, 0.1


def _C():
    return el.vti_stiffness(VP, VS, EPS, DELTA, RHO, GAMMA)


def test_thomsen_relations():
    C = _C()
    ez, ex = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    vz = np.sort(np.linalg.eigvalsh(el.christoffel(C, ez, RHO)))
    vx = np.sort(np.linalg.eigvalsh(el.christoffel(C, ex, RHO)))
    assert np.allclose(vz, sorted([VP ** 2, VS ** 2, VS ** 2]), rtol=1e-13)
    assert np.allclose(vx, sorted([VP ** 2 * (1 + 2 * EPS), VS ** 2, VS ** 2 * (1 + 2 * GAMMA)]), rtol=1e-13)
    c11, c33, c13, c44 = C[0, 0], C[2, 2], C[0, 2], C[3, 3]
    assert np.isclose(((c13 + c44) ** 2 - (c33 - c44) ** 2) / (2 * c33 * (c33 - c44)), DELTA, rtol=1e-12)
    assert np.isclose((c11 - c33) / (2 * c33), EPS, rtol=1e-13)
    assert np.allclose(C, C.T)
    assert np.linalg.eigvalsh(C)[0] > 0


def _linear_field(points, E):
    """u(x) = E x at physical coordinates, stacked node-major (x, y, z components)."""
    return (points @ E.T).ravel()


def _corner_points(h):
    # corner c in C order over array axes (z, y, x); physical coordinates (x, y, z)
    return np.array([[c[2] * h, c[1] * h, c[0] * h] for c in itertools.product((0, 1), repeat=3)])


def _energy_density(C, E):
    e = 0.5 * (E + E.T)
    v = np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])
    return 0.5 * v @ C @ v


def test_element_patch_test_and_rigid_motions():
    C, h = _C(), 0.37
    K = el.voxel_stiffness(C, h)
    assert np.allclose(K, K.T, atol=1e-14 * np.abs(K).max())
    pts = _corner_points(h)
    rng = np.random.default_rng(5)
    for _ in range(5):
        E = rng.standard_normal((3, 3))
        u = _linear_field(pts, E)
        assert np.isclose(0.5 * u @ K @ u, h ** 3 * _energy_density(C, E), rtol=1e-12)
        W = E - E.T                                       # infinitesimal rotation
        for r in (_linear_field(pts, W), np.tile(rng.standard_normal(3), 8)):
            assert np.abs(K @ r).max() <= 1e-12 * np.abs(K).max() * np.abs(r).max()


def _block(n, bc, medium="uniform"):
    grid = synth.Grid(n=(n, n, n), h=1.0 / n, bc=((bc, bc),) * 3)
    rng = np.random.default_rng(9)
    if medium == "uniform":
        Cv = np.broadcast_to(_C(), (n, n, n, 6, 6)).copy()
        rho = np.full((n, n, n), RHO)
    else:
        # per voxel: Vp in [2, 4.5], Vs / Vp = 0.5, eps and delta in [0, 0.2] (the elastic workload's ranges)
        vp = rng.uniform(2.0, 4.5, n ** 3)
        eps, delta = rng.uniform(0.0, 0.2, n ** 3), rng.uniform(0.0, 0.2, n ** 3)
        rho = rng.uniform(1.5, 2.5, (n, n, n))
        Cv = np.stack([el.vti_stiffness(vp[i], 0.5 * vp[i], eps[i], delta[i], r)
                       for i, r in enumerate(rho.ravel())]).reshape(n, n, n, 6, 6)
    return grid, el.ElasticOperator(grid, Cv, rho), rho


def _node_points(grid, op):
    flat = np.nonzero(op.index >= 0)[0]
    z, y, x = np.unravel_index(flat, grid.node_shape)
    return np.stack([x, y, z], axis=1) * grid.h


@pytest.mark.parametrize("medium", ["uniform", "layered"])
def test_free_block_patch_test_and_null_space(medium):
    grid, op, rho = _block(4, "N", medium)
    A = op.A.toarray()
    assert np.allclose(A, A.T, atol=1e-13 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert ev[-1] <= 1e-12 * np.abs(ev).max()
    assert np.sum(ev > -1e-10 * np.abs(ev).max()) == 6          # 3 translations + 3 rotations
    pts = _node_points(grid, op)
    rng = np.random.default_rng(3)
    W = rng.standard_normal((3, 3))
    for r in (_linear_field(pts, W - W.T), np.tile([1.0, -2.0, 0.5], len(pts))):
        assert np.abs(A @ r).max() <= 1e-12 * np.abs(A).max() * np.abs(r).max()
    if medium == "uniform":
        E = rng.standard_normal((3, 3))
        u = _linear_field(pts, E)
        assert np.isclose(-0.5 * u @ A @ u, _energy_density(_C(), E), rtol=1e-12)   # unit volume
    assert np.isclose(op.B.sum() / 3, rho.sum() * grid.h ** 3, rtol=1e-13)


def test_dirichlet_block_is_negative_definite_and_leapfrog_conserves_energy():
    grid, op, _ = _block(4, "D", "layered")
    ev = np.linalg.eigvalsh(op.A.toarray())
    assert ev[-1] < 0
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.5 * fine.tau_critical(lam)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal((op.N, 1))
    g = np.zeros((op.N, 1))
    q = np.zeros((1, op.N))
    w = np.zeros(300)
    e0 = fine.fine_energy(op.A, op.B, u0, u0, tau)
    # step from (u0, u0) and measure the energy of the last two levels
    u, uo = u0.copy(), u0.copy()
    for n in range(300):
        un = 2 * u - uo + tau * tau * (op.A @ u) / op.B[:, None]
        uo, u = u, un
    assert np.isclose(fine.fine_energy(op.A, op.B, u, uo, tau), e0, rtol=1e-11)
    assert fine.fine_leapfrog(op.A, op.B, g, q, w, tau, 10).shape == (10, 1, 1)
