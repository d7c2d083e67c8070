"""Pins of the oracle's fine-grid assembly and leapfrog (Section 1, Eq. wave_fll).

Checked against: the textbook stencil built by an independent route (Kronecker
sums of 1D operators), symmetry / non-positivity / zero row sums (Section 1:
0 >= A = A^T), the exact discrete modal solution of leapfrog in a homogeneous
box, conservation of the discrete leapfrog energy, and the CFL bound.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import fine


def _grid(n, bc, h=None):
    return synth.Grid(n=tuple(n), h=h if h else 1.0 / n[-1], bc=tuple(bc))


def _media(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 3.0, n), rng.uniform(0.5, 2.5, n)


@pytest.mark.parametrize("n,bc", [((6, 7), (("D", "D"), ("D", "D"))),
                                  ((5, 6), (("D", "N"), ("N", "D"))),
                                  ((4, 5, 3), (("D", "N"), ("D", "D"), ("N", "N")))])
def test_assembly_symmetric_nonpositive(n, bc):
    g = _grid(n, bc)
    s, r = _media(n)
    op = fine.FineOperator(g, s, r)
    A = op.A.toarray()
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert ev[-1] <= 1e-12 * abs(ev[0])
    assert np.all(op.B > 0)
    # zero row sums on rows with no removed (Dirichlet) neighbour
    keep = op.keep
    ids = np.arange(keep.size).reshape(keep.shape)
    for idx in np.ndindex(*keep.shape):
        u = op.index[ids[idx]]
        if u < 0:
            continue
        touches = False
        for a in range(len(n)):
            for dlt in (-1, 1):
                j = list(idx)
                j[a] += dlt
                if 0 <= j[a] < keep.shape[a] and not keep[tuple(j)]:
                    touches = True
        if not touches:
            assert abs(A[u].sum()) <= 1e-13 * abs(A[u, u])


def _kron_1d(nv, h, lo, hi):
    """1D stiffness K (edge weight 1/h) and masses M (h, h/2 at a kept wall) on the kept nodes."""
    nn = nv + 1
    K = np.zeros((nn, nn))
    for i in range(nv):
        K[i, i] -= 1 / h
        K[i + 1, i + 1] -= 1 / h
        K[i, i + 1] += 1 / h
        K[i + 1, i] += 1 / h
    M = np.full(nn, h)
    M[0] = M[-1] = h / 2
    keep = np.ones(nn, bool)
    if lo == "D":
        keep[0] = False
    if hi == "D":
        keep[-1] = False
    return K[np.ix_(keep, keep)], np.diag(M[keep])


@pytest.mark.parametrize("n,bc", [((5, 7), (("D", "D"), ("D", "D"))),
                                  ((6, 5), (("D", "N"), ("D", "D"))),
                                  ((4, 3, 5), (("D", "N"), ("N", "D"), ("D", "D")))])
def test_uniform_medium_is_textbook_stencil(n, bc):
    """Uniform sigma, rho: A = sigma * sum_a (x)_{b != a} M_b (x) K_a, B = rho * (x)_a M_a."""
    h = 0.1
    g = _grid(n, bc, h)
    sig, rho = 2.5, 1.5
    op = fine.FineOperator(g, np.full(n, sig), np.full(n, rho))
    ks = [_kron_1d(n[a], h, *bc[a]) for a in range(len(n))]
    A = 0
    for a in range(len(n)):
        term = np.ones((1, 1))
        for b in range(len(n)):
            term = np.kron(term, ks[b][0] if b == a else ks[b][1])
        A = A + term
    B = np.ones((1, 1))
    for b in range(len(n)):
        B = np.kron(B, ks[b][1])
    assert np.allclose(op.A.toarray(), sig * A, rtol=0, atol=1e-14 * sig * np.abs(A).max())
    assert np.allclose(op.B, rho * np.diag(B), rtol=1e-15)
    # interior rows: (sigma/rho) * textbook (sum of neighbours - 2d u) / h^2
    L = op.A.toarray() / op.B[:, None]
    d = len(n)
    inner = [i for i in range(op.N) if np.count_nonzero(L[i]) == 2 * d + 1]
    assert inner, "no interior rows"
    for i in inner:
        nb = [j for j in range(op.N) if j != i and L[i, j] != 0]
        if not np.allclose(L[i, nb], sig / rho / h ** 2):
            continue                                   # a Neumann-wall row (half weights, half mass)
        assert abs(L[i, i] + 2 * d * sig / rho / h ** 2) < 1e-9 / h ** 2


def test_leapfrog_discrete_modal_closed_form():
    """Homogeneous Dirichlet box, initial sine mode: u^n = cos(n theta) phi, cos theta = 1 - tau^2 lam / 2."""
    nx, ny = 12, 9
    h = 1.0 / 12
    g = synth.Grid(n=(ny, nx), h=h, bc=(("D", "D"), ("D", "D")))
    c2 = 2.0
    op = fine.FineOperator(g, np.full((ny, nx), c2), np.ones((ny, nx)))
    j, k = 3, 2                                   # mode numbers along x and y
    yy, xx = np.meshgrid(np.arange(1, ny), np.arange(1, nx), indexing="ij")
    phi = (np.sin(math.pi * j * xx / nx) * np.sin(math.pi * k * yy / ny)).ravel()[:, None]
    lam = c2 * (4 / h ** 2) * (math.sin(math.pi * j / (2 * nx)) ** 2 + math.sin(math.pi * k / (2 * ny)) ** 2)
    tau = 0.9 * 2 / math.sqrt(c2 * 8 / h ** 2)
    th = math.acos(1 - tau * tau * lam / 2)
    nst = 400
    q = np.eye(op.N)[[5, 40, 77]]
    out = fine.fine_leapfrog(op.A, op.B, np.zeros((op.N, 1)), q, np.zeros(nst), tau, nst,
                             u0=phi, um1=math.cos(th) * phi)
    ref = np.cos(th * np.arange(nst))[:, None, None] * (q @ phi)[None]
    assert np.max(np.abs(out - ref)) < 1e-11


def test_leapfrog_energy_conserved():
    n = (7, 8, 6)
    g = _grid(n, (("D", "N"), ("D", "D"), ("N", "D")))
    s, r = _media(n, 3)
    op = fine.FineOperator(g, s, r)
    lam = fine.lambda_max(op.A, op.B)
    tau = 0.8 * fine.tau_critical(lam)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal((op.N, 2))
    um1 = rng.standard_normal((op.N, 2))
    e0 = fine.fine_energy(op.A, op.B, u0, um1, tau)
    u, uo = u0, um1
    binv = 1.0 / op.B[:, None]
    for _ in range(300):
        u, uo = 2 * u - uo + tau * tau * binv * (op.A @ u), u
    # recompute through the oracle's stepping for the last level pair
    e1 = fine.fine_energy(op.A, op.B, u, uo, tau)
    assert abs(e1 - e0) <= 1e-11 * abs(e0)
    out = fine.fine_leapfrog(op.A, op.B, np.zeros((op.N, 2)), np.eye(op.N)[:3], np.zeros(300), tau, 300,
                             u0=u0, um1=um1)
    ref = np.zeros_like(out)
    u, uo = u0, um1
    for n_ in range(300):
        ref[n_] = u[:3]
        u, uo = 2 * u - uo + tau * tau * binv * (op.A @ u), u
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_cfl_bound():
    n = (8, 9)
    g = _grid(n, (("D", "D"), ("D", "D")))
    s, r = _media(n, 5)
    op = fine.FineOperator(g, s, r)
    Ad = op.A.toarray()
    lam = float(np.max(np.linalg.eigvals(-Ad / op.B[:, None]).real))
    assert abs(fine.lambda_max(op.A, op.B) - lam) < 1e-9 * lam
    rng = np.random.default_rng(2)
    x0 = rng.standard_normal((op.N, 1))
    for frac, grows in ((0.99, False), (1.01, True)):
        tau = frac * 2 / math.sqrt(lam)
        out = fine.fine_leapfrog(op.A, op.B, np.zeros((op.N, 1)), np.eye(op.N), np.zeros(600), tau, 600,
                                 u0=x0, um1=x0)
        amp = np.max(np.abs(out[-50:]))
        assert (amp > 1e6 * np.max(np.abs(x0))) == grows


def test_voxel_assembly_local_sum():
    """The per-voxel rule: each voxel adds sigma h^(d-2)/2^(d-1) per edge and rho h^d/2^d per corner."""
    h = 0.25
    s = np.array([[3.0]])
    r = np.array([[2.0]])
    edges, mass = fine.voxel_block_terms(s, r, h)
    assert np.allclose(mass, 2.0 * h * h / 4)
    for e in edges:
        assert np.allclose(e, 3.0 / 2)
    s3 = np.array([[[3.0]]])
    edges, mass = fine.voxel_block_terms(s3, s3 * 0 + 2.0, h)
    assert np.allclose(mass, 2.0 * h ** 3 / 8)
    for e in edges:
        assert np.allclose(e, 3.0 * h / 4)
