"""Host part of the library's layer-count rule (mss_layer_rule_cell), on the CPU.

The rule's definition (a reading of the dipping-layer workload's per-cell m_i): the ROM transfer
function of m layers is F^m(z) = S_m^T (A_m + z I)^{-1} S_m with A_m, S_m the leading m K
rows/columns of the largest projection (Eq. tfprj, nested Krylov spaces); the error of m is the
largest relative Frobenius distance to F^{m_hi} over z_j = -w_j^2 + i w_j omega_max / 10,
w_j = j omega_max / n_freq.  The library evaluates every m from one block LDL^T per point; here it
is checked against that definition written out with dense complex solves of each leading block,
on random projections (symmetric A with eigenvalues spread over the band, as a ROM's are), and
the chosen m against the smallest admissible one.  The library is loaded on the CPU (no device
work in this entry point).
"""
import numpy as np
import pytest


def _definition(A, S, K, mh, om, n_freq):
    errs = np.zeros(mh + 1)
    for j in range(1, n_freq + 1):
        w = j * om / n_freq
        z = -w * w + 1j * w * om / 10.0
        F = {}
        for m in range(1, mh + 1):
            n = m * K
            F[m] = S[:n].T @ np.linalg.solve(A[:n, :n] + z * np.eye(n), S[:n])
        for m in range(1, mh):
            errs[m] = max(errs[m], np.linalg.norm(F[m] - F[mh]) / np.linalg.norm(F[mh]))
    return errs


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.mark.parametrize("K,mh,seed", [(3, 4, 0), (7, 6, 1), (12, 5, 2)])
def test_layer_rule_cell_matches_definition(P, K, mh, seed):
    rng = np.random.default_rng(seed)
    n = K * mh
    om = 3.0
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(0, 2 * om * om, n // 2), rng.uniform(0, 20 * om * om, n - n // 2)])
    A = (q * lam) @ q.T
    A = 0.5 * (A + A.T)
    S = rng.standard_normal((n, K))
    ref = _definition(A, S, K, mh, om, 8)
    for tol in (1e-1, 1e-3, 1e-9):
        m, errs = P.Rom.layer_rule_cell(A, S, K, om, (1, mh), tol)
        assert errs[mh] == 0.0
        np.testing.assert_allclose(errs[1:mh], ref[1:mh], rtol=1e-9, atol=1e-14)
        admissible = [k for k in range(1, mh + 1) if (ref[k] if k < mh else 0.0) <= tol]
        assert m == admissible[0]


def test_layer_rule_cell_m_lo_and_errors(P):
    rng = np.random.default_rng(7)
    K, mh = 4, 5
    n = K * mh
    M = rng.standard_normal((n, n))
    A = M @ M.T
    S = rng.standard_normal((n, K))
    m, errs = P.Rom.layer_rule_cell(A, S, K, 2.0, (3, mh), 1e-12)
    assert errs[1] == errs[2] == 0.0 and errs[mh] == 0.0 and m >= 3
    with pytest.raises(P.MssError):
        P.Rom.layer_rule_cell(A, S, K, 2.0, (4, 3), 1e-3)      # m_lo > m_hi
    with pytest.raises(P.MssError):
        P.Rom.layer_rule_cell(A, S, K, -1.0, (1, mh), 1e-3)    # omega_max <= 0
