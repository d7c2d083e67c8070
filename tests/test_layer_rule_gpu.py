"""The per-cell layer-count rule in the library (mss_layer_rule) against the oracle's rule.

The rule (a reading of the dipping-layer workload's per-cell m_i, Section 7) keeps the smallest m
whose ROM transfer function (Eq. tfprj) is within a tolerance of the largest m's at damped test
frequencies.  The library builds the largest m's projection on the GPU (the builder of
mss_build_roms) and evaluates every m from one block LDL^T per test point on the host; the oracle
(``rom.layer_count_rule``, pinned in ``tests/test_oracle_layer_rule.py``) takes dense solves of
each leading block.  Both must give the same m per cell and errors within the builder's CG
tolerance; the chosen m then builds through mss_build_roms.
"""
import numpy as np
import pytest

import synth
from oracle import fine, partition, rom

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-7])
def test_layer_rule_matches_oracle(P, tol):
    """32^3 dipping medium, eight 16^3 cells, 6 modes per face; tolerances that pick m = 3 to 6."""
    wl = synth.workload_3d_dipping(32, 16, m=4, n_modes=6, n_steps=10)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes[:2]) + list(wl.rcv_nodes[:2])]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    bases = [rom.face_basis(f, wl.n_modes) for f in part.faces]
    w = rom.omega_max(wl.f_max)
    s = -w * w
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, np.asarray(io, np.int32))
    cm, err = P.Rom.layer_rule(LP, wl.n_modes, s, w, (3, 6), tol, cg_tol=1e-13)
    assert len(cm) == len(part.cells)
    for cid in range(len(part.cells)):
        m, e, errs = rom.layer_count_rule(part, cid, bases, s, w, (3, 6), tol)
        # same m unless the oracle's error sits within the CG tolerance of the threshold
        near = any(abs(errs[k] - tol) <= 1e-6 * tol + 1e-10 for k in range(3, 7))
        if not near:
            assert int(cm[cid]) == m, (cid, int(cm[cid]), m, errs)
            assert abs(err[cid] - e) <= 1e-6 * max(e, tol) + 1e-10, (cid, err[cid], e)
        assert err[cid] <= tol or cm[cid] == 6
    # the chosen layer counts build (SPD coefficients)
    R = P.Rom.build(LP, 6, wl.n_modes, s, cell_m=cm)
    assert R is not None
