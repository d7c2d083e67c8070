"""CFL check of the on-line step (mss_sim_check_stability) against the oracle's global ROM pencil.

The leapfrog of M x_tt = -K x is stable iff tau^2 lambda_max(M^-1 K) < 4; the oracle assembles
M and K of the coupled ROM (rom_pencil) and takes lambda_max from a dense generalized eigen-
solve.  Just below tau_crit the GPU check passes and leaves the sim's state untouched; just
above it reports MSS_ERR_CFL.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import freq

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

CFL = 6


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.fixture(scope="module")
def case():
    topo = synth.box_topology((3, 2, 2), modes=5, m=[2, 3, 4] * 4, io_cells=[(0, 2), (7, 3)], seed=8,
                              ragged_modes=True)
    co = synth.random_coefficients(topo, seed=8)
    src, rcv = synth.random_io(topo, 8, 4, seed=8)
    Kg, Mg, _ = freq.rom_pencil(topo, co)
    lam = float(sla.eigh(Kg, Mg, eigvals_only=True)[-1])
    return topo, co, src, rcv, 2.0 / np.sqrt(lam)


def _sim(P, case, prec, tau):
    topo, co, src, rcv, _ = case
    R = P.Rom.import_(topo, co)
    R.set_io(8, src, 4, rcv)
    return P.Sim(R, prec, tau)


@pytest.mark.parametrize("prec", [0, 1])
def test_cfl_check_brackets_the_oracle_limit(P, case, prec):
    tau_crit = case[4]
    sim = _sim(P, case, prec, 0.95 * tau_crit)
    w = torch.tensor(synth.ricker(np.arange(50) * 0.95 * tau_crit, 0.5), device="cuda")
    dt = torch.float64 if prec == 0 else torch.float32
    tr = torch.zeros((50, 4, 8), device="cuda", dtype=dt)
    sim.step(20, w, tr)
    torch.cuda.synchronize()
    before = sim.save_state()
    g = sim.check_stability(300, seed=1)
    assert 0 < g < 1e3
    after = sim.save_state()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1]) and before[2] == after[2]
    bad = _sim(P, case, prec, 1.05 * tau_crit)
    with pytest.raises(P.MssError) as e:
        bad.check_stability(300, seed=1)
    assert e.value.status == CFL
