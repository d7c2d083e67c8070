"""The fine-grid leapfrog on CSR rows (mss_fine_create_unknowns) on the GPU: the elastic VTI pencil
assembled by the library against the oracle's leapfrog on the oracle's pencil, and the acoustic
operator against the stencil kernels of mss_fine_create.

The leapfrog is u^{n+1} = 2u^n - u^{n-1} + tau^2 B^{-1}(A u^n - g w(t_n)), trace n = q^T u^n
(Section 1); the elastic pencil is the one of Section 7's elastic experiment (pinned in
``tests/test_oracle_elastic.py``, assembled by the library in ``tests/test_lib_elastic.py``).
Bars: FP64 within 1e-12, FP32 within 1e-4 (relative L2 over the whole trace).
"""
import numpy as np
import pytest

import synth
from oracle import elastic as el
from oracle import fine

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


def _run(P, fs, nst, w, R, S, prec):
    dt = torch.float64 if prec == P.FP64 else torch.float32
    tr = torch.zeros((nst, R, S), device="cuda", dtype=dt)
    fs.step(nst, torch.tensor(w, device="cuda"), tr)
    torch.cuda.synchronize()
    return tr.cpu().numpy().astype(np.float64)


def test_elastic_fine_leapfrog_matches_oracle(P):
    n = (6, 5, 4)
    g = synth.Grid(n=n, h=0.25, bc=(("D", "N"), ("N", "N"), ("N", "D")))
    C = np.zeros(n + (6, 6))
    rho = np.zeros(n)
    for i in range(n[0]):
        f = 1.0 + 0.5 * i / (n[0] - 1)
        C[i] = el.vti_stiffness(3.0 * f, 1.5 * f, 0.12, 0.05, 2.0 * f, 0.08)
        rho[i] = 2.0 * f
    ref_op = el.ElasticOperator(g, C, rho)
    L = P.Operator.elastic(g, C, rho)
    src = [ref_op.unknown((3, 2, 2), 2), ref_op.unknown((4, 1, 1), 0), ref_op.unknown((2, 3, 2), 1)]
    rcv = [ref_op.unknown((5, 4, 2), c) for c in range(3)] + [ref_op.unknown((1, 2, 3), 2)]
    lam = fine.lambda_max(ref_op.A, ref_op.B)
    tau = 0.5 * fine.tau_critical(lam)
    nst = 300
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    G = np.zeros((ref_op.N, len(src)))
    for j, u in enumerate(src):
        G[u, j] = 1.0
    Q = np.zeros((len(rcv), ref_op.N))
    for j, u in enumerate(rcv):
        Q[j, u] = 1.0
    ref = fine.fine_leapfrog(ref_op.A, ref_op.B, G, Q, w, tau, nst)
    assert np.linalg.norm(ref) > 0
    for prec, tol in ((P.FP64, 1e-12), (P.FP32, 1e-4)):
        fs = P.FineSim.at_unknowns(L, prec, tau, src, rcv)
        out = _run(P, fs, nst, w, len(rcv), len(src), prec)
        assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref), prec


def test_csr_leapfrog_equals_stencil_kernels_on_the_acoustic_operator(P):
    n = (8, 7, 6)
    g = synth.Grid(n=n, h=1.0 / 8, bc=(("D", "N"), ("D", "D"), ("N", "D")))
    rng = np.random.default_rng(9)
    s, r = rng.uniform(0.5, 3, n), rng.uniform(0.5, 2.5, n)
    L = P.Operator(g, s, r)
    srcn = [(4, 3, 3), (2, 5, 1), (6, 2, 4), (5, 5, 5)]
    rcvn = [(7, 6, 2), (3, 3, 3), (1, 1, 5)]
    op = fine.FineOperator(g, s, r)
    tau = 0.5 * fine.tau_critical(fine.lambda_max(op.A, op.B))
    nst = 200
    w = synth.ricker(np.arange(nst) * tau, 0.05 / tau)
    a = _run(P, P.FineSim(L, P.FP64, tau, srcn, rcvn), nst, w, 3, 4, P.FP64)
    b = _run(P, P.FineSim.at_unknowns(L, P.FP64, tau, [L.node(p) for p in srcn], [L.node(p) for p in rcvn]),
             nst, w, 3, 4, P.FP64)
    assert np.linalg.norm(a) > 0
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
    with pytest.raises(P.MssError):
        P.FineSim.at_unknowns(L, P.FP64, tau, [L.N], [0])
