"""The paper's own boundary basis through the GPU off-line builder (mss_partition_set_face_bases ->
mss_build_roms) against the oracle's build on the same bases.

Section 4.1 builds S_f from the frequency-limited Gramian of the face traces (Eq. trgr); the
oracle computes it from the propagative eigenpairs of the whole pencil (``rom.gramian_bases``).
Two bases are passed to the library: the Gramian's leading eigenvectors, and a hybrid (the
Gramian's numerical range, completed by DCT modes orthogonalised against it), which keeps every
column inside the propagative subspace where the Gramian has rank and adds smooth modes beyond
it.  Given S_f the S-fraction coefficients are unique (Section 5), so Gamma^k, Gamma-hat^k and
the face masses are compared entry by entry (the bar of the other off-line tests, 1e-7: CG at
1e-13 against the oracle's exact factorisations), and the FP64 on-line traces to 1e-7.
"""
import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-7


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _hybrid(part, gram, n_modes, cutoff=1e-8):
    """Gramian eigenvectors above ``cutoff`` of the largest eigenvalue, then DCT modes projected
    off them and orthonormalised (QR), up to n_modes columns per face."""
    out = []
    for f, G in zip(part.faces, gram):
        if G is None:
            out.append(None)
            continue
        w, Q = np.linalg.eigh(G)
        w, Q = w[::-1], Q[:, ::-1]
        r = int(np.sum(w > cutoff * max(w[0], 1e-300)))
        M = min(n_modes, len(f.nodes))
        keep = Q[:, :min(r, M)]
        if keep.shape[1] < M:
            dct = rom.face_basis(f, len(f.nodes))
            extra = dct - keep @ (keep.T @ dct)
            q, rr = np.linalg.qr(extra)
            order = np.argsort(-np.abs(np.diag(rr)), kind="stable")[:M - keep.shape[1]]
            keep = np.hstack([keep, q[:, np.sort(order)]])
        out.append(keep)
    return out


@pytest.fixture(scope="module")
def case():
    """32^3 layered medium at the one-cell band: eight 16^3 cells, five propagative modes."""
    wl = synth.workload_3d_layers(32, 16, m=3, n_modes=6, n_src=2, n_steps=300, band="cell")
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    s = -rom.omega_max(wl.f_max) ** 2
    modes = rom.propagative_modes(part.op.A, part.op.B, -s)
    return wl, op, part, s, modes, rom.face_gramians(part, modes)


@pytest.mark.parametrize("kind", ["gramian", "hybrid"])
def test_gpu_build_on_paper_face_bases(P, case, kind):
    wl, op, part, s, modes, gram = case
    if kind == "gramian":
        given = [None if f.kind == "io" else b for f, b in zip(part.faces, rom.gramian_bases(part, -s, 6, modes))]
    else:
        given = _hybrid(part, gram, 6)
    bases = [rom.face_basis(f, 6) if b is None else b for f, b in zip(part.faces, given)]
    for b in given:
        if b is not None:
            assert np.allclose(b.T @ b, np.eye(b.shape[1]), atol=1e-12)
    R = rom.build_rom(part, wl.m, wl.n_modes, s, bases=bases)
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, np.concatenate([wl.src_nodes, wl.rcv_nodes]).astype(np.int32))
    LP.set_face_bases(given)
    LR = P.Rom.build(LP, wl.m, wl.n_modes, s, cg_tol=1e-13)
    cm, cfp, cf, fM, fc, g, gh, fm = LR.export()
    assert list(fM) == list(R.topology.face_M)
    o = 0
    for c in range(R.topology.n_cells):
        K = int(R.topology.cell_K()[c])
        for k in range(wl.m):
            for arr, ref in ((g, R.coeffs.gamma[c][k]), (gh, R.coeffs.gamma_hat[c][k])):
                blk = arr[o + k * K * K:o + (k + 1) * K * K].reshape(K, K)
                assert np.linalg.norm(blk - ref) <= TOL * np.linalg.norm(ref), (c, k)
        o += wl.m * K * K
    o = 0
    for f, M in enumerate(fM):
        ref = R.coeffs.face_mass[f]
        assert np.linalg.norm(fm[o:o + M * M].reshape(M, M) - ref) <= TOL * np.linalg.norm(ref)
        o += M * M
    # end to end: projected I/O through the library's own bases, FP64 stepping vs the oracle
    lam = fine.lambda_max(op.A, op.B)
    tau = wl.cfl_fraction * fine.tau_critical(lam)
    gp, qp = part.prime_vectors(wl.src_nodes), part.prime_vectors(wl.rcv_nodes)
    gt = rom.project_io(part, R.bases, gp)
    qt = [x.T for x in rom.project_io(part, R.bases, qp)]
    w = synth.ricker(np.arange(wl.n_steps) * tau, wl.f_peak)
    cr = online.corner_rows(part.corner_groups(), R.bases)
    ref = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, wl.n_steps, corners=cr)
    LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
    sim = P.Sim(LR, P.FP64, tau, corner_correction=True)
    tr = torch.zeros((wl.n_steps, len(wl.rcv_nodes), len(wl.src_nodes)), device="cuda", dtype=torch.float64)
    sim.step(wl.n_steps, torch.tensor(w, device="cuda"), tr)
    torch.cuda.synchronize()
    out = tr.cpu().numpy()
    assert np.linalg.norm(out - ref) <= TOL * np.linalg.norm(ref)

