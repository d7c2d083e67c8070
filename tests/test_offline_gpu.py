"""Off-line stage on the GPU (mss_build_roms, FP64) against the oracle.

Given the face bases, the S-fraction coefficients are unique (Section 5), so the GPU's
Gamma^k, Gamma-hat^k and face masses are compared entry by entry with the oracle's.  The GPU
solves the shifted systems by CG to a relative residual of 1e-13 where the oracle factors them
exactly; the Krylov basis then differs by ~1e-13 times the conditioning of the block
orthogonalisation and Lanczos steps (~1e3..1e5 here), hence the 1e-7 bar on coefficients and
on end-to-end traces.  Integer data (topology, corner groups) are compared exactly.
"""
import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

COEF_TOL = 1e-7


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _setup(wl):
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    lam = fine.lambda_max(op.A, op.B) if op.N <= 2000 else None
    return op, part, io, lam


def _cases():
    yield "2d_16cells", synth.workload_2d_layers(32, 8, m=3, n_modes=4, n_steps=200)
    yield "3d_8cells", synth.workload_3d_layers(16, 8, m=3, n_modes=6, n_src=2, n_steps=150)


@pytest.mark.parametrize("name,wl", list(_cases()))
def test_build_roms_matches_oracle(P, name, wl):
    op, part, io, _ = _setup(wl)
    s = -rom.omega_max(wl.f_max) ** 2
    R = rom.build_rom(part, wl.m, wl.n_modes, s)
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, io)
    LR = P.Rom.build(LP, wl.m, wl.n_modes, s, cg_tol=1e-13)
    cm, cfp, cf, fM, fc, g, gh, fm = LR.export()
    assert list(fM) == list(R.topology.face_M)
    assert list(cm) == list(R.topology.cell_m)
    for c in range(len(part.cells)):
        assert list(cf[cfp[c]:cfp[c + 1]]) == R.topology.cell_faces[c]
    # coefficients, cell by cell
    o = 0
    for c in range(len(part.cells)):
        K = int(R.topology.cell_K()[c])
        for k in range(wl.m):
            for lib_arr, ref in ((g, R.coeffs.gamma[c][k]), (gh, R.coeffs.gamma_hat[c][k])):
                blk = lib_arr[o + k * K * K:o + (k + 1) * K * K].reshape(K, K)
                assert np.linalg.norm(blk - ref) <= COEF_TOL * np.linalg.norm(ref), (c, k)
        o += wl.m * K * K
    o = 0
    for f, M in enumerate(R.topology.face_M):
        blk = fm[o:o + M * M].reshape(M, M)
        assert np.linalg.norm(blk - R.coeffs.face_mass[f]) <= COEF_TOL * np.linalg.norm(R.coeffs.face_mass[f])
        o += M * M
    # face bases are the same closed form on both sides
    bases = LR.face_bases()
    o = 0
    for f, B in enumerate(R.bases):
        assert np.allclose(bases[o:o + B.size].reshape(B.shape), B, rtol=0, atol=1e-14)
        o += B.size


@pytest.mark.parametrize("name,wl", [("2d_16cells", synth.workload_2d_layers(32, 8, m=3, n_modes=4, n_steps=10)),
                                     ("3d_8cells", synth.workload_3d_layers(16, 8, m=3, n_modes=6, n_src=2,
                                                                           n_steps=10))])
def test_io_projection_and_corners_match_oracle(P, name, wl):
    """g~_f = S_f^T g|_f, q~_f = S_f^T q|_f (Eqs. BEINCr, solatrec; corner-set nodes spread over their
    hanging copies by b_{k_f}/b_k) and the Appendix D rows of the GPU-built ROM, entry by entry
    against the oracle's projections of the same nodes."""
    op, part, io, _ = _setup(wl)
    s = -rom.omega_max(wl.f_max) ** 2
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, io)
    LR = P.Rom.build(LP, wl.m, wl.n_modes, s)
    LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
    src, rcv, groups = LR.export_io()
    bases = [rom.face_basis(f, wl.n_modes) for f in part.faces]
    nS, nR = len(wl.src_nodes), len(wl.rcv_nodes)
    gt = rom.project_io(part, bases, part.prime_vectors(wl.src_nodes))
    qt = rom.project_io(part, bases, part.prime_vectors(wl.rcv_nodes))
    got_g = online.dense_io(_topo(LR), src, nS, "src")
    got_q = online.dense_io(_topo(LR), rcv, nR, "rcv")
    scale_g = max(np.max(np.abs(x)) for x in gt)
    scale_q = max(np.max(np.abs(x)) for x in qt)
    assert scale_g > 0 and scale_q > 0
    for f in range(len(part.faces)):
        assert np.max(np.abs(got_g[f] - gt[f]), initial=0.0) <= 1e-13 * scale_g, f
        assert np.max(np.abs(got_q[f].T - qt[f]), initial=0.0) <= 1e-13 * scale_q, f
    ref = online.corner_rows(part.corner_groups(), bases)
    assert len(groups) == len(ref) and LR.info()[7] == len(ref)

    def canon(gs):
        out = []
        for g in gs:
            out.append(sorted((int(f), tuple(np.round(np.asarray(r), 12)), round(float(w), 12)) for (f, r, w) in g))
        return sorted(out)

    a, b = canon(groups), canon(ref)
    for ga, gb in zip(a, b):
        assert [m[0] for m in ga] == [m[0] for m in gb]
        for ma, mb in zip(ga, gb):
            assert np.max(np.abs(np.asarray(ma[1]) - np.asarray(mb[1]))) <= 1e-12
            assert abs(ma[2] - mb[2]) <= 1e-12


def _topo(LR):
    cm, cfp, cf, fM, fc, _, _, _ = LR.export()
    return synth.RomTopology(np.asarray(cm, np.int64), [list(cf[cfp[c]:cfp[c + 1]]) for c in range(len(cm))],
                             np.asarray(fM, np.int64), [[int(x) for x in r if x >= 0] for r in fc])


@pytest.mark.parametrize("corners", [False, True])
def test_full_pipeline_traces_match_oracle(P, corners):
    """assemble -> partition -> GPU ROMs -> projected I/O -> FP64 and FP32 stepping vs the oracle
    pipeline on the 2D layered workload (16 cells)."""
    wl = synth.workload_2d_layers(32, 8, m=3, n_modes=4, n_steps=300)
    op, part, io, lam = _setup(wl)
    tau = wl.cfl_fraction * fine.tau_critical(lam)
    s = -rom.omega_max(wl.f_max) ** 2
    R = rom.build_rom(part, wl.m, wl.n_modes, s)
    gp, qp = part.prime_vectors(wl.src_nodes), part.prime_vectors(wl.rcv_nodes)
    gt = rom.project_io(part, R.bases, gp)
    qt = [x.T for x in rom.project_io(part, R.bases, qp)]
    w = synth.ricker(np.arange(wl.n_steps) * tau, wl.f_peak)
    cr = online.corner_rows(part.corner_groups(), R.bases) if corners else None
    ref = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, wl.n_steps, corners=cr)
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    assert abs(L.lambda_max(1e-12) - lam) <= 1e-8 * lam
    LP = P.Partition(L, wl.cell, io)
    LR = P.Rom.build(LP, wl.m, wl.n_modes, s, cg_tol=1e-13)
    LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
    wd = torch.tensor(w, device="cuda")
    for prec, tol in ((P.FP64, COEF_TOL), (P.FP32, 1e-3)):
        sim = P.Sim(LR, prec, tau, corner_correction=corners)
        tr = torch.zeros((wl.n_steps, len(wl.rcv_nodes), 1), device="cuda",
                         dtype=torch.float64 if prec == P.FP64 else torch.float32)
        sim.step(wl.n_steps, wd, tr)
        torch.cuda.synchronize()
        out = tr.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(out - ref) <= tol * np.linalg.norm(ref), prec


def test_build_errors(P):
    wl = synth.workload_2d_layers(16, 4, m=3, n_modes=4, n_steps=10)
    op, part, io, _ = _setup(wl)
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, io)
    with pytest.raises(P.MssError) as e:
        P.Rom.build(LP, 40, 4, -100.0)                 # m K exceeds the cell
    assert e.value.status == 3
    with pytest.raises(P.MssError) as e:
        P.Rom.build(LP, 2, 4, +1.0)                    # shift must be negative
    assert e.value.status == 1
