"""Surrogate off-line path on the GPU: skeleton ROM, slot packing, screen, exact fallback, training gain.

The learned surrogate replaces the rational-Krylov/Lanczos part of the off-line stage (Alg.
alg1red steps 1.2-1.4) for cells the network can predict; everything it hands to the on-line
stage passes a transfer-function screen at the shift s, and cells that fail are rebuilt
exactly.  The checks here:

* the skeleton's Gamma-hat^1 is the exact S^T B^-1 S of the cell boundary (first Markov
  parameter, Eq. GammaTrans with G_1 = beta_1^T) and equals the oracle's Lanczos-made one;
* the fixed-slot Cholesky packing agrees with a packing written here from the oracle's
  coefficients (mask bit-exact), and unpacking it reproduces the oracle's coefficients;
* the screen equals the oracle's ||U^1(s) - F(s)|| / ||F(s)|| (Eqs. GammaU1st, GammaUrem,
  tfgamma against Eq. tfcur) for exact and perturbed coefficients, and is ~0 for the exact ROM
  (the rational Krylov space holds (A + sB)^-1 C, so the Galerkin ROM interpolates F at s);
* inference with an untrained network falls back on every cell and leaves the exact ROM;
* training on a medium family lowers the screen error of held-out media well below the
  untrained network's and the target-mean predictor's.  It does not bring it to the 1e-3
  screen bar: a 3e-3 relative perturbation of the packed factors already moves the transfer
  function by ~4e-2, so at this network size the fallback rebuilds most cells.
"""
import numpy as np
import pytest

import synth
from oracle import fine, freq, partition, rom

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

COEF_TOL = 1e-7       # library off-line stage vs oracle (CG to 1e-13 against direct solves)
SLOT_MODES = 3


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


@pytest.fixture(scope="module")
def case(P):
    wl = synth.medium_family(16, 8, 2, m=2, n_modes=SLOT_MODES)[1]
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    s = -rom.omega_max(wl.f_max) ** 2
    R = rom.build_rom(part, wl.m, wl.n_modes, s, keep=True)
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, io)
    io_slots = max([len(f.parents) for f in part.faces if f.kind == "io"] + [0])
    return dict(wl=wl, op=op, part=part, s=s, R=R, LP=LP, io_slots=io_slots, nc=len(part.cells))


def _slot_rows(part, cid, bases, io_slots):
    rows = []
    for f in part.cells[cid].faces:
        F = part.faces[f]
        M = bases[f].shape[1]
        if F.kind == "io":
            assert M <= io_slots
            base = 6 * SLOT_MODES
        else:
            base = (2 * F.axis + (1 if F.cells[0] == cid else 0)) * SLOT_MODES
        rows += [base + j for j in range(M)]
    assert rows == sorted(rows)
    return rows


def _pack_oracle(R, part, cells, io_slots, noise=0.0, seed=0):
    """Targets and mask written from the oracle's coefficients (Cholesky factors, log diagonal)."""
    Kp = 6 * SLOT_MODES + io_slots
    tri = Kp * (Kp + 1) // 2
    rng = np.random.default_rng(seed)
    T, Mk = [], []
    for c in cells:
        blocks = list(R.coeffs.gamma[c]) + list(R.coeffs.gamma_hat[c][1:])
        rows = _slot_rows(part, c, R.bases, io_slots)
        t = np.zeros(len(blocks) * tri)
        mk = np.zeros(len(blocks) * tri, np.float32)
        for q, M in enumerate(blocks):
            Lc = np.linalg.cholesky(0.5 * (M + M.T))
            K = Lc.shape[0]
            for a in range(K):
                for b in range(a + 1):
                    o = q * tri + rows[a] * (rows[a] + 1) // 2 + rows[b]
                    t[o] = np.log(Lc[a, a]) if a == b else Lc[a, b]
                    mk[o] = 1.0
        if noise:
            t = t + noise * rng.standard_normal(t.size) * mk * (np.abs(t) + 0.1 * np.max(np.abs(t)))
        T.append(t)
        Mk.append(mk)
    return np.array(T), np.array(Mk)


def _unpack_oracle(t, R, part, c, io_slots, m):
    """Coefficients L L^T from one packed vector (the inverse of _pack_oracle)."""
    Kp = 6 * SLOT_MODES + io_slots
    tri = Kp * (Kp + 1) // 2
    rows = _slot_rows(part, c, R.bases, io_slots)
    K = len(rows)
    out = []
    for q in range(2 * m - 1):
        Lc = np.zeros((K, K))
        for a in range(K):
            for b in range(a + 1):
                v = t[q * tri + rows[a] * (rows[a] + 1) // 2 + rows[b]]
                Lc[a, b] = np.exp(v) if a == b else v
        out.append(Lc @ Lc.T)
    return out[:m], [R.coeffs.gamma_hat[c][0]] + out[m:]


def _blocks(export, c, m):
    cm, cfp, cf, fM, fc, g, gh, fm = export
    K = int(sum(fM[cf[cfp[c]:cfp[c + 1]]]))
    o = sum(int(cm[i]) * int(sum(fM[cf[cfp[i]:cfp[i + 1]]])) ** 2 for i in range(c))
    G = [g[o + k * K * K:o + (k + 1) * K * K].reshape(K, K) for k in range(m)]
    H = [gh[o + k * K * K:o + (k + 1) * K * K].reshape(K, K) for k in range(m)]
    return G, H


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_cell_inputs(P, case):
    wl, part, LP = case["wl"], case["part"], case["LP"]
    cells = np.arange(case["nc"])
    x, f = LP.cell_inputs(cells, SLOT_MODES, case["io_slots"])
    c3 = wl.cell[0]
    for c in cells:
        z, y, xx = (int(v) * c3 for v in part.cells[c].coords)
        sl = (slice(z, z + c3), slice(y, y + c3), slice(xx, xx + c3))
        assert np.array_equal(x[c, 0], np.log(wl.sigma[sl]).astype(np.float32))
        assert np.array_equal(x[c, 1], np.log(wl.rho[sl]).astype(np.float32))
        flags = np.zeros(7, np.float32)
        for fid in part.cells[c].faces:
            F = part.faces[fid]
            if F.kind == "io":
                flags[6] = len(F.parents) / case["io_slots"]
            else:
                flags[2 * F.axis + (1 if F.cells[0] == c else 0)] = 1.0
        assert np.array_equal(f[c], flags)


def test_pack_matches_oracle(P, case):
    R, part = case["R"], case["part"]
    cells = np.arange(case["nc"])
    LR = P.Rom.build(case["LP"], 2, SLOT_MODES, case["s"], cg_tol=1e-13)
    t, mk = LR.pack(cells, SLOT_MODES, case["io_slots"], 2)
    to, mko = _pack_oracle(R, part, cells, case["io_slots"])
    assert np.array_equal(mk, mko)
    for c in cells:
        assert np.linalg.norm(t[c] - to[c]) <= 1e-6 * np.linalg.norm(to[c]), c
    assert np.all(t[mk == 0] == 0)


def test_skeleton_and_unpack_match_oracle(P, case):
    R, part, m = case["R"], case["part"], 2
    SK = P.Rom.skeleton(case["LP"], m, SLOT_MODES, case["s"], cg_tol=1e-13)
    ex = SK.export()
    for c in range(case["nc"]):
        G, H = _blocks(ex, c, m)
        assert _rel(H[0], R.coeffs.gamma_hat[c][0]) <= 1e-10, c
        assert all(np.all(g == 0) for g in G) and np.all(H[1] == 0)
    fM, fm = ex[3], ex[7]
    o = 0
    for f, M in enumerate(fM):
        blk = fm[o:o + M * M].reshape(M, M)
        assert _rel(blk, R.coeffs.face_mass[f]) <= 1e-10, f
        o += M * M
    cells = np.arange(case["nc"])
    to, _ = _pack_oracle(R, part, cells, case["io_slots"])
    SK.unpack(cells, SLOT_MODES, case["io_slots"], to)
    ex = SK.export()
    for c in cells:
        G, H = _blocks(ex, c, m)
        for k in range(m):
            assert _rel(G[k], R.coeffs.gamma[c][k]) <= 1e-12, (c, k)
        assert _rel(H[1], R.coeffs.gamma_hat[c][1]) <= 1e-12, c


def test_screen_matches_oracle(P, case):
    R, part, s, m = case["R"], case["part"], case["s"], 2
    cells = np.arange(case["nc"])
    SK = P.Rom.skeleton(case["LP"], m, SLOT_MODES, s, cg_tol=1e-13)
    to, _ = _pack_oracle(R, part, cells, case["io_slots"])
    SK.unpack(cells, SLOT_MODES, case["io_slots"], to)
    err = SK.screen(cells)
    # interpolation at the shift: the exact ROM's transfer function equals F(s)
    for c in cells:
        cl = part.build_cell(c)
        F = freq.cell_tf(cl.A, cl.B, R.cells[c].C, s)
        U = freq.sfraction_tf(R.coeffs.gamma[c], R.coeffs.gamma_hat[c], s)
        assert np.linalg.norm(U - F) <= 1e-9 * np.linalg.norm(F), c
    assert np.all(err <= 1e-8), err
    tp, _ = _pack_oracle(R, part, cells, case["io_slots"], noise=3e-3, seed=5)
    SK.unpack(cells, SLOT_MODES, case["io_slots"], tp)
    err = SK.screen(cells)
    for c in cells:
        cl = part.build_cell(c)
        F = freq.cell_tf(cl.A, cl.B, R.cells[c].C, s)
        gam, gh = _unpack_oracle(tp[c], R, part, c, case["io_slots"], m)
        U = freq.sfraction_tf(gam, gh, s)
        ref = np.linalg.norm(U - F) / np.linalg.norm(F)
        assert ref > 1e-5
        assert abs(err[c] - ref) <= 1e-6 * ref, (c, err[c], ref)


def test_rebuild_cells_matches_oracle(P, case):
    R, m = case["R"], 2
    SK = P.Rom.skeleton(case["LP"], m, SLOT_MODES, case["s"], cg_tol=1e-13)
    sel = [1, 5]
    SK.rebuild_cells(sel)
    ex = SK.export()
    for c in range(case["nc"]):
        G, H = _blocks(ex, c, m)
        if c in sel:
            for k in range(m):
                assert _rel(G[k], R.coeffs.gamma[c][k]) <= COEF_TOL, (c, k)
                assert _rel(H[k], R.coeffs.gamma_hat[c][k]) <= COEF_TOL, (c, k)
        else:
            assert np.all(G[0] == 0)


def test_infer_untrained_falls_back_to_exact(P, case):
    R, part, m = case["R"], case["part"], 2
    io_slots = case["io_slots"]
    Kp = 6 * SLOT_MODES + io_slots
    D = (2 * m - 1) * Kp * (Kp + 1) // 2
    c3 = case["wl"].cell[0]
    cells = np.arange(case["nc"])
    sur = P.Surrogate(c3, 7, D, channels=8, hidden=32, seed=3)
    to, mko = _pack_oracle(R, part, cells, io_slots)
    sur.fit_output_transform(to, mko)
    SK = P.Rom.skeleton(case["LP"], m, SLOT_MODES, case["s"], cg_tol=1e-13)
    err, fb = sur.infer(SK, cells, SLOT_MODES, io_slots, tol=1e-3)
    assert np.all(fb == 1) and np.all(err > 1e-3)
    ex = SK.export()
    for c in cells:
        G, H = _blocks(ex, c, m)
        for k in range(m):
            assert _rel(G[k], R.coeffs.gamma[c][k]) <= COEF_TOL, (c, k)
            assert _rel(H[k], R.coeffs.gamma_hat[c][k]) <= COEF_TOL, (c, k)
    # no fallback: the ROM holds exactly the unpacked predictions
    SK2 = P.Rom.skeleton(case["LP"], m, SLOT_MODES, case["s"], cg_tol=1e-13)
    err2, fb2 = sur.infer(SK2, cells, SLOT_MODES, io_slots, tol=1e300)
    assert np.all(fb2 == 0) and np.allclose(err2, err, rtol=1e-12, atol=0)
    x, f = case["LP"].cell_inputs(cells, SLOT_MODES, io_slots)
    xd, fd = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    y = torch.zeros(len(cells), D, device="cuda")
    sur.predict(xd, fd, y)
    torch.cuda.synchronize()
    SK3 = P.Rom.skeleton(case["LP"], m, SLOT_MODES, case["s"], cg_tol=1e-13)
    SK3.unpack(cells, SLOT_MODES, io_slots, y.cpu().numpy().astype(np.float64))
    assert all(np.array_equal(a, b) for a, b in zip(SK2.export(), SK3.export()))


def test_training_lowers_screen_error(P):
    """Train on 12 media of a family, screen 2 held-out media: the trained network's median
    transfer-function error is well below the untrained network's and the target mean's."""
    m, io_slots = 2, 2
    fam = synth.medium_family(32, 8, 14, m=m, n_modes=SLOT_MODES)
    s = -(2 * np.pi * fam[0].f_max) ** 2
    Kp = 6 * SLOT_MODES + io_slots
    D = (2 * m - 1) * Kp * (Kp + 1) // 2
    data = []
    for wl in fam:
        L = P.Operator(wl.grid, wl.sigma, wl.rho)
        io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
        LP = P.Partition(L, wl.cell, io)
        cells = np.arange(int(LP.info()[0]))
        LR = P.Rom.build(LP, m, SLOT_MODES, s, cg_tol=1e-12)
        t, mk = LR.pack(cells, SLOT_MODES, io_slots, m)
        x, f = LP.cell_inputs(cells, SLOT_MODES, io_slots)
        data.append(dict(L=L, LP=LP, cells=cells, t=t, mk=mk, x=x, f=f))
    train, test = data[:12], data[12:]
    T = np.concatenate([d["t"] for d in train])
    MK = np.concatenate([d["mk"] for d in train])
    X = torch.from_numpy(np.concatenate([d["x"] for d in train])).cuda()
    Fe = torch.from_numpy(np.concatenate([d["f"] for d in train])).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    Md = torch.from_numpy(MK).cuda()
    sur = P.Surrogate(8, 7, D, channels=16, hidden=128, seed=1)
    sur.fit_output_transform(T, MK)

    def screen_median(model):
        errs = []
        for d in test:
            SK = P.Rom.skeleton(d["LP"], m, SLOT_MODES, s, cg_tol=1e-12)
            if model is None:
                mean = (T * MK).sum(0) / np.maximum(MK.sum(0), 1)
                SK.unpack(d["cells"], SLOT_MODES, io_slots, np.repeat(mean[None, :], len(d["cells"]), 0))
                errs.append(SK.screen(d["cells"]))
            else:
                e, _ = model.infer(SK, d["cells"], SLOT_MODES, io_slots, tol=1e300)
                errs.append(e)
        return float(np.median(np.concatenate(errs)))

    e_untrained = screen_median(sur)
    e_mean = screen_median(None)
    loss = torch.zeros(1, device="cuda")
    g = torch.Generator().manual_seed(0)
    n = X.shape[0]
    first = last = None
    for it in range(1500):
        idx = torch.randint(0, n, (64,), generator=g).cuda()
        sur.train_step(X[idx].contiguous(), Fe[idx].contiguous(), Td[idx].contiguous(), 2e-3 if it < 1000 else 5e-4,
                       loss=loss, mask=Md[idx].contiguous())
        if it == 0:
            first = float(loss.item())
    last = float(loss.item())
    e_trained = screen_median(sur)
    print("screen median: untrained %.3e mean %.3e trained %.3e; loss %.3e -> %.3e"
          % (e_untrained, e_mean, e_trained, first, last))
    # measured on a GB300: untrained 0.53, target mean 0.51, trained 0.11; loss 0.62 -> 0.024
    assert last < 0.1 * first
    assert e_trained < 0.35 * e_untrained
    assert e_trained < 0.35 * e_mean
