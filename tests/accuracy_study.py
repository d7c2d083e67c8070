"""Reproduces the oracle's accuracy study of the method against the fine grid (CPU, FP64).

Not a test (pytest does not collect it): a command-line script over the oracle, for the tables
of the design document's accuracy section.  It runs the 3D layered recipe with 16^3-voxel cells,
builds the oracle ROM for the chosen layers, face modes and face basis, steps the ROM
(Appendix D corners) and the fine-grid leapfrog on the original graph with the same time step,
and prints the receiver relative L2 error.

    python tests/accuracy_study.py --n 64 --band cell --modes 15 28 45 --m 4
    python tests/accuracy_study.py --n 64 --band nyquist --modes 15 --m 6
    python tests/accuracy_study.py --n 64 --band nyquist --modes 15 --m 8 --clamp-last
    python tests/accuracy_study.py --n 32 --band cell --modes 6 10 --basis gramian
    python tests/accuracy_study.py --n 64 --band cell --modes 15 28 45 --basis gramian --eig chebyshev
    python tests/accuracy_study.py --workload 2d --modes 2 3 4 --basis gramian
    python tests/accuracy_study.py --n 64 --band cell --modes 45 --sources 8 --fp32 plain fp64-last chol-last

``--clamp-last`` sets the near-zero eigenvalues of the last coefficient to zero so that builds
with many layers pass (the floating-cell experiment).  ``--fp32`` re-runs the ROM stepping in
float32 with the last flux product either plain, in FP64, or through the Cholesky factor of the
last coefficient.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import fine, online, partition, rom  # noqa: E402


def clamped_gamma_trans(alphas, betas):
    """rom.gamma_trans with the last coefficient projected onto the positive semidefinite cone."""
    m = len(alphas)
    G = betas[0].T.copy()
    Gprev = np.zeros_like(G)
    gam, gh = [], []
    for k in range(m):
        Gh = 0.5 * (G @ G.T + (G @ G.T).T)
        Gi = np.linalg.inv(G)
        Gk = -Gi.T @ alphas[k] @ Gi - Gprev
        Gk = 0.5 * (Gk + Gk.T)
        if k + 1 == m:
            w, Q = np.linalg.eigh(Gk)
            Gk = (Q * np.maximum(w, 0.0)) @ Q.T
        gam.append(Gk)
        gh.append(Gh)
        if k + 1 < m:
            G = np.linalg.solve(G.T @ Gk, betas[k + 1].T)
        Gprev = Gk
    return gam, gh


def chebyshev_modes(A, Bd, lam_cut: float, p: int = 200, deg: int = 150, iters: int = 15, seed: int = 0):
    """Approximate propagative eigenpairs (lam <= lam_cut) of the pencil for grids where shift-invert
    Lanczos is too slow: subspace iteration on B^{-1/2}(-A)B^{-1/2} with a degree-``deg`` Chebyshev
    filter that damps [lam_cut, lam_max], Rayleigh-Ritz after each pass.  Modes near the cut
    converge slowest; the residuals are printed.  Returns (lam, Z) with Z^T B Z = I."""
    bh = 1.0 / np.sqrt(Bd)
    M = (sp.diags(bh) @ (-A) @ sp.diags(bh)).tocsr()
    lmax = 1.05 * fine.lambda_max(A, Bd)
    e, c = (lmax - lam_cut) / 2, (lmax + lam_cut) / 2
    X = np.linalg.qr(np.random.default_rng(seed).standard_normal((M.shape[0], p)))[0]
    for it in range(iters):
        Y0, Y1 = X, (M @ X - c * X) / e
        for _ in range(2, deg + 1):
            Y0, Y1 = Y1, 2 * (M @ Y1 - c * Y1) / e - Y0
        X = np.linalg.qr(Y1)[0]
        H = X.T @ (M @ X)
        w, V = np.linalg.eigh(0.5 * (H + H.T))
        X = X @ V
        res = np.linalg.norm(M @ X - X * w, axis=0)
        keep = w <= lam_cut
        print("chebyshev pass %d: %d modes below the cut, largest residual %.2e (cut %.3g)"
              % (it, int(keep.sum()), res[keep].max() if keep.any() else 0.0, lam_cut), flush=True)
    keep = w <= lam_cut
    return w[keep], bh[:, None] * X[:, keep]


def hybrid_bases(part, modes, n_modes: int, rel_tol: float = 1e-8):
    """Face bases that start with the range of the face's Gramian (eigenvalues above rel_tol of the
    largest, at most n_modes) and continue with the DCT modes orthogonalised against it (the DCT
    order of ``rom.face_basis``), n_modes columns in all.  I/O faces keep S_f = I."""
    out = []
    for f, G in zip(part.faces, rom.face_gramians(part, modes)):
        if G is None:
            out.append(np.eye(len(f.nodes)))
            continue
        w, Q = np.linalg.eigh(G)
        w, Q = w[::-1], Q[:, ::-1]
        M = min(n_modes, len(f.nodes))
        cols = [Q[:, j] for j in range(min(M, int(np.sum(w > rel_tol * w[0]))))]
        for d in rom.face_basis(f, len(f.nodes)).T:
            if len(cols) >= M:
                break
            for _ in range(2):
                for c in cols:
                    d = d - (c @ d) * c
            nd = np.linalg.norm(d)
            if nd > 1e-6:
                cols.append(d / nd)
        out.append(np.stack(cols, axis=1))
    return out


def rom_leapfrog_fp32(R, gt, qt, w, tau, n_steps, corners, last="plain"):
    """The oracle's ROM leapfrog with every array in float32; ``last`` is how the last flux
    product Gamma^m (U^{m+1} - U^m) is formed: "plain", "fp64-last" or "chol-last"."""
    dt = np.float32
    topo, co = R.topology, R.coeffs
    S, Rn = gt[0].shape[1], qt[0].shape[0]
    K = topo.cell_K()
    Minv = [np.linalg.inv(M).astype(dt) for M in co.face_mass]
    G = [[g.astype(dt) for g in co.gamma[i]] for i in range(topo.n_cells)]
    H = [[h.astype(dt) for h in co.gamma_hat[i]] for i in range(topo.n_cells)]
    L = [np.linalg.cholesky(co.gamma[i][-1]).astype(dt) for i in range(topo.n_cells)] if last == "chol-last" else None
    fu = [np.zeros((int(M), S), dt) for M in topo.face_M]
    fo = [x.copy() for x in fu]
    cu = [[np.zeros((int(K[i]), S), dt) for _ in range(int(topo.cell_m[i]) - 1)] for i in range(topo.n_cells)]
    cold = [[x.copy() for x in c] for c in cu]
    g32 = [x.astype(dt) for x in gt]
    q32 = [x.astype(dt) for x in qt]
    cr = [[(f, sr.astype(dt), dt(wt)) for (f, sr, wt) in grp] for grp in corners]
    out = np.zeros((n_steps, Rn, S))
    t2 = dt(tau * tau)
    for n in range(n_steps):
        for f in range(topo.n_faces):
            out[n] += (q32[f] @ fu[f]).astype(np.float64)
        fs = [np.zeros((int(M), S), dt) for M in topo.face_M]
        new_cells = []
        for i in range(topo.n_cells):
            m = int(topo.cell_m[i])
            U = ([np.concatenate([fu[f] for f in topo.cell_faces[i]], axis=0)] + list(cu[i])
                 + [np.zeros((int(K[i]), S), dt)])
            F = []
            for k in range(m):
                D = U[k + 1] - U[k]
                if k == m - 1 and last == "fp64-last":
                    F.append((co.gamma[i][k] @ D.astype(np.float64)).astype(dt))
                elif k == m - 1 and last == "chol-last":
                    F.append(L[i] @ (L[i].T @ D))
                else:
                    F.append(G[i][k] @ D)
            o = 0
            for f in topo.cell_faces[i]:
                Mf = int(topo.face_M[f])
                fs[f] += F[0][o:o + Mf]
                o += Mf
            new_cells.append([dt(2) * cu[i][k - 1] - cold[i][k - 1] + t2 * (H[i][k] @ (F[k] - F[k - 1]))
                              for k in range(1, m)])
        nf = [dt(2) * fu[f] - fo[f] + t2 * (Minv[f] @ (fs[f] - g32[f] * dt(w[n]))) for f in range(topo.n_faces)]
        online.corner_correct(nf, cr)
        fo, fu = fu, nf
        cold, cu = cu, new_cells
    return out


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", choices=["3d", "2d"], default="3d",
                    help="3d: layered 3D recipe with 16^3-voxel cells; 2d: the 64^2 layered 2D workload")
    ap.add_argument("--n", type=int, default=32, help="voxels per edge of the 3D recipe (16^3-voxel cells)")
    ap.add_argument("--band", choices=["cell", "nyquist"], default="cell")
    ap.add_argument("--modes", type=int, nargs="+", default=[15])
    ap.add_argument("--m", type=int, default=4)
    ap.add_argument("--sources", type=int, default=2)
    ap.add_argument("--steps", type=int, default=0, help="time steps (default: 1500 at n=32, 3000 else)")
    ap.add_argument("--basis", choices=["dct", "gramian", "hybrid"], default="dct")
    ap.add_argument("--eig", choices=["lanczos", "chebyshev"], default="lanczos",
                    help="eigensolver of the Gramian basis (chebyshev: approximate, for 64^3 and up)")
    ap.add_argument("--clamp-last", action="store_true")
    ap.add_argument("--fp32", nargs="*", default=[], choices=["plain", "fp64-last", "chol-last"])
    a = ap.parse_args()
    if a.workload == "2d":
        nst = a.steps or 2000
        wl = synth.workload_2d_layers(64, 8, m=a.m, n_modes=a.modes[0], n_steps=nst)
    else:
        nst = a.steps or (1500 if a.n <= 32 else 3000)
        wl = synth.workload_3d_layers(a.n, 16, m=a.m, n_modes=a.modes[0], n_src=a.sources, n_steps=nst,
                                      band=a.band)
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    tau = 0.5 * fine.tau_critical(fine.lambda_max(op.A, op.B))
    lam = rom.omega_max(wl.f_max) ** 2
    w = synth.ricker(np.arange(nst) * tau, wl.f_peak)
    g = np.zeros((op.A.shape[0], len(wl.src_nodes)))
    q = np.zeros((len(wl.rcv_nodes), op.A.shape[0]))
    for j, p in enumerate(wl.src_nodes):
        g[op.node_unknown(tuple(p)), j] = 1.0
    for j, p in enumerate(wl.rcv_nodes):
        q[j, op.node_unknown(tuple(p))] = 1.0
    ref = fine.fine_leapfrog(op.A.tocsr(), op.B, g, q, w, tau, nst)
    if a.clamp_last:
        rom.gamma_trans = clamped_gamma_trans
    modes = None
    if a.basis in ("gramian", "hybrid"):
        modes = (chebyshev_modes(op.A, op.B, lam) if a.eig == "chebyshev"
                 else rom.propagative_modes(op.A, op.B, lam))
    for nm in a.modes:
        t0 = time.perf_counter()
        bases = None
        if a.basis == "gramian":
            bases = rom.gramian_bases(part, lam, nm, modes=modes)
        elif a.basis == "hybrid":
            bases = hybrid_bases(part, modes, nm)
        R = rom.build_rom(part, a.m, nm, -lam, bases=bases)
        gt = rom.project_io(part, R.bases, part.prime_vectors(wl.src_nodes))
        qt = [x.T for x in rom.project_io(part, R.bases, part.prime_vectors(wl.rcv_nodes))]
        corners = online.corner_rows(part.corner_groups(), R.bases)
        tr = online.rom_leapfrog(R.topology, R.coeffs, gt, qt, w, tau, nst, corners=corners)
        line = "%s basis=%s modes=%d m=%d sources=%d steps=%d: rel-L2 ROM FP64 vs fine %.4e" % (
            wl.name + ("" if a.workload == "2d" else " band=" + a.band), a.basis, nm, a.m, len(wl.src_nodes), nst,
            rel(tr, ref))
        for v in a.fp32:
            t32 = rom_leapfrog_fp32(R, gt, qt, w, tau, nst, corners, v)
            line += "; FP32 %s: vs ROM FP64 %.3e, vs fine %.3e" % (v, rel(t32, tr), rel(t32, ref))
        print(line + " (%.0f s)" % (time.perf_counter() - t0), flush=True)


if __name__ == "__main__":
    main()
