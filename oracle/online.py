"""On-line stage: explicit leapfrog of the coupled S-fraction ROM (Algorithm alg1red, stage 2).

State: face unknowns u~_f (M_f x S; shared by the cells of the face, Eq. contred) and
hidden layers U^k_i, k = 2..m_i (K~_i x S) of every cell; U^1_i is the cell's faces'
u~_f stacked in the cell's face order, U^{m_i+1}_i = 0.  With omega^2 -> -d^2/dt^2:

  fluxes     F^k_i = Gamma^k_i (U^{k+1}_i - U^k_i),                      k = 1..m_i
  interior   d^2/dt^2 U^k_i = Gamma-hat^k_i (F^k_i - F^{k-1}_i),        k = 2..m_i   (Eq. intrtstep_td)
  faces      d^2/dt^2 u~_f = M_f^{-1} (sum_{i ∋ f} F^1_i|_f - g~_f w(t))             (Eq. bdrytstep)
  receivers  r = sum_f q~_f^T u~_f                                                   (Eq. solatrec)

Reading of Eq. bdrytstep: its source term is printed as "+ delta(t) g~" without
the mass inverse and with the sign opposite to Eq. firsttstep_conj_td; the form
above follows from A u - B u_tt = g w(t) and M_f = sum (Gamma-hat^1_{i,f})^{-1}.
Time integration (unspecified, "any standard scheme"): leapfrog with the right
hand side at the current step, zero initial state (Algorithm alg1red, stage 2).
Trace sample n is taken from the state at step n, before it is advanced.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np


def cell_offsets(topo, i: int) -> List[Tuple[int, int]]:
    """(face, offset) of each face block inside cell i's boundary vector."""
    out, o = [], 0
    for f in topo.cell_faces[i]:
        out.append((f, o))
        o += int(topo.face_M[f])
    return out


def dense_io(topo, entries, n_idx: int, kind: str) -> List[np.ndarray]:
    """(face, index, values) entries -> per face g~ (M_f x n) or q~ (n x M_f)."""
    out = [np.zeros((int(M), n_idx)) for M in topo.face_M]
    for f, j, v in entries:
        out[f][:, j] += np.asarray(v, dtype=np.float64)
    if kind == "rcv":
        out = [o.T.copy() for o in out]
    return out


def _fluxes(topo, coeffs, i, faces_u, cells_U, S):
    m = int(topo.cell_m[i])
    K = sum(int(topo.face_M[f]) for f in topo.cell_faces[i])
    U = [np.concatenate([faces_u[f] for f in topo.cell_faces[i]], axis=0)] + list(cells_U[i])
    U.append(np.zeros((K, S)))
    return [coeffs.gamma[i][k] @ (U[k + 1] - U[k]) for k in range(m)]


def corner_correct(faces_u: List[np.ndarray], corners) -> None:
    """Appendix D correction, in place, of the face unknowns of the new time level.

    ``corners``: per corner-set node k, a list of (face f, S_f row s_l of the hanging
    node l = k_f, weight b_l / b_k).  Steps: u^_l = s_l . u~_f; the corner value is the
    mass-weighted mean of the u^_l; every u~_f gains s_l (mean - u^_l).  All
    corrections use the uncorrected values.
    """
    deltas = []
    for grp in corners:
        uh = [s @ faces_u[f] for (f, s, _) in grp]
        mean = sum(wt * x for (_, _, wt), x in zip(grp, uh))
        for (f, s, _), x in zip(grp, uh):
            deltas.append((f, np.outer(s, mean - x)))
    for f, d in deltas:
        faces_u[f] += d


def corner_rows(corner_groups, bases):
    """Attach the S_f rows to the (face, row, weight) groups of a partition."""
    return [[(f, bases[f][r, :].copy(), wt) for (f, r, wt) in grp] for grp in corner_groups]


def rom_leapfrog(topo, coeffs, gt: List[np.ndarray], qt: List[np.ndarray], w: np.ndarray, tau: float,
                 n_steps: int, state: Optional[tuple] = None, return_state: bool = False, corners=None,
                 lifted=None):
    """Leapfrog of the coupled ROM.  gt[f]: (M_f, S); qt[f]: (R, M_f); w: waveform samples.

    ``state`` = ((faces_now, cells_now), (faces_old, cells_old)) or None for zero.
    ``corners``: optional Appendix D correction data (see corner_correct), applied to
    every new face level.
    ``lifted``: optional receivers inside cells, a list of (cell i, weights (m_i, K_i)) read as
    sum_k w_k^T U^k_i (``rom.receiver_lift``); their traces follow the R face receivers.
    Returns traces (n_steps, R + len(lifted), S) (and the final two levels if asked).
    """
    S = gt[0].shape[1] if len(gt) else 1
    R = qt[0].shape[0] if len(qt) else 0
    Minv = [np.linalg.inv(M) for M in coeffs.face_mass]
    K = topo.cell_K()
    if state is None:
        fu = [np.zeros((int(M), S)) for M in topo.face_M]
        fo = [np.zeros((int(M), S)) for M in topo.face_M]
        cu = [[np.zeros((int(K[i]), S)) for _ in range(int(topo.cell_m[i]) - 1)] for i in range(topo.n_cells)]
        co = [[np.zeros((int(K[i]), S)) for _ in range(int(topo.cell_m[i]) - 1)] for i in range(topo.n_cells)]
    else:
        (fu, cu), (fo, co) = state
        fu = [np.array(x, dtype=np.float64) for x in fu]
        fo = [np.array(x, dtype=np.float64) for x in fo]
        cu = [[np.array(x, dtype=np.float64) for x in c] for c in cu]
        co = [[np.array(x, dtype=np.float64) for x in c] for c in co]
    lifted = lifted or []
    out = np.zeros((n_steps, R + len(lifted), S))
    t2 = tau * tau
    for n in range(n_steps):
        for f in range(topo.n_faces):
            out[n, :R] += qt[f] @ fu[f]
        for j, (i, wts) in enumerate(lifted):
            U = [np.concatenate([fu[f] for f in topo.cell_faces[i]], axis=0)] + list(cu[i])
            out[n, R + j] = sum(wts[k] @ U[k] for k in range(len(U)))
        flux_sum = [np.zeros((int(M), S)) for M in topo.face_M]
        new_cells = []
        for i in range(topo.n_cells):
            F = _fluxes(topo, coeffs, i, fu, cu, S)
            for f, o in cell_offsets(topo, i):
                flux_sum[f] += F[0][o:o + int(topo.face_M[f])]
            m = int(topo.cell_m[i])
            nc = []
            for k in range(1, m):                      # layer k+1 in the paper's numbering
                acc = coeffs.gamma_hat[i][k] @ (F[k] - F[k - 1])
                nc.append(2.0 * cu[i][k - 1] - co[i][k - 1] + t2 * acc)
            new_cells.append(nc)
        new_faces = []
        for f in range(topo.n_faces):
            a = Minv[f] @ (flux_sum[f] - gt[f] * w[n])
            new_faces.append(2.0 * fu[f] - fo[f] + t2 * a)
        if corners:
            corner_correct(new_faces, corners)
        fo, fu = fu, new_faces
        co, cu = cu, new_cells
    if return_state:
        return out, ((fu, cu), (fo, co))
    return out


def rom_energy(topo, coeffs, new, old, tau: float) -> float:
    """Conserved leapfrog energy of the source-free ROM:
    E = 1/2 |(x^{n+1}-x^n)/tau|_M^2 + 1/2 sum_i sum_k (D_k x^{n+1})^T Gamma^k_i (D_k x^n),
    M = blockdiag(M_f, (Gamma-hat^k_i)^{-1}), D_k x = U^{k+1}_i - U^k_i.
    """
    (fn, cn), (fo, co) = new, old
    S = fn[0].shape[1]
    e = 0.0
    for f in range(topo.n_faces):
        d = (fn[f] - fo[f]) / tau
        e += 0.5 * float(np.sum(d * (coeffs.face_mass[f] @ d)))
    for i in range(topo.n_cells):
        m = int(topo.cell_m[i])
        for k in range(1, m):
            d = (cn[i][k - 1] - co[i][k - 1]) / tau
            e += 0.5 * float(np.sum(d * np.linalg.solve(coeffs.gamma_hat[i][k], d)))
        K = sum(int(topo.face_M[f]) for f in topo.cell_faces[i])
        Un = [np.concatenate([fn[f] for f in topo.cell_faces[i]], axis=0)] + list(cn[i]) + [np.zeros((K, S))]
        Uo = [np.concatenate([fo[f] for f in topo.cell_faces[i]], axis=0)] + list(co[i]) + [np.zeros((K, S))]
        for k in range(m):
            e += 0.5 * float(np.sum((Un[k + 1] - Un[k]) * (coeffs.gamma[i][k] @ (Uo[k + 1] - Uo[k]))))
    return e
