"""Frequency-domain forms: transfer functions and the coupled ROM of Algorithm alg2red.

* Cell transfer function (NtD map), Eq. tfcur, projected as in Eq. project:
      F~_i(z) = C^T (A_i + z B_i)^{-1} C,   C = P^Gamma S_i.
* ROM transfer function, Eq. tfprj:  F~^m_i(z) = S^mT (A^m + z I)^{-1} S^m.
* S-fraction transfer function, Eqs. GammaU1st, GammaUrem, tfgamma: U^1 of
      Gamma^1 (U^2 - U^1) + z (Gamma-hat^1)^{-1} U^1 = I,
      Gamma^k (U^{k+1} - U^k) - Gamma^{k-1} (U^k - U^{k-1}) + z (Gamma-hat^k)^{-1} U^k = 0,
  U^{m+1} = 0.
* Algorithm alg2red: solve Eqs. firsttstep_conj, GammaUremi with Eq. contred for u~ given g~.
"""
from __future__ import annotations

from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .online import cell_offsets


def cell_tf(A, Bd, C, z: complex) -> np.ndarray:
    M = (A + z * sp.diags(Bd)).tocsc()
    return C.T @ spla.splu(M).solve(C.astype(complex) if np.iscomplexobj(z) else C)


def rom_tf(Am, Sm, z) -> np.ndarray:
    return Sm.T @ np.linalg.solve(Am + z * np.eye(Am.shape[0]), Sm)


def sfraction_tf(gamma: List[np.ndarray], gamma_hat: List[np.ndarray], z) -> np.ndarray:
    """U^1 of the three-point matrix scheme (block tridiagonal solve)."""
    m = len(gamma)
    K = gamma[0].shape[0]
    dt = np.result_type(gamma[0], z)
    L = np.zeros((m * K, m * K), dtype=dt)
    for k in range(m):
        sl = slice(k * K, (k + 1) * K)
        L[sl, sl] = -gamma[k] + z * np.linalg.inv(gamma_hat[k])
        if k > 0:
            L[sl, sl] -= gamma[k - 1]
            L[sl, slice((k - 1) * K, k * K)] = gamma[k - 1]
        if k + 1 < m:
            L[sl, slice((k + 1) * K, (k + 2) * K)] = gamma[k]
    E = np.zeros((m * K, K), dtype=dt)
    E[:K] = np.eye(K)
    return np.linalg.solve(L, E)[:K]


def rom_pencil(topo, coeffs):
    """Global ROM as M x_tt = -K x: x = (all u~_f, then U^2..U^m of every cell).

    Face rows: sum_i P~^T Gamma^1_i (U^2_i - U^1_i) - M_f u~_f,tt (Eq. bdrytstep);
    layer rows: Gamma^k (U^{k+1}-U^k) - Gamma^{k-1} (U^k-U^{k-1}) - (Gamma-hat^k)^{-1} U^k_tt
    (Eq. intrtstep_td).  Returns (K, M, face_offsets) with K = -(stiffness part).
    """
    Mf = [int(M) for M in topo.face_M]
    Kc = topo.cell_K()
    foff = np.concatenate([[0], np.cumsum(Mf)]).astype(int)
    n = int(foff[-1])
    coff = []
    for i in range(topo.n_cells):
        coff.append(n)
        n += (int(topo.cell_m[i]) - 1) * int(Kc[i])
    Kg = np.zeros((n, n))
    Mg = np.zeros((n, n))
    for f in range(topo.n_faces):
        Mg[foff[f]:foff[f + 1], foff[f]:foff[f + 1]] = coeffs.face_mass[f]
    for i in range(topo.n_cells):
        m, K = int(topo.cell_m[i]), int(Kc[i])
        offs = cell_offsets(topo, i)

        def cols(k):
            if k == 0:
                return np.concatenate([np.arange(foff[f], foff[f] + Mf[f]) for f, _ in offs])
            return np.arange(coff[i] + (k - 1) * K, coff[i] + k * K)
        for k in range(m):
            # energy term (U^{k+1} - U^k)^T Gamma^k (U^{k+1} - U^k): D_k = [-I at layer k, +I at k+1]
            G = coeffs.gamma[i][k]
            ck = cols(k)
            Kg[np.ix_(ck, ck)] += G
            if k + 1 < m:
                ck1 = cols(k + 1)
                Kg[np.ix_(ck1, ck1)] += G
                Kg[np.ix_(ck, ck1)] -= G
                Kg[np.ix_(ck1, ck)] -= G
        for k in range(1, m):
            r = cols(k)
            Mg[np.ix_(r, r)] = np.linalg.inv(coeffs.gamma_hat[i][k])
    return Kg, Mg, foff


def coupled_rom_solve(topo, coeffs, gt: List[np.ndarray], z) -> List[np.ndarray]:
    """Algorithm alg2red, step 2: u~_f for all faces given g~_f (M_f x S) at Laplace point z.

    Solves (-K + z M) x = [g~; 0] with the global pencil of rom_pencil (Eqs.
    firsttstep_conj, GammaUremi with conjugation Eq. contred built in).
    """
    Kg, Mg, foff = rom_pencil(topo, coeffs)
    S = gt[0].shape[1]
    rhs = np.zeros((Kg.shape[0], S), dtype=np.result_type(1.0, z))
    for f in range(topo.n_faces):
        rhs[foff[f]:foff[f + 1]] = gt[f]
    x = np.linalg.solve(-Kg + z * Mg, rhs)
    return [x[foff[f]:foff[f + 1]] for f in range(topo.n_faces)]
