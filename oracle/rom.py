"""Per-cell reduced-order models and their matrix S-fraction coefficients.

Steps (Algorithm alg1red, stage 1):
 (0) face bases S_f (Section 4.1);
 (1.1) projection subspace V_m and projected pencil A^m, B^m = I, S^m (Eq. npks, Eq. tfprj);
 (1.2) block Lanczos of (A^m, S^m) to block-tridiagonal (T, R) (Appendix C, Eq. NtDtri);
 (1.3) S-fraction coefficients Gamma^k, Gamma-hat^k by the block-diagonal change of
       variables (Eq. GammaTrans);
 (1.4) projected sources/receivers g~_f = S_f^T g|_f, q~_f = S_f^T q|_f (Eq. BEINCr, Eq. solatrec),
 plus the face masses M_f of Eq. bdrytstep.

Readings (where the paper is silent, garbled or inconsistent):
* Face basis: the paper's POD/Gramian basis depends on a method it leaves to a
  missing reference.  Here S_f holds the lowest-wavenumber discrete cosine (DCT-II)
  modes of the face's node grid, Euclidean-orthonormal by construction (S_f^T S_f = I),
  ordered by (a/n1)^2 + (b/n2)^2 then (a, b); these are the Neumann modes of a
  uniform face and do not depend on the medium.  I/O faces keep S_f = I.
  The paper's exact frequency-limited Gramian (Eq. trgr, from the propagative eigenpairs
  of the whole pencil) is ``face_gramians`` / ``gramian_bases``; it checks that reading
  and can replace it through ``build_rom(..., bases=...)``.
* Krylov subspace (Eq. npks): the pencil form with K = (A+sB)^{-1} B and the
  zero-power block B^{-1} P S (Remark Sinsubspace), i.e. the block Krylov space
  span{B^{-1}C, K B^{-1}C, ..., K^{m-1} B^{-1}C}, C = P^Gamma S; note K B^{-1} C =
  (A+sB)^{-1} C, so it holds (A+sB)^{-1}C, ..., and makes Gamma-hat^1 = C^T B^{-1} C
  exact and block-diagonal over faces.  Built block by block (the paper's "block
  Lanczos iteration" remark) with B-inner-product Gram-Schmidt, two passes.
* Shift: s = -omega_max^2.
* GammaTrans: the printed recursion is not symmetric; the symmetric form that
  makes F~ = U^1 of Eq. GammaU1st/GammaUrem exact is used:
      G_1 = beta_1^T,  Gamma^0 = 0,
      Gamma-hat^k = G_k G_k^T,
      Gamma^k = -G_k^{-T} alpha_k G_k^{-1} - Gamma^{k-1},
      G_{k+1} = (G_k^T Gamma^k)^{-1} beta_{k+1}^T,
  with beta from QR (positive diagonal).
* The last coefficient Gamma^m may be positive semidefinite (floating cells: the constant
  mode); it is accepted through a Cholesky factor with floored pivots (``psd_cholesky``).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synth import RomCoefficients, RomTopology


class RomError(RuntimeError):
    """A failed precondition of the construction (deflation, breakdown, non-SPD)."""


# --------------------------------------------------------------------------- face bases
def dct_modes(n: int) -> np.ndarray:
    """Orthonormal DCT-II vectors on n points: column a is c_a cos(pi a (j + 1/2) / n)."""
    j = np.arange(n)[:, None]
    a = np.arange(n)[None, :]
    c = np.where(a == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
    return c * np.cos(np.pi * a * (j + 0.5) / n)


def face_mode_order(shape: Sequence[int]):
    """Mode indices of a face grid, lowest tangential wavenumber first."""
    if len(shape) == 0:
        return [()]
    if len(shape) == 1:
        return [(a,) for a in range(shape[0])]
    n1, n2 = shape
    modes = [(a, b) for a in range(n1) for b in range(n2)]
    modes.sort(key=lambda ab: (ab[0] * ab[0] * n2 * n2 + ab[1] * ab[1] * n1 * n1, ab[0], ab[1]))
    return modes


def face_basis(face, n_modes: int) -> np.ndarray:
    """S_f (K_f x M_f) with S_f^T S_f = I (Section 4.1; see module readings)."""
    K = len(face.nodes)
    if face.kind == "io":
        return np.eye(K)
    shape = face.shape
    M = min(n_modes, K)
    order = face_mode_order(shape)[:M]
    if len(shape) == 0:
        return np.ones((1, 1))
    if len(shape) == 1:
        return dct_modes(shape[0])[:, [o[0] for o in order]]
    p1, p2 = dct_modes(shape[0]), dct_modes(shape[1])
    return np.stack([np.kron(p1[:, a], p2[:, b]) for (a, b) in order], axis=1)


def propagative_modes(A: sp.spmatrix, Bd: np.ndarray, lam_max: float, dense_limit: int = 6000):
    """Eigenpairs of the pencil below the band limit (Eq. specdec): -A z_l = lam_l B z_l with
    lam_l <= lam_max (eigenvalues of -B^{-1}A, reading R16) and z_l^T B z_l = 1.

    Dense symmetric-definite eigensolver up to ``dense_limit`` unknowns; above it, shift-invert
    Lanczos (ARPACK) on B^{-1/2}(-A)B^{-1/2} about zero, with the number of requested pairs doubled
    until one of them lies above the band.  Returns (lam ascending, Z as columns).
    """
    N = A.shape[0]
    if N <= dense_limit:
        lam, Z = sla.eigh(-A.toarray(), np.diag(Bd), subset_by_value=(-np.inf, lam_max))
        return lam, Z
    bh = 1.0 / np.sqrt(Bd)
    Ms = (sp.diags(bh) @ (-A) @ sp.diags(bh)).tocsc()
    k = 64
    while True:
        k = min(k, N - 2)
        lam, W = spla.eigsh(Ms, k=k, sigma=0.0, which="LM")
        order = np.argsort(lam)
        lam, W = lam[order], W[:, order]
        if lam[-1] > lam_max or k >= N - 2:
            keep = lam <= lam_max
            return lam[keep], bh[:, None] * W[:, keep]
        k *= 2


def face_gramians(part, modes) -> List[Optional[np.ndarray]]:
    """Frequency-limited Gramians of Eq. trgr, one per interior face (None for I/O faces).

    G_f = sum over the given propagative modes of v_l v_l^T, v_l = z_l restricted to the face's
    nodes in face order (a hanging copy of a corner-set node takes the node's value);
    ``modes`` = (lam, Z) from ``propagative_modes``.
    """
    Z = modes[1]
    out: List[Optional[np.ndarray]] = []
    for f in part.faces:
        if f.kind == "io":
            out.append(None)
            continue
        V = Z[np.asarray(f.parents, dtype=np.int64), :]
        out.append(V @ V.T)
    return out


def gramian_bases(part, lam_max: float, n_modes: int, modes=None) -> List[np.ndarray]:
    """S_f from the frequency-limited Gramian of Eq. trgr, the paper's own boundary basis.

    S_f = the eigenvectors of G_f (``face_gramians``) of the ``n_modes`` largest eigenvalues,
    S_f^T S_f = I.  G_f has rank at most the number of propagative modes, so columns beyond it
    span part of its null space.  z_l are the B-normalised eigenvectors of the original pencil
    with lam_l <= lam_max (``propagative_modes``, or ``modes`` = (lam, Z) given).  I/O faces
    keep S_f = I.
    """
    if modes is None:
        modes = propagative_modes(part.op.A, part.op.B, lam_max)
    out = []
    for f, G in zip(part.faces, face_gramians(part, modes)):
        if G is None:
            out.append(np.eye(len(f.nodes)))
            continue
        w, Q = np.linalg.eigh(G)
        M = min(n_modes, len(f.nodes))
        out.append(Q[:, ::-1][:, :M].copy())
    return out


# --------------------------------------------------------------------------- Krylov ROM (Eq. npks, tfprj)
def _b_orthonormalize(Y: np.ndarray, Bd: np.ndarray, prev: List[np.ndarray], scale: float) -> np.ndarray:
    """Two-pass block Gram-Schmidt in the B inner product, then B-orthonormal basis of the block."""
    for _ in range(2):
        for Vp in prev:
            Y = Y - Vp @ (Vp.T @ (Bd[:, None] * Y))
    G = Y.T @ (Bd[:, None] * Y)
    G = 0.5 * (G + G.T)
    ev = np.linalg.eigvalsh(G)
    if ev[0] <= 1e-20 * max(scale, ev[-1]):
        raise RomError("Krylov deflation: block is (numerically) linearly dependent (Assumption ass1)")
    R = np.linalg.cholesky(G).T
    return sla.solve_triangular(R, Y.T, trans="T", lower=False).T


def krylov_rom(A: sp.spmatrix, Bd: np.ndarray, C: np.ndarray, m: int, s: float):
    """B-orthonormal basis V of span{B^{-1}C, K B^{-1}C, .., K^{m-1} B^{-1}C}, K=(A+sB)^{-1}B.

    Returns V (N x mK), A^m = V^T A V, S^m = V^T C  (B^m = V^T B V = I).
    """
    N, K = C.shape
    if m * K > N:
        raise RomError("m * K exceeds the cell size")
    lu = spla.splu((A + s * sp.diags(Bd)).tocsc())
    X = C / Bd[:, None]
    blocks: List[np.ndarray] = []
    scale = float(np.max(np.abs(X.T @ (Bd[:, None] * X))))
    for j in range(m):
        if j > 0:
            X = lu.solve(Bd[:, None] * blocks[-1])
            scale = float(np.max(np.abs(X.T @ (Bd[:, None] * X))))
        blocks.append(_b_orthonormalize(X, Bd, blocks, scale))
    V = np.hstack(blocks)
    Am = V.T @ (A @ V)
    Am = 0.5 * (Am + Am.T)
    Sm = V.T @ C
    return V, Am, Sm


# --------------------------------------------------------------------------- block Lanczos (Appendix C)
def _qr_pos(W: np.ndarray):
    """QR with a positive diagonal of R."""
    Q, R = np.linalg.qr(W)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn, sgn[:, None] * R


def block_lanczos(Am: np.ndarray, Sm: np.ndarray, m: int, return_q: bool = False):
    """Block tridiagonal form T = Q^T A^m Q, R = Q^T S^m = [beta_1, 0, ..]^T (Eq. NtDtri).

    Returns (alpha[0..m-1], beta[0..m-1]) with alpha[k] = alpha_{k+1}, beta[k] = beta_{k+1};
    A^m Q_k = Q_{k-1} beta_k^T + Q_k alpha_k + Q_{k+1} beta_{k+1}; full reorthogonalisation.
    With ``return_q`` also the Lanczos blocks Q_1..Q_m.
    """
    K = Sm.shape[1]
    Q1, b1 = _qr_pos(Sm)
    Qs = [Q1]
    alphas, betas = [], [b1]
    nrm = max(np.linalg.norm(Am, 2), 1e-300)
    for k in range(m):
        Qk = Qs[k]
        W = Am @ Qk
        if k > 0:
            W = W - Qs[k - 1] @ betas[k].T
        a = Qk.T @ W
        a = 0.5 * (a + a.T)
        alphas.append(a)
        if k == m - 1:
            break
        W = W - Qk @ a
        for _ in range(2):
            for Qj in Qs:
                W = W - Qj @ (Qj.T @ W)
        Qn, bn = _qr_pos(W)
        if np.min(np.abs(np.diag(bn))) < 1e-13 * nrm:
            raise RomError("block Lanczos breakdown")
        Qs.append(Qn)
        betas.append(bn)
    if return_q:
        return alphas, betas, Qs
    return alphas, betas


# --------------------------------------------------------------------------- S-fraction coefficients (Eq. GammaTrans)
PSD_FLOOR = 1e-13      # pivot floor of the last coefficient, relative to its largest diagonal entry
PSD_NEG_TOL = 1e-8     # most negative pivot still read as rounding of a semidefinite matrix


def psd_cholesky(M: np.ndarray, floor: float = PSD_FLOOR, neg_tol: float = PSD_NEG_TOL):
    """Lower factor L of a positive semidefinite M, L L^T = M + E (reading R24).

    Column-by-column Cholesky in which a pivot d_j <= floor * s (s = max_i M_ii) is raised to
    floor * s; a pivot below -neg_tol * s means M is indefinite beyond rounding (COEF_NOT_SPD).
    E is then diagonal with 0 <= E_jj <= (floor + neg_tol) s, and L L^T is checked to stay that
    close to M (a floored pivot met early could otherwise amplify rounding).  Returns (L, number
    of floored pivots).
    """
    n = M.shape[0]
    s = float(np.max(np.diag(M)))
    if not s > 0:
        raise RomError("last coefficient has no positive diagonal")
    L = np.zeros_like(M)
    floored = 0
    for j in range(n):
        d = M[j, j] - L[j, :j] @ L[j, :j]
        if d <= floor * s:
            if d < -neg_tol * s:
                raise RomError("last coefficient is indefinite (pivot %.3e of scale %.3e)" % (d, s))
            d = floor * s
            floored += 1
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] = (M[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    if floored and np.max(np.abs(L @ L.T - M)) > 10.0 * (floor + neg_tol) * s:
        raise RomError("semidefinite factor of the last coefficient lost accuracy")
    return L, floored


def gamma_trans(alphas: List[np.ndarray], betas: List[np.ndarray], return_g: bool = False):
    """Gamma^k, Gamma-hat^k (k = 1..m) from the block Lanczos coefficients (module readings).

    Gamma^1..Gamma^{m-1} and every Gamma-hat^k must be SPD.  The last coefficient Gamma^m may be
    positive semidefinite (reading R24): a cell with no Dirichlet node has the constant as a null
    vector of A_i, which the Krylov space nearly contains, so Gamma^m has an eigenvalue at the
    level of rounding.  It is factored by ``psd_cholesky``; if a pivot had to be floored, Gamma^m
    is replaced by L L^T (exactly semidefinite, within 1e-8 of the computed matrix)."""
    m = len(alphas)
    G = betas[0].T.copy()
    Gprev = np.zeros_like(G)
    gam, gh, Gs = [], [], []
    for k in range(m):
        Gs.append(G.copy())
        Gh = G @ G.T
        Gi = np.linalg.inv(G)
        Gk = -Gi.T @ alphas[k] @ Gi - Gprev
        Gk = 0.5 * (Gk + Gk.T)
        Gh = 0.5 * (Gh + Gh.T)
        if k + 1 == m:
            L, floored = psd_cholesky(Gk)
            if floored:
                Gk = L @ L.T
                Gk = 0.5 * (Gk + Gk.T)
        for M, nm in (((Gk, "Gamma"),) if k + 1 < m else ()) + ((Gh, "Gamma-hat"),):
            try:
                np.linalg.cholesky(M)
            except np.linalg.LinAlgError:
                raise RomError("%s^%d is not SPD" % (nm, k + 1))
        gam.append(Gk)
        gh.append(Gh)
        if k + 1 < m:
            G = np.linalg.solve(G.T @ Gk, betas[k + 1].T)
        Gprev = Gk
    if return_g:
        return gam, gh, Gs
    return gam, gh


# --------------------------------------------------------------------------- whole-partition build
@dataclasses.dataclass
class CellRom:
    gamma: List[np.ndarray]
    gamma_hat: List[np.ndarray]
    V: Optional[np.ndarray] = None
    Am: Optional[np.ndarray] = None
    Sm: Optional[np.ndarray] = None
    C: Optional[np.ndarray] = None


@dataclasses.dataclass
class Rom:
    """Everything the on-line stage needs, plus the face bases for projections."""

    topology: RomTopology
    coeffs: RomCoefficients
    bases: List[np.ndarray]
    cells: Dict[int, CellRom]


def cell_input_matrix(part, cid: int, bases: List[np.ndarray]) -> np.ndarray:
    """C = P^Gamma S_i: block-diagonal face bases on the cell's boundary rows, zero inside."""
    c = part.build_cell(cid)
    M = sum(bases[f].shape[1] for f in c.faces)
    C = np.zeros((len(c.nodes), M))
    r = o = 0
    for f in c.faces:
        S = bases[f]
        C[r:r + S.shape[0], o:o + S.shape[1]] = S
        r += S.shape[0]
        o += S.shape[1]
    return C


def layer_count_rule(part, cid: int, bases: List[np.ndarray], s: float, omega_max: float,
                     m_range=(3, 6), tol: float = 1e-4, n_freq: int = 8):
    """Per-cell number of S-fraction layers (reading R22 of the 256^3 dipping-layer workload):
    the smallest m in ``m_range`` whose ROM transfer function (Eq. tfprj) is within ``tol`` of the
    largest m's at ``n_freq`` test frequencies.

    Test points: z_j = -w_j^2 + i w_j omega_max / 10, w_j = j omega_max / n_freq (j = 1..n_freq),
    damped frequencies that keep clear of the real-axis poles.  Error: the largest
    ||F~^m(z_j) - F~^mmax(z_j)||_F / ||F~^mmax(z_j)||_F.  The block Krylov spaces are nested (each
    block is B-orthogonalised against the earlier ones), so A^m and S^m of every m are leading
    blocks of the largest m's.  Returns (m, error at m, errors of every m in the range).
    """
    lo, hi = int(m_range[0]), int(m_range[1])
    cell = part.build_cell(cid)
    C = cell_input_matrix(part, cid, bases)
    K = C.shape[1]
    _, Am, Sm = krylov_rom(cell.A, cell.B, C, hi, s)
    zs = [-(w * w) + 1j * w * omega_max / 10.0 for w in omega_max * np.arange(1, n_freq + 1) / n_freq]
    ref = [Sm.T @ np.linalg.solve(Am + z * np.eye(Am.shape[0]), Sm) for z in zs]
    errs = {}
    for m in range(lo, hi + 1):
        n = m * K
        errs[m] = max(float(np.linalg.norm(Sm[:n].T @ np.linalg.solve(Am[:n, :n] + z * np.eye(n), Sm[:n]) - R)
                            / np.linalg.norm(R)) for z, R in zip(zs, ref))
    m = next(k for k in range(lo, hi + 1) if errs[k] <= tol)
    return m, errs[m], errs


def build_cell_rom(part, cid: int, bases: List[np.ndarray], m: int, s: float, keep=False) -> CellRom:
    c = part.build_cell(cid)
    C = cell_input_matrix(part, cid, bases)
    V, Am, Sm = krylov_rom(c.A, c.B, C, m, s)
    al, be = block_lanczos(Am, Sm, m)
    gam, gh = gamma_trans(al, be)
    if keep:
        return CellRom(gam, gh, V, Am, Sm, C)
    return CellRom(gam, gh)


def receiver_lift(cr: CellRom, rows: Sequence[int]) -> np.ndarray:
    """Weights that read fine-grid values inside a cell off its S-fraction state (Remark MFEM:
    the ROM is a Galerkin method, u_i ~ V x with x the projected state).

    In the Lanczos basis x = sum_k Q_k z_k (Eq. NtDtri, mass I), and the S-fraction variables of
    Eq. GammaTrans are U^k = G_k z_k (their mass is (Gamma-hat^k)^{-1} = G_k^{-T} G_k^{-1}), so the
    value at cell-local node n is sum_k w_k^T U^k with w_k = G_k^{-T} Q_k^T V^T e_n; U^1 is the cell's
    face state.  ``cr`` must come from ``build_cell_rom(..., keep=True)``.  Returns (len(rows), m, K).
    """
    m = len(cr.gamma)
    K = cr.Sm.shape[1]
    al, be, Q = block_lanczos(cr.Am, cr.Sm, m, return_q=True)
    _, _, Gs = gamma_trans(al, be, return_g=True)
    out = np.zeros((len(rows), m, K))
    for j, n in enumerate(rows):
        v = cr.V[int(n), :]
        for k in range(m):
            out[j, k] = np.linalg.solve(Gs[k].T, Q[k].T @ v)
    return out


def face_masses(part, bases, cell_roms: Dict[int, CellRom]) -> List[np.ndarray]:
    """M_f = sum_{i ∋ f} (Gamma-hat^1_{i,f})^{-1} (Eq. bdrytstep), the f-block of Gamma-hat^1_i."""
    out = []
    for f in part.faces:
        M = np.zeros((bases[f.id].shape[1],) * 2)
        for c in f.cells:
            o = 0
            for g in part.cells[c].faces:
                if g == f.id:
                    break
                o += bases[g].shape[1]
            mf = bases[f.id].shape[1]
            blk = cell_roms[c].gamma_hat[0][o:o + mf, o:o + mf]
            M += np.linalg.inv(blk)
        out.append(0.5 * (M + M.T))
    return out


def build_rom(part, m, n_modes: int, s: float, keep=False, bases=None) -> Rom:
    """All cells (m scalar or per cell) -> topology, coefficients and face bases.

    ``bases``: per-face S_f to use instead of the DCT modes of ``face_basis`` (for example
    ``gramian_bases``)."""
    if bases is None:
        bases = [face_basis(f, n_modes) for f in part.faces]
    ms = [int(m)] * len(part.cells) if np.isscalar(m) else [int(x) for x in m]
    cells = {c.id: build_cell_rom(part, c.id, bases, ms[c.id], s, keep) for c in part.cells}
    fm = face_masses(part, bases, cells)
    topo = RomTopology(np.array(ms, dtype=np.int64), [list(c.faces) for c in part.cells],
                       np.array([b.shape[1] for b in bases], dtype=np.int64),
                       [list(f.cells) for f in part.faces])
    coeffs = RomCoefficients([cells[i].gamma for i in range(len(part.cells))],
                             [cells[i].gamma_hat for i in range(len(part.cells))], fm)
    return Rom(topo, coeffs, bases, cells)


def project_io(part, bases: List[np.ndarray], vectors: np.ndarray) -> List[np.ndarray]:
    """Per face S_f^T v|_f for prime-space columns v (Eq. BEINCr g~ and Eq. solatrec q~): (M_f, n)."""
    return [bases[f.id].T @ vectors[f.nodes, :] for f in part.faces]


def omega_max(f_max: float) -> float:
    return 2.0 * np.pi * f_max
