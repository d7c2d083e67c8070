"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the reduced-order method.  It only draws
media (stiffness sigma and density rho per voxel), source/receiver positions,
the source waveform, and random symmetric-positive-definite coefficient sets
with a given cell/face topology.  Every generator is a pure function of its
arguments and a seed (numpy PCG64).

Conventions
-----------
* A grid has ``dim`` axes; voxel arrays are indexed in array order
  ``[z][y][x]`` (3D) or ``[y][x]`` (2D), x fastest.  Node ``p`` (a tuple in the
  same array order) sits at the corner of voxels; a grid of ``n`` voxels along
  an axis has ``n + 1`` nodes along it.
* ``bc[a] = (lo, hi)`` with ``'D'`` (Dirichlet: the wall nodes are removed)
  or ``'N'`` (Neumann: the wall nodes are kept) for array axis ``a``.
* The acoustic problem is ``div(sigma grad u) - rho u_tt = g w(t)`` (Section 1),
  with a Ricker waveform ``w``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 1604_06750


# --------------------------------------------------------------------------- grids
@dataclasses.dataclass(frozen=True)
class Grid:
    """A box of voxels of edge ``h``; ``n`` voxels per array axis."""

    n: Tuple[int, ...]
    h: float
    bc: Tuple[Tuple[str, str], ...]

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def node_shape(self) -> Tuple[int, ...]:
        return tuple(k + 1 for k in self.n)


@dataclasses.dataclass
class Workload:
    """One synthetic workload: medium, partition, sources, receivers, time axis."""

    name: str
    grid: Grid
    sigma: np.ndarray
    rho: np.ndarray
    cell: Tuple[int, ...]          # voxels per coarse cell along each array axis
    m: int                         # S-fraction layers per cell
    n_modes: int                   # face modes kept per interior face
    src_nodes: np.ndarray          # (S, dim) int node coordinates
    rcv_nodes: np.ndarray          # (R, dim) int node coordinates
    n_steps: int
    cfl_fraction: float            # tau = cfl_fraction * tau_crit(fine grid)
    f_peak: float                  # Ricker peak frequency
    f_max: float                   # band limit (Ricker spectrum < 1e-4 of peak)


# --------------------------------------------------------------------------- waveform
def ricker(t: np.ndarray, f_peak: float, t0: Optional[float] = None) -> np.ndarray:
    """Ricker wavelet with peak frequency ``f_peak`` delayed by ``t0`` (default 1.5/f_peak)."""
    if t0 is None:
        t0 = 1.5 / f_peak
    a = (math.pi * f_peak * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ricker_band_limit(f_peak: float, rel: float = 1e-4) -> float:
    """Frequency above which the Ricker amplitude spectrum stays below ``rel`` of its peak.

    The amplitude spectrum is proportional to x exp(1 - x) with x = (f/f_peak)^2
    (normalised to 1 at the peak); solved for x > 1 by bisection.
    """
    lo, hi = 1.0, 200.0
    target = math.log(rel)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.log(mid) + 1.0 - mid > target:
            lo = mid
        else:
            hi = mid
    return f_peak * math.sqrt(0.5 * (lo + hi))


# --------------------------------------------------------------------------- random fields
def gaussian_random_field(shape: Sequence[int], corr_len: float, rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field with covariance exp(-r^2 / corr_len^2), unit sample variance.

    White noise filtered in Fourier space by the transform of a Gaussian kernel of
    standard deviation corr_len/2 (voxels), then normalised to zero mean, unit variance.
    """
    xi = rng.standard_normal(tuple(shape))
    spec = np.fft.fftn(xi)
    sd = corr_len / 2.0
    mult = np.ones(tuple(shape))
    for ax, n in enumerate(shape):
        k = np.fft.fftfreq(n)
        f = np.exp(-2.0 * (math.pi * sd * k) ** 2)
        sh = [1] * len(shape)
        sh[ax] = n
        mult = mult * f.reshape(sh)
    g = np.real(np.fft.ifftn(spec * mult))
    g -= g.mean()
    g /= g.std()
    return g


def _layer_index(n_axis: int, n_layers: int) -> np.ndarray:
    """Layer index (0 = top, i.e. the high end of the axis) of each voxel along an axis."""
    j = np.arange(n_axis)
    return np.minimum(n_layers - 1, ((n_axis - 1 - j) * n_layers) // n_axis)


def peak_frequency(sigma: np.ndarray, rho: np.ndarray, h: float) -> float:
    """Ricker peak at one tenth of the grid Nyquist at the slowest voxel: c_min / (20 h)."""
    c_min = float(np.sqrt(np.min(sigma / rho)))
    return c_min / (20.0 * h)


def cell_wavelength_peak(sigma: np.ndarray, rho: np.ndarray, h: float, cell_edge: int,
                         wavelengths: float = 1.0) -> float:
    """Ricker peak whose band limit (``ricker_band_limit``) puts ``wavelengths`` minimum
    wavelengths across a cell.

    The shortest wavelength c_min / f_max, at the slowest voxel, equals the cell edge
    ``cell_edge * h`` divided by ``wavelengths``; 1 is the operating point of the paper's
    experiments (Section 7: coarse cells about one minimum wavelength across).
    """
    c_min = float(np.sqrt(np.min(sigma / rho)))
    return wavelengths * c_min / (cell_edge * h) / ricker_band_limit(1.0)


# --------------------------------------------------------------------------- workloads
def workload_2d_layers(n: int = 64, cell: int = 8, m: int = 4, n_modes: int = 4,
                       n_steps: int = 2000, seed_index: int = 0) -> Workload:
    """2D acoustic, n x n voxels, Dirichlet walls, 3 horizontal layers with +-10% noise.

    Layers top to bottom: sigma (1, 2.5, 4), rho (1, 1.5, 2); every voxel's sigma
    and rho multiplied by independent (1 + U(-0.1, 0.1)).  One point source at the
    grid centre node, receivers at the top interior row in the middle of each
    column of cells.  At n=64, cell=8 this is the 64-cell 2D workload.
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    grid = Grid(n=(n, n), h=1.0 / n, bc=(("D", "D"), ("D", "D")))
    li = _layer_index(n, 3)                       # along y (array axis 0)
    s0 = np.array([1.0, 2.5, 4.0])[li][:, None] * np.ones((n, n))
    r0 = np.array([1.0, 1.5, 2.0])[li][:, None] * np.ones((n, n))
    sigma = s0 * (1.0 + rng.uniform(-0.1, 0.1, (n, n)))
    rho = r0 * (1.0 + rng.uniform(-0.1, 0.1, (n, n)))
    src = np.array([[n // 2, n // 2]])
    nc = n // cell
    rcv = np.array([[n - 1, cell // 2 + cell * j] for j in range(nc)])
    fp = peak_frequency(sigma, rho, grid.h)
    return Workload("2d_layers_%d" % n, grid, sigma, rho, (cell, cell), m, n_modes, src, rcv,
                    n_steps, 0.5, fp, ricker_band_limit(fp))


def workload_3d_layers(n: int = 128, cell: int = 16, m: int = 4, n_modes: int = 15,
                       n_src: int = 16, n_steps: int = 4000, seed_index: int = 1,
                       band: str = "nyquist", cell_wavelengths: float = 1.0) -> Workload:
    """3D acoustic, n^3 voxels, Neumann top, Dirichlet elsewhere, 4 layers, lognormal noise.

    Layers top to bottom: sigma (1, 2, 4, 8), rho (1, 1.5, 2, 2.5); sigma multiplied
    by exp(0.1 g - 0.005) with g a unit-variance Gaussian random field of correlation
    length 4 voxels.  Sources on a surface line, receivers on a surface lattice,
    all placed off the cell skeleton (they ride on per-cell I/O faces).
    At n=128, cell=16 this is the 512-cell, 16-source surface workload.
    ``band``: ``"nyquist"`` puts the Ricker peak at one tenth of the grid Nyquist
    (``peak_frequency``; cells are then about 2.9 minimum wavelengths across at 16^3);
    ``"cell"`` puts ``cell_wavelengths`` minimum wavelengths across a cell
    (``cell_wavelength_peak``; 1 by default).
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    grid = Grid(n=(n, n, n), h=1.0 / n, bc=(("D", "N"), ("D", "D"), ("D", "D")))
    li = _layer_index(n, 4)                       # along z (array axis 0); top = high z
    s0 = np.array([1.0, 2.0, 4.0, 8.0])[li][:, None, None] * np.ones((n, n, n))
    rho = np.array([1.0, 1.5, 2.0, 2.5])[li][:, None, None] * np.ones((n, n, n))
    g = gaussian_random_field((n, n, n), 4.0, rng)
    sigma = s0 * np.exp(0.1 * g - 0.005)
    q = cell // 4                                 # quarter-cell offset: off the skeleton
    xs = [q + 2 * q * j for j in range(n // (2 * q))][:n_src]
    y_src = n // 2 + cell // 2
    src = np.array([[n, y_src, x] for x in xs])
    ys = [cell // 2 + cell * l for l in range(n // cell)]
    xr = [q + 2 * q * j for j in range(n // (2 * q))]
    rcv = np.array([[n, y, x] for y in ys for x in xr])
    if band == "nyquist":
        fp = peak_frequency(sigma, rho, grid.h)
    elif band == "cell":
        fp = cell_wavelength_peak(sigma, rho, grid.h, cell, cell_wavelengths)
    else:
        raise ValueError("band must be 'nyquist' or 'cell'")
    return Workload("3d_layers_%d" % n, grid, sigma, rho, (cell, cell, cell), m, n_modes, src, rcv,
                    n_steps, 0.5, fp, ricker_band_limit(fp))


def medium_family(n: int = 32, cell: int = 8, n_media: int = 16, m: int = 2, n_modes: int = 3,
                  seed_index: int = 11) -> List[Workload]:
    """Media for training and testing a learned surrogate of the off-line stage.

    The 3D layered recipe of ``workload_3d_layers`` (Neumann top, Dirichlet elsewhere, 4 layers,
    Gaussian-random-field log-perturbation of sigma with correlation length 4 voxels), with the
    layer values drawn per medium: sigma = 2^U(0, 3), rho = U(1, 2.5), field amplitude U(0, 0.2),
    and the layer boundaries shifted by up to a quarter cell.  Sources on a surface line and one
    receiver lattice, off the cell skeleton, identical for all media.  f_peak / f_max are those of
    the slowest medium the recipe can draw (c_min = sqrt(1 / 2.5) exp(-0.6)), so one shift serves
    the whole family.
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    grid = Grid(n=(n, n, n), h=1.0 / n, bc=(("D", "N"), ("D", "D"), ("D", "D")))
    q = cell // 4
    xs = [q + 2 * q * j for j in range(n // (2 * q))][:2]
    src = np.array([[n, n // 2 + cell // 2, x] for x in xs])
    rcv = np.array([[n, cell // 2 + cell * l, x] for l in range(n // cell) for x in xs])
    c_min = math.sqrt(1.0 / 2.5) * math.exp(-0.6)
    fp = c_min / (20.0 * grid.h)
    out = []
    for k in range(n_media):
        sig_l = 2.0 ** rng.uniform(0.0, 3.0, 4)
        rho_l = rng.uniform(1.0, 2.5, 4)
        amp = rng.uniform(0.0, 0.2)
        shift = int(rng.integers(-(cell // 4), cell // 4 + 1))
        j = np.clip(np.arange(n) + shift, 0, n - 1)
        li = _layer_index(n, 4)[j]
        g = gaussian_random_field((n, n, n), 4.0, rng)
        sigma = sig_l[li][:, None, None] * np.exp(amp * g)
        rho = rho_l[li][:, None, None] * np.ones((n, n, n))
        out.append(Workload("family_%d_%d" % (n, k), grid, sigma, rho, (cell, cell, cell), m, n_modes, src, rcv,
                            400, 0.5, fp, ricker_band_limit(fp)))
    return out


def workload_3d_dipping(n: int = 256, cell: int = 16, m: int = 4, n_modes: int = 15,
                        n_steps: int = 6000, seed_index: int = 2) -> Workload:
    """3D acoustic, n^3 voxels, Dirichlet walls, lognormal GRF background + 2 dipping interfaces.

    sigma = exp(0.3 g - 0.045) with g a unit-variance GRF of correlation length
    ``cell`` voxels, multiplied by 2 below an interface dipping 10 degrees and by a
    further 3 below one dipping 25 degrees; rho grows linearly with depth from 1
    (top) to 2.5 (bottom).  Sources on a (n/cell)^2 lattice of face centres on the
    skeleton plane one cell below the top, receivers on a line in the same plane.
    """
    rng = np.random.default_rng(SEED_BASE + seed_index)
    grid = Grid(n=(n, n, n), h=1.0 / n, bc=(("D", "D"), ("D", "D"), ("D", "D")))
    g = gaussian_random_field((n, n, n), float(cell), rng)
    sigma = np.exp(0.3 * g - 0.045)
    zc = (np.arange(n) + 0.5)[:, None, None]       # voxel centre, array axis 0 = z
    xc = (np.arange(n) + 0.5)[None, None, :]
    depth = n - zc                                 # measured from the top (high z)
    d1 = 0.35 * n + math.tan(math.radians(10.0)) * (xc - 0.5 * n)
    d2 = 0.70 * n + math.tan(math.radians(25.0)) * (xc - 0.5 * n)
    sigma = sigma * np.where(depth > d1, 2.0, 1.0) * np.where(depth > d2, 3.0, 1.0)
    rho = np.broadcast_to(1.0 + 1.5 * depth / n, (n, n, n)).copy()
    zp = n - cell
    nc = n // cell
    src = np.array([[zp, cell // 2 + cell * j, cell // 2 + cell * i] for j in range(nc) for i in range(nc)])
    yr = n // 2 + cell // 2
    rcv = np.array([[zp, yr, 1 + 2 * i] for i in range(min(128, n // 2))])
    fp = peak_frequency(sigma, rho, grid.h)
    return Workload("3d_dipping_%d" % n, grid, sigma, rho, (cell, cell, cell), m, n_modes, src, rcv,
                    n_steps, 0.5, fp, ricker_band_limit(fp))


def workload_1d(n: int = 16, cell: int = 8, seed_index: int = 7) -> Workload:
    """1D string of n voxels, Dirichlet ends, random sigma, rho in [0.5, 2]."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    grid = Grid(n=(n,), h=1.0 / n, bc=(("D", "D"),))
    sigma = rng.uniform(0.5, 2.0, n)
    rho = rng.uniform(0.5, 2.0, n)
    fp = peak_frequency(sigma, rho, grid.h)
    return Workload("1d_%d" % n, grid, sigma, rho, (cell,), cell, 1, np.array([[cell]]), np.array([[cell]]),
                    100, 0.5, fp, ricker_band_limit(fp))


# --------------------------------------------------------------------------- synthetic ROM coefficient sets
@dataclasses.dataclass
class RomTopology:
    """Cells and faces of a coarse box partition, without any coefficient values.

    ``cell_faces[i]`` lists the faces of cell i in the order their modes appear in
    the cell's boundary vector; ``face_M[f]`` is the number of modes of face f;
    ``face_cells[f]`` its one or two cells (lower cell first).
    """

    cell_m: np.ndarray
    cell_faces: List[List[int]]
    face_M: np.ndarray
    face_cells: List[List[int]]

    @property
    def n_cells(self) -> int:
        return len(self.cell_faces)

    @property
    def n_faces(self) -> int:
        return len(self.face_M)

    def cell_K(self) -> np.ndarray:
        return np.array([int(sum(self.face_M[f] for f in fs)) for fs in self.cell_faces], dtype=np.int64)


def box_topology(n_cells: Sequence[int], modes: int, m: int | Sequence[int] = 4,
                 io_cells: Sequence[Tuple[int, int]] = (), seed: int = 0,
                 ragged_modes: bool = False) -> RomTopology:
    """Face graph of a box of cells (C order), walls without faces.

    ``io_cells`` adds, per (cell, K) pair, a one-sided face with K modes.
    ``ragged_modes`` draws each interior face's mode count in [modes//2, modes].
    ``m`` may be a per-cell sequence.
    """
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    n_cells = tuple(n_cells)
    d = len(n_cells)
    nc = int(np.prod(n_cells))
    strides = [int(np.prod(n_cells[a + 1:])) for a in range(d)]
    faces_M: List[int] = []
    faces_cells: List[List[int]] = []
    cell_faces: List[List[int]] = [[] for _ in range(nc)]
    for a in range(d):
        for idx in np.ndindex(*n_cells):
            if idx[a] + 1 >= n_cells[a]:
                continue
            c0 = sum(i * s for i, s in zip(idx, strides))
            c1 = c0 + strides[a]
            mf = int(rng.integers(max(1, modes // 2), modes + 1)) if ragged_modes else modes
            f = len(faces_M)
            faces_M.append(mf)
            faces_cells.append([c0, c1])
    for c, k in io_cells:
        faces_M.append(int(k))
        faces_cells.append([int(c)])
    for f, cs in enumerate(faces_cells):
        for c in cs:
            cell_faces[c].append(f)
    for fs in cell_faces:
        fs.sort()
    if np.isscalar(m):
        cm = np.full(nc, int(m), dtype=np.int64)
    else:
        cm = np.asarray(m, dtype=np.int64)
    return RomTopology(cm, cell_faces, np.array(faces_M, dtype=np.int64), faces_cells)


def _random_spd(n: int, rng: np.random.Generator, scale: float, spread: float) -> np.ndarray:
    """Random SPD matrix: scale * (Q diag(d) Q^T), eigenvalues d in [1/spread, 1]."""
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = np.exp(rng.uniform(-math.log(spread), 0.0, n))
    return scale * (q * d) @ q.T


@dataclasses.dataclass
class RomCoefficients:
    """S-fraction coefficient blocks of every cell and face matrices, FP64.

    ``gamma[i][k]`` (k = 0..m_i-1) is Gamma^{k+1} of cell i, ``gamma_hat[i][k]``
    (k = 0..m_i-1) is Gamma-hat^{k+1}; ``face_mass[f]`` is the face mass M_f.
    """

    gamma: List[List[np.ndarray]]
    gamma_hat: List[List[np.ndarray]]
    face_mass: List[np.ndarray]


def random_coefficients(topo: RomTopology, seed: int = 0, spread: float = 4.0) -> RomCoefficients:
    """Random SPD Gamma, Gamma-hat (per cell) and face masses with entries of order one.

    Gamma-hat^1 is drawn block-diagonal over the cell's faces; each face mass is
    drawn SPD.  Used to exercise on-line stepping on any topology and size.
    """
    rng = np.random.default_rng(SEED_BASE + 200 + seed)
    K = topo.cell_K()
    gam, gh = [], []
    for i in range(topo.n_cells):
        k = int(K[i])
        gi, hi = [], []
        for layer in range(int(topo.cell_m[i])):
            gi.append(_random_spd(k, rng, 1.0, spread))
            if layer == 0:
                blocks = [_random_spd(int(topo.face_M[f]), rng, 1.0, spread) for f in topo.cell_faces[i]]
                h1 = np.zeros((k, k))
                o = 0
                for b in blocks:
                    h1[o:o + len(b), o:o + len(b)] = b
                    o += len(b)
                hi.append(h1)
            else:
                hi.append(_random_spd(k, rng, 1.0, spread))
        gam.append(gi)
        gh.append(hi)
    fm = [_random_spd(int(mf), rng, 1.0, spread) for mf in topo.face_M]
    return RomCoefficients(gam, gh, fm)


def random_io(topo: RomTopology, n_src: int, n_rcv: int, seed: int = 0, density: float = 0.1):
    """Random projected source/receiver vectors on a random subset of faces.

    Returns (src_entries, rcv_entries): lists of (face, index, values[M_f]).
    """
    rng = np.random.default_rng(SEED_BASE + 300 + seed)
    src, rcv = [], []
    nf = topo.n_faces
    for s in range(n_src):
        fs = rng.choice(nf, size=max(1, int(density * nf)) if nf > 10 else 1, replace=False)
        for f in sorted(fs.tolist()):
            src.append((int(f), s, rng.standard_normal(int(topo.face_M[f]))))
    for r in range(n_rcv):
        fs = rng.choice(nf, size=2 if nf > 2 else 1, replace=False)
        for f in sorted(fs.tolist()):
            rcv.append((int(f), r, rng.standard_normal(int(topo.face_M[f]))))
    return src, rcv


def many_source_case(n_cells: Sequence[int] = (16, 16, 16), modes: int = 15, m_range: Tuple[int, int] = (3, 6),
                     n_src: int = 256, n_rcv: int = 128, seed_index: int = 3):
    """Synthetic coupled ROM of the shape of the 256^3 dipping-layer workload's on-line stage.

    A box of 16^3 cells with walls (so wall cells have 3..5 faces and uneven K_i), ``modes``
    modes per interior face, layer counts m_i drawn uniformly in ``m_range``, random SPD
    coefficients with eigenvalues in [1/2, 1], ``n_src`` sources each projected on ~0.1% of
    the faces and ``n_rcv`` receivers on two faces each.  Returns (topology, coefficients,
    source entries, receiver entries).
    """
    rng = np.random.default_rng(SEED_BASE + 500 + seed_index)
    nc = int(np.prod(n_cells))
    ms = rng.integers(m_range[0], m_range[1] + 1, nc)
    topo = box_topology(n_cells, modes=modes, m=ms, seed=seed_index)
    co = random_coefficients(topo, seed=seed_index, spread=2.0)
    src, rcv = random_io(topo, n_src, n_rcv, seed=seed_index, density=0.001)
    return topo, co, src, rcv


def random_state(topo: RomTopology, n_src: int, seed: int = 0):
    """Random face and interior states (two time levels), for energy and resume tests."""
    rng = np.random.default_rng(SEED_BASE + 400 + seed)
    K = topo.cell_K()
    lv = []
    for _ in range(2):
        faces = [rng.standard_normal((int(mf), n_src)) for mf in topo.face_M]
        cells = [[rng.standard_normal((int(K[i]), n_src)) for _ in range(int(topo.cell_m[i]) - 1)]
                 for i in range(topo.n_cells)]
        lv.append((faces, cells))
    return lv
