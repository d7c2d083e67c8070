"""ctypes binding of the plain C leapfrog loops in ``oracle/c/leapfrog.c`` (FP64, OpenMP).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  The C loops restate
``online.rom_leapfrog`` (without the Appendix D correction) and ``fine.fine_leapfrog`` step for
step, so that the host cores can be timed on them; ``tests/test_oracle_c.py`` checks them against
the NumPy oracle.  ``build()`` compiles the library with gcc (``-O3 -fopenmp``); it is built by
``__graft_entry__.build()`` and on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "leapfrog.c")
OUT = os.path.join(HERE, "_build", "liboracle_leapfrog.so")
_lib: Optional[C.CDLL] = None


def build(force: bool = False) -> str:
    """Compile the C loops (OpenMP if the compiler has it, else serial).  Returns the path."""
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + ".tmp"
    base = ["gcc", "-O3", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("gcc failed on the oracle's C loops:\n" + r.stderr)
    os.replace(tmp, OUT)
    return OUT


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        try:
            _lib = C.CDLL(build())
        except OSError:                 # a stale library from another machine: rebuild it here
            _lib = C.CDLL(build(force=True))
        P = C.c_void_p
        _lib.oracle_threads.restype = C.c_int
        _lib.oracle_rom_leapfrog.restype = C.c_int
        _lib.oracle_rom_leapfrog.argtypes = [C.c_int] * 4 + [P] * 18 + [C.c_double, C.c_int, P]
        _lib.oracle_fine_leapfrog.restype = C.c_int
        _lib.oracle_fine_leapfrog.argtypes = [C.c_int64, C.c_int, C.c_int] + [P] * 9 + [C.c_double, C.c_int, P]
    return _lib


def threads() -> int:
    return int(lib().oracle_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class RomLeapfrog:
    """The coupled ROM marshalled once into the C layout; ``run`` steps it from a zero state."""

    def __init__(self, topo, coeffs, gt: List[np.ndarray], qt: List[np.ndarray]):
        nc, nf = topo.n_cells, topo.n_faces
        S = gt[0].shape[1] if len(gt) else 1
        R = qt[0].shape[0] if len(qt) else 0
        K = topo.cell_K().astype(np.int32)
        m = np.asarray(topo.cell_m, dtype=np.int32)
        fM = np.asarray(topo.face_M, dtype=np.int32)
        face_row = np.concatenate([[0], np.cumsum(fM)]).astype(np.int64)
        cfp = np.concatenate([[0], np.cumsum([len(x) for x in topo.cell_faces])]).astype(np.int64)
        cf = np.array([f for x in topo.cell_faces for f in x], dtype=np.int32)
        # the cells of each face, ascending, with the face's offset inside each cell's boundary vector
        members = [[] for _ in range(nf)]
        for i in range(nc):
            o = 0
            for f in topo.cell_faces[i]:
                members[f].append((i, o))
                o += int(fM[f])
        fcp = np.concatenate([[0], np.cumsum([len(x) for x in members])]).astype(np.int64)
        fcell = np.array([c for x in members for (c, _) in sorted(x)], dtype=np.int32)
        foff = np.array([o for x in members for (_, o) in sorted(x)], dtype=np.int32)
        coef_off = np.zeros(nc, np.int64)
        gam, gh = [], []
        o = 0
        for i in range(nc):
            coef_off[i] = o
            for k in range(int(m[i])):
                gam.append(np.asarray(coeffs.gamma[i][k], dtype=np.float64).ravel())
                gh.append(np.asarray(coeffs.gamma_hat[i][k], dtype=np.float64).ravel())
                o += int(K[i]) * int(K[i])
        minv_off = np.zeros(nf, np.int64)
        mv = []
        o = 0
        for f in range(nf):
            minv_off[f] = o
            mv.append(np.linalg.inv(coeffs.face_mass[f]).ravel())
            o += int(fM[f]) ** 2
        state_off = np.concatenate([[0], np.cumsum((m - 1).astype(np.int64) * K)])[:nc].astype(np.int64)
        g = np.concatenate([np.asarray(x, dtype=np.float64).reshape(int(fM[f]), S) for f, x in enumerate(gt)], axis=0)
        q = (np.concatenate([np.asarray(x, dtype=np.float64).reshape(R, int(fM[f])) for f, x in enumerate(qt)],
                            axis=1) if R else np.zeros((0, 0)))
        self.sizes = (nc, nf, S, R)
        self.arrays = [np.ascontiguousarray(a) for a in (m, K, cfp, cf, fM, face_row, fcp, fcell, foff,
                                                         np.concatenate(gam), np.concatenate(gh), coef_off,
                                                         np.concatenate(mv), minv_off, state_off, g, q)]

    def run(self, w: np.ndarray, tau: float, n_steps: int) -> np.ndarray:
        nc, nf, S, R = self.sizes
        wv = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        out = np.zeros((n_steps, R, S))
        rc = lib().oracle_rom_leapfrog(nc, nf, S, R, *[_p(a) for a in self.arrays], _p(wv), C.c_double(tau),
                                       int(n_steps), _p(out))
        if rc != 0:
            raise MemoryError("oracle_rom_leapfrog: scratch allocation failed")
        return out


def rom_leapfrog(topo, coeffs, gt: List[np.ndarray], qt: List[np.ndarray], w: np.ndarray, tau: float,
                 n_steps: int) -> np.ndarray:
    """Same arguments and result as ``online.rom_leapfrog`` (zero initial state, no corners)."""
    return RomLeapfrog(topo, coeffs, gt, qt).run(w, tau, n_steps)


def fine_leapfrog(A: sp.spmatrix, B: np.ndarray, g: np.ndarray, q, w: np.ndarray, tau: float,
                  n_steps: int) -> np.ndarray:
    """Same arguments and result as ``fine.fine_leapfrog`` (zero initial state; q dense or sparse)."""
    A = sp.csr_matrix(A)
    Q = sp.csr_matrix(q)
    N, S = g.shape
    R = Q.shape[0]
    ap, ac, av = (np.ascontiguousarray(A.indptr, np.int64), np.ascontiguousarray(A.indices, np.int64),
                  np.ascontiguousarray(A.data, np.float64))
    qp, qc, qv = (np.ascontiguousarray(Q.indptr, np.int64), np.ascontiguousarray(Q.indices, np.int64),
                  np.ascontiguousarray(Q.data, np.float64))
    Bv = np.ascontiguousarray(B, np.float64)
    gv = np.ascontiguousarray(g, np.float64)
    wv = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    out = np.zeros((n_steps, R, S))
    rc = lib().oracle_fine_leapfrog(int(N), int(S), int(R), _p(ap), _p(ac), _p(av), _p(Bv), _p(gv), _p(qp),
                                    _p(qc), _p(qv), _p(wv), C.c_double(tau), int(n_steps), _p(out))
    if rc != 0:
        raise MemoryError("oracle_fine_leapfrog: allocation failed")
    return out
