"""GB300 implementation of the multiscale S-fraction reduced-order method.

Thin Python binding of the C ABI in ``include/mss.h`` (libmss.so, built in-tree
by ``paper_1604_06750_gb300.build``).  Every call marshals arguments and calls
the native library; all arithmetic of the method runs there (host C++ for the
index-heavy partitioning, CUDA kernels for everything else).  PyTorch is used
only for device buffers and streams.  Importing succeeds without a GPU; a
missing library raises ``MssError`` at first use -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmss.so")

FP64, FP32, FP32_TC, BF16_TC, TF32_TC = 0, 1, 2, 3, 4
SCHED_GRAPH, SCHED_GRAPH_STREAM, SCHED_PERSIST, SCHED_PERSIST_STREAM, SCHED_GRAPH_SPLIT = 0, 1, 2, 3, 4
SCHED_COUNT = 5
SIM_CORNERS, SIM_FACTOR_LAST = 1, 2
DEBUG_GRID_EXTRA_ARRIVALS, DEBUG_TC_EXTRA_TX = 1, 2
DIRICHLET, NEUMANN = 0, 1

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "KRYLOV_DEFLATION", 4: "LANCZOS_BREAKDOWN",
           5: "COEF_NOT_SPD", 6: "CFL", 7: "TIMEOUT", 8: "CUDA", 9: "OOM", 10: "NOT_CONVERGED", 11: "STATE"}


class MssError(RuntimeError):
    """A failed library call: ``status`` is the mss_status code, the message mss_last_error()."""

    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3), ("h", C.c_double), ("bc", (C.c_int32 * 2) * 3)]


class _RomParams(C.Structure):
    _fields_ = [("m", C.c_int32), ("n_modes", C.c_int32), ("shift", C.c_double), ("cg_tol", C.c_double),
                ("cg_maxit", C.c_int32), ("reserved", C.c_int32)]


class _RomDesc(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("n_faces", C.c_int32), ("cell_m", C.c_void_p),
                ("cell_face_ptr", C.c_void_p), ("cell_faces", C.c_void_p), ("face_M", C.c_void_p),
                ("face_cells", C.c_void_p), ("gamma", C.c_void_p), ("gamma_hat", C.c_void_p),
                ("face_mass", C.c_void_p)]


class StepBuffers(C.Structure):
    """mss_step_buffers: caller-owned device buffers of the allocation-free step (see mss.h)."""

    _fields_ = [(n, C.c_int32) for n in ("precision", "n_cells", "n_faces", "n_src", "n_rcv", "max_K", "max_m",
                                          "max_M", "cur", "reserved")] + \
               [("face_rows", C.c_int64), ("tau", C.c_double)] + \
               [(n, C.c_void_p) for n in ("cell_K", "cell_m", "cell_coef", "cell_ghat", "cell_state", "cell_row",
                                          "row_face_row", "row_side", "face_M", "face_two", "face_row", "face_minv",
                                          "fsrc_ptr", "fsrc_index", "fsrc_val", "rcv_ptr", "rcv_face", "rcv_off",
                                          "coef", "minv", "src_val", "rcv_val")] + \
               [("face_state", C.c_void_p * 2), ("cell_state_buf", C.c_void_p * 2)]


_lib = None

# (name, restype, argtypes); void* for every pointer
_P = C.c_void_p
_SIGS = [
    ("mss_status_string", C.c_char_p, [C.c_int32]),
    ("mss_last_error", C.c_char_p, []),
    ("mss_version", C.c_char_p, []),
    ("mss_assemble", C.c_int32, [_P, _P, _P, _P]),
    ("mss_operator_info", C.c_int32, [_P, _P]),
    ("mss_operator_export", C.c_int32, [_P, _P, _P, _P, _P]),
    ("mss_operator_node", C.c_int32, [_P, _P, _P]),
    ("mss_operator_lambda_max", C.c_int32, [_P, C.c_double, _P]),
    ("mss_operator_destroy", None, [_P]),
    ("mss_partition_create", C.c_int32, [_P, _P, _P, _P, C.c_int32, _P, _P]),
    ("mss_partition_info", C.c_int32, [_P, _P]),
    ("mss_partition_faces", C.c_int32, [_P, _P, _P, _P, _P, _P, _P]),
    ("mss_partition_cell", C.c_int32, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    ("mss_partition_set_face_bases", C.c_int32, [_P, C.c_int32, _P, _P]),
    ("mss_partition_destroy", None, [_P]),
    ("mss_assemble_elastic", C.c_int32, [_P, _P, _P, _P]),
    ("mss_build_roms", C.c_int32, [_P, _P, _P, _P, _P]),
    ("mss_layer_rule", C.c_int32, [_P, _P, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32, _P, _P, _P]),
    ("mss_layer_rule_cell", C.c_int32, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32,
                                        _P, _P]),
    ("mss_rom_import", C.c_int32, [_P, _P]),
    ("mss_rom_info", C.c_int32, [_P, _P]),
    ("mss_rom_export", C.c_int32, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("mss_rom_face_bases", C.c_int32, [_P, _P, _P]),
    ("mss_rom_set_io_nodes", C.c_int32, [_P, _P, C.c_int32, _P, _P, C.c_int32, _P, _P]),
    ("mss_rom_set_io", C.c_int32, [_P, C.c_int32, C.c_int32, _P, _P, _P, C.c_int32, C.c_int32, _P, _P, _P]),
    ("mss_rom_set_corners", C.c_int32, [_P, C.c_int32, _P, _P, _P, _P]),
    ("mss_rom_export_io", C.c_int32, [_P] * 12),
    ("mss_partition_set_lift_nodes", C.c_int32, [_P, C.c_int32, _P]),
    ("mss_rom_destroy", None, [_P]),
    ("mss_sim_create", C.c_int32, [_P, C.c_int32, C.c_double, C.c_int32, _P]),
    ("mss_sim_info", C.c_int32, [_P, _P]),
    ("mss_sim_reset", C.c_int32, [_P, _P]),
    ("mss_step", C.c_int32, [_P, C.c_int64, _P, _P, C.c_int32, _P]),
    ("mss_run_host", C.c_int32, [_P, C.c_int64, _P, _P, _P]),
    ("mss_step_profile", C.c_int32, [_P, C.c_int64, _P, _P, _P, _P]),
    ("mss_sim_save_state", C.c_int32, [_P, _P, _P, _P]),
    ("mss_sim_load_state", C.c_int32, [_P, _P, _P, C.c_int64]),
    ("mss_sim_destroy", None, [_P]),
    ("mss_fine_create", C.c_int32, [_P, C.c_int32, C.c_double, C.c_int32, _P, C.c_int32, _P, _P]),
    ("mss_fine_create_unknowns", C.c_int32, [_P, C.c_int32, C.c_double, C.c_int32, _P, C.c_int32, _P, _P]),
    ("mss_fine_reset", C.c_int32, [_P, _P]),
    ("mss_fine_step", C.c_int32, [_P, C.c_int64, _P, _P, C.c_int32, _P]),
    ("mss_fine_destroy", None, [_P]),
    ("mss_step_noalloc", C.c_int32, [_P, C.c_int64, _P, _P, _P]),
    ("mss_surrogate_create", C.c_int32, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _P]),
    ("mss_surrogate_info", C.c_int32, [_P, _P]),
    ("mss_surrogate_get_params", C.c_int32, [_P, _P]),
    ("mss_surrogate_set_params", C.c_int32, [_P, _P]),
    ("mss_surrogate_forward", C.c_int32, [_P, C.c_int32, _P, _P, _P, _P]),
    ("mss_surrogate_backward", C.c_int32, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    ("mss_surrogate_train_step", C.c_int32, [_P, C.c_int32, _P, _P, _P, _P, C.c_float, _P, _P]),
    ("mss_surrogate_destroy", None, [_P]),
    ("mss_surrogate_cell_inputs", C.c_int32, [_P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P]),
    ("mss_surrogate_pack", C.c_int32, [_P, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P, _P]),
    ("mss_surrogate_unpack", C.c_int32, [_P, _P, C.c_int32, _P, C.c_int32, C.c_int32, _P]),
    ("mss_rom_skeleton", C.c_int32, [_P, _P, _P, _P]),
    ("mss_rom_rebuild_cells", C.c_int32, [_P, _P, C.c_int32, _P, _P]),
    ("mss_surrogate_screen", C.c_int32, [_P, _P, C.c_int32, _P, _P, _P]),
    ("mss_surrogate_set_output_transform", C.c_int32, [_P, _P, _P]),
    ("mss_surrogate_fit_output_transform", C.c_int32, [_P, C.c_int32, _P, _P]),
    ("mss_surrogate_predict", C.c_int32, [_P, C.c_int32, _P, _P, _P, _P]),
    ("mss_sim_set_schedule", C.c_int32, [_P, C.c_int32]),
    ("mss_sim_get_schedule", C.c_int32, [_P, _P, _P, _P]),
    ("mss_sim_set_tile", C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32]),
    ("mss_sim_debug", C.c_int32, [_P, C.c_int32, C.c_int32]),
    ("mss_sim_check_stability", C.c_int32, [_P, C.c_int32, C.c_uint64, C.c_double, _P, _P]),
    ("mss_sim_clear_error", C.c_int32, [_P, _P]),
    ("mss_sim_autotune", C.c_int32, [_P, C.c_int32, _P, _P, _P]),
    ("mss_surrogate_infer", C.c_int32, [_P, _P, _P, C.c_int32, _P, C.c_int32, C.c_int32, C.c_double, _P, _P, _P]),
]

EXPORTED = [s[0] for s in _SIGS]


def lib() -> C.CDLL:
    """Load libmss.so (built by ``build.build()``); raises MssError if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MssError(8, "native library %s is missing: run paper_1604_06750_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise MssError(status, lib().mss_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _arr(x, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _devptr(t) -> int:
    return int(t.data_ptr())


class _Handle:
    _destroy = None

    def __init__(self):
        self._h = C.c_void_p()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and h.value and _lib is not None and self._destroy:
            getattr(_lib, self._destroy)(h)
            self._h = C.c_void_p()


class Operator(_Handle):
    """A and diag(B) of the fine grid (mss_assemble)."""

    _destroy = "mss_operator_destroy"

    def __init__(self, grid, sigma: np.ndarray, rho: np.ndarray):
        super().__init__()
        g = _Grid()
        g.dim = len(grid.n)
        for a in range(g.dim):
            g.n[a] = int(grid.n[a])
            for s in range(2):
                g.bc[a][s] = NEUMANN if grid.bc[a][s] == "N" else DIRICHLET
        g.h = float(grid.h)
        self.grid = grid
        self._sigma = _arr(sigma, np.float64).ravel()
        self._rho = _arr(rho, np.float64).ravel()
        _check(lib().mss_assemble(C.byref(g), _ptr(self._sigma), _ptr(self._rho), C.byref(self._h)))
        info = np.zeros(2, np.int64)
        _check(lib().mss_operator_info(self._h, _ptr(info)))
        self.N, self.nnz = int(info[0]), int(info[1])

    @classmethod
    def elastic(cls, grid, stiffness: np.ndarray, rho: np.ndarray) -> "Operator":
        """mss_assemble_elastic: per-voxel Voigt stiffness (n0, n1, n2, 6, 6) and density."""
        self = cls.__new__(cls)
        _Handle.__init__(self)
        g = _Grid()
        g.dim = len(grid.n)
        for a in range(g.dim):
            g.n[a] = int(grid.n[a])
            for s in range(2):
                g.bc[a][s] = NEUMANN if grid.bc[a][s] == "N" else DIRICHLET
        g.h = float(grid.h)
        self.grid = grid
        self._stiffness = _arr(stiffness, np.float64).ravel()
        self._rho = _arr(rho, np.float64).ravel()
        self._sigma = self._rho        # no scalar coefficient; the partition refuses this operator anyway
        _check(lib().mss_assemble_elastic(C.byref(g), _ptr(self._stiffness), _ptr(self._rho), C.byref(self._h)))
        info = np.zeros(2, np.int64)
        _check(lib().mss_operator_info(self._h, _ptr(info)))
        self.N, self.nnz = int(info[0]), int(info[1])
        return self

    def export(self):
        """(rowptr, col, val, bdiag) as numpy arrays."""
        rp = np.zeros(self.N + 1, np.int64)
        col = np.zeros(self.nnz, np.int64)
        val = np.zeros(self.nnz)
        b = np.zeros(self.N)
        _check(lib().mss_operator_export(self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(b)))
        return rp, col, val, b

    def node(self, p) -> int:
        n = _arr(p, np.int32)
        u = np.zeros(1, np.int64)
        _check(lib().mss_operator_node(self._h, _ptr(n), _ptr(u)))
        return int(u[0])

    def lambda_max(self, tol: float = 1e-8) -> float:
        out = np.zeros(1)
        _check(lib().mss_operator_lambda_max(self._h, C.c_double(tol), _ptr(out)))
        return float(out[0])


class Partition(_Handle):
    """Box partition with corner set removed and I/O faces (mss_partition_create)."""

    _destroy = "mss_partition_destroy"

    def __init__(self, op: Operator, cell: Sequence[int], io_nodes=()):
        super().__init__()
        self.op = op
        c = _arr(list(cell) + [1] * (3 - len(cell)), np.int32)
        self.cell_size = c.copy()
        io = _arr(np.asarray(io_nodes).reshape(-1, len(cell)) if len(io_nodes) else np.zeros((0, len(cell))),
                  np.int32)
        _check(lib().mss_partition_create(op._h, _ptr(op._sigma), _ptr(op._rho), _ptr(c), int(io.shape[0]),
                                          _ptr(io), C.byref(self._h)))
        self._info = None

    def info(self) -> np.ndarray:
        if self._info is None:
            info = np.zeros(8, np.int64)
            _check(lib().mss_partition_info(self._h, _ptr(info)))
            self._info = info
        return self._info

    def faces(self):
        info = self.info()
        F, fn = int(info[1]), int(info[5])
        kind = np.zeros(F, np.int32)
        cells = np.zeros(2 * F, np.int32)
        shape = np.zeros(2 * F, np.int32)
        ptr = np.zeros(F + 1, np.int64)
        nodes = np.zeros(fn, np.int64)
        par = np.zeros(fn, np.int64)
        _check(lib().mss_partition_faces(self._h, _ptr(kind), _ptr(cells), _ptr(shape), _ptr(ptr), _ptr(nodes),
                                         _ptr(par)))
        return kind, cells.reshape(F, 2), shape.reshape(F, 2), ptr, nodes, par

    def set_lift_nodes(self, nodes) -> None:
        """mss_partition_set_lift_nodes: receivers inside cells read through the Galerkin lift."""
        a = _arr(np.zeros((0, 1)) if nodes is None or len(nodes) == 0 else nodes, np.int32)
        _check(lib().mss_partition_set_lift_nodes(self._h, int(a.shape[0]) if a.size else 0, _ptr(a)))

    def set_face_bases(self, bases) -> None:
        """Caller-supplied face bases (mss_partition_set_face_bases): one K_f x M_f array per face,
        or None for a face that keeps the DCT modes; ``bases=None`` clears them."""
        if bases is None:
            _check(lib().mss_partition_set_face_bases(self._h, 0, None, None))
            return
        fM = np.array([0 if b is None else np.asarray(b).shape[1] for b in bases], np.int32)
        flat = [np.ascontiguousarray(b, dtype=np.float64).ravel() for b in bases if b is not None]
        data = np.concatenate(flat) if flat else np.zeros(1)
        _check(lib().mss_partition_set_face_bases(self._h, int(len(bases)), _ptr(fM), _ptr(data)))

    def cell(self, c: int):
        cnt = np.zeros(4, np.int64)
        _check(lib().mss_partition_cell(self._h, int(c), _ptr(cnt), None, None, None, None, None, None))
        n, nnz, nf, K = (int(x) for x in cnt)
        faces = np.zeros(nf, np.int32)
        nodes = np.zeros(n, np.int64)
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(nnz, np.int64)
        val = np.zeros(nnz)
        b = np.zeros(n)
        _check(lib().mss_partition_cell(self._h, int(c), _ptr(cnt), _ptr(faces), _ptr(nodes), _ptr(rp), _ptr(col),
                                        _ptr(val), _ptr(b)))
        return dict(faces=faces, nodes=nodes, K=K, rowptr=rp, col=col, val=val, B=b)


    def cell_inputs(self, cells, slot_modes: int, io_slots: int):
        """Surrogate inputs of the listed cells: (x [n][2][c][c][c] log sigma/log rho, feat [n][7])."""
        c = _arr(cells, np.int32)
        e = int(self.cell_size[0])
        x = np.zeros((len(c), 2, e, e, e), np.float32)
        f = np.zeros((len(c), 7), np.float32)
        _check(lib().mss_surrogate_cell_inputs(self._h, len(c), _ptr(c), int(slot_modes), int(io_slots), _ptr(x),
                                               _ptr(f)))
        return x, f


class Rom(_Handle):
    """Cell ROMs / S-fraction coefficients, projected I/O, corner data (mss_rom)."""

    _destroy = "mss_rom_destroy"

    @classmethod
    def build(cls, part: Partition, m: int, n_modes: int, shift: float, cg_tol: float = 1e-12,
              cg_maxit: int = 5000, cell_m=None, stream=None) -> "Rom":
        self = cls()
        p = _RomParams(m=int(m), n_modes=int(n_modes), shift=float(shift), cg_tol=float(cg_tol),
                       cg_maxit=int(cg_maxit), reserved=0)
        cm = None if cell_m is None else _arr(cell_m, np.int32)
        _check(lib().mss_build_roms(part._h, C.byref(p), None if cm is None else _ptr(cm), _stream(stream),
                                    C.byref(self._h)))
        self.part = part
        return self

    @staticmethod
    def layer_rule(part: Partition, n_modes: int, shift: float, omega_max: float, m_range=(3, 6), tol: float = 1e-4,
                   n_freq: int = 8, cg_tol: float = 1e-12, cg_maxit: int = 5000, stream=None):
        """Per-cell layer counts (mss_layer_rule): returns (cell_m int32[C], err float64[C])."""
        p = _RomParams(m=int(m_range[1]), n_modes=int(n_modes), shift=float(shift), cg_tol=float(cg_tol),
                       cg_maxit=int(cg_maxit), reserved=0)
        n = int(part.info()[0])
        cm = np.zeros(n, np.int32)
        err = np.zeros(n, np.float64)
        _check(lib().mss_layer_rule(part._h, C.byref(p), int(m_range[0]), int(m_range[1]), C.c_double(omega_max),
                                    C.c_double(tol), int(n_freq), _ptr(cm), _ptr(err), _stream(stream)))
        return cm, err

    @staticmethod
    def layer_rule_cell(A, S, K: int, omega_max: float, m_range=(3, 6), tol: float = 1e-4, n_freq: int = 8):
        """mss_layer_rule_cell on a given projection (host only): returns (m, errs[m_hi + 1])."""
        A = _arr(A, np.float64)
        S = _arr(S, np.float64)
        mo = np.zeros(1, np.int32)
        errs = np.zeros(int(m_range[1]) + 1, np.float64)
        _check(lib().mss_layer_rule_cell(_ptr(A), _ptr(S), int(K), int(m_range[0]), int(m_range[1]),
                                         C.c_double(omega_max), C.c_double(tol), int(n_freq), _ptr(mo), _ptr(errs)))
        return int(mo[0]), errs

    @classmethod
    def skeleton(cls, part: Partition, m: int, n_modes: int, shift: float, cg_tol: float = 1e-12,
                 cg_maxit: int = 5000, cell_m=None) -> "Rom":
        """Off-line stage without Krylov/Lanczos: exact Gamma-hat^1, face masses, corner data."""
        self = cls()
        p = _RomParams(m=int(m), n_modes=int(n_modes), shift=float(shift), cg_tol=float(cg_tol),
                       cg_maxit=int(cg_maxit), reserved=0)
        cm = None if cell_m is None else _arr(cell_m, np.int32)
        _check(lib().mss_rom_skeleton(part._h, C.byref(p), None if cm is None else _ptr(cm), C.byref(self._h)))
        self.part = part
        return self

    def rebuild_cells(self, cells, stream=None) -> None:
        """Exact off-line construction of the listed cells (same parameters as the ROM's)."""
        c = _arr(cells, np.int32)
        _check(lib().mss_rom_rebuild_cells(self._h, self.part._h, len(c), _ptr(c) if len(c) else None,
                                           _stream(stream)))

    def screen(self, cells, stream=None) -> np.ndarray:
        """Relative transfer-function error of the listed cells at the ROM's shift."""
        c = _arr(cells, np.int32)
        err = np.zeros(len(c))
        _check(lib().mss_surrogate_screen(self._h, self.part._h, len(c), _ptr(c), _ptr(err), _stream(stream)))
        return err

    def pack(self, cells, slot_modes: int, io_slots: int, m: int):
        """(targets [n][(2m-1) Kp(Kp+1)/2] FP64, mask FP32) in the surrogate's fixed slot layout."""
        c = _arr(cells, np.int32)
        Kp = 6 * slot_modes + io_slots
        D = (2 * m - 1) * Kp * (Kp + 1) // 2
        t = np.zeros((len(c), D))
        mk = np.zeros((len(c), D), np.float32)
        _check(lib().mss_surrogate_pack(self._h, self.part._h, len(c), _ptr(c), int(slot_modes), int(io_slots),
                                        _ptr(t), _ptr(mk)))
        return t, mk

    def unpack(self, cells, slot_modes: int, io_slots: int, packed) -> None:
        """Write packed Gamma^k, Gamma-hat^(k>=2) of the listed cells into this ROM."""
        c = _arr(cells, np.int32)
        v = _arr(packed, np.float64)
        _check(lib().mss_surrogate_unpack(self._h, self.part._h, len(c), _ptr(c), int(slot_modes), int(io_slots),
                                          _ptr(v)))

    @classmethod
    def import_(cls, topology, coeffs) -> "Rom":
        """From a topology (cell_m, cell_faces, face_M, face_cells) and per-cell/face FP64 blocks."""
        self = cls()
        cm = _arr(topology.cell_m, np.int32)
        cfp = _arr(np.concatenate([[0], np.cumsum([len(f) for f in topology.cell_faces])]), np.int32)
        cf = _arr(np.concatenate([np.asarray(f, np.int64) for f in topology.cell_faces]), np.int32)
        fM = _arr(topology.face_M, np.int32)
        fc = np.full((len(topology.face_cells), 2), -1, np.int32)
        for f, cs in enumerate(topology.face_cells):
            fc[f, :len(cs)] = cs
        fc = _arr(fc.ravel(), np.int32)
        g = _arr(np.concatenate([np.asarray(x).ravel() for cg in coeffs.gamma for x in cg]), np.float64)
        gh = _arr(np.concatenate([np.asarray(x).ravel() for cg in coeffs.gamma_hat for x in cg]), np.float64)
        fm = _arr(np.concatenate([np.asarray(x).ravel() for x in coeffs.face_mass]), np.float64)
        d = _RomDesc(n_cells=len(cm), n_faces=len(fM), cell_m=_ptr(cm).value, cell_face_ptr=_ptr(cfp).value,
                     cell_faces=_ptr(cf).value, face_M=_ptr(fM).value, face_cells=_ptr(fc).value,
                     gamma=_ptr(g).value, gamma_hat=_ptr(gh).value, face_mass=_ptr(fm).value)
        _check(lib().mss_rom_import(C.byref(d), C.byref(self._h)))
        return self

    def info(self) -> np.ndarray:
        info = np.zeros(8, np.int64)
        _check(lib().mss_rom_info(self._h, _ptr(info)))
        return info

    def export(self):
        """(cell_m, cell_face_ptr, cell_faces, face_M, face_cells, gamma, gamma_hat, face_mass) flat arrays."""
        info = self.info()
        nc, nf = int(info[0]), int(info[1])
        cm = np.zeros(nc, np.int32)
        cfp = np.zeros(nc + 1, np.int32)
        _check(lib().mss_rom_export(self._h, _ptr(cm), _ptr(cfp), None, None, None, None, None, None))
        cf = np.zeros(int(cfp[-1]), np.int32)
        fM = np.zeros(nf, np.int32)
        fc = np.zeros(2 * nf, np.int32)
        g = np.zeros(int(info[4]))
        gh = np.zeros(int(info[4]))
        fm = np.zeros(int(info[5]))
        _check(lib().mss_rom_export(self._h, _ptr(cm), _ptr(cfp), _ptr(cf), _ptr(fM), _ptr(fc), _ptr(g), _ptr(gh),
                                    _ptr(fm)))
        return cm, cfp, cf, fM, fc.reshape(nf, 2), g, gh, fm

    def face_bases(self) -> np.ndarray:
        n = np.zeros(1, np.int64)
        _check(lib().mss_rom_face_bases(self._h, _ptr(n), None))
        out = np.zeros(int(n[0]))
        _check(lib().mss_rom_face_bases(self._h, _ptr(n), _ptr(out)))
        return out

    def set_io_nodes(self, part: Partition, src_nodes, rcv_nodes, src_w=None, rcv_w=None):
        s = _arr(src_nodes, np.int32)
        r = _arr(rcv_nodes, np.int32)
        sw = None if src_w is None else _arr(src_w, np.float64)
        rw = None if rcv_w is None else _arr(rcv_w, np.float64)
        _check(lib().mss_rom_set_io_nodes(self._h, part._h, int(s.shape[0]), _ptr(s),
                                          None if sw is None else _ptr(sw), int(r.shape[0]), _ptr(r),
                                          None if rw is None else _ptr(rw)))

    def set_io(self, n_src: int, src_entries, n_rcv: int, rcv_entries):
        """Entries: lists of (face, index, values[M_f])."""
        def pack(ent):
            f = _arr([e[0] for e in ent], np.int32)
            i = _arr([e[1] for e in ent], np.int32)
            v = _arr(np.concatenate([np.asarray(e[2], np.float64).ravel() for e in ent]) if ent else np.zeros(0),
                     np.float64)
            return f, i, v
        sf, si, sv = pack(src_entries)
        rf, ri, rv = pack(rcv_entries)
        _check(lib().mss_rom_set_io(self._h, int(n_src), len(src_entries), _ptr(sf), _ptr(si), _ptr(sv), int(n_rcv),
                                    len(rcv_entries), _ptr(rf), _ptr(ri), _ptr(rv)))

    def export_io(self):
        """mss_rom_export_io: (sources, receivers, corner groups) as lists of (face, index, values[M_f])
        entries and of groups of (face, row values[M_f], weight)."""
        n = np.zeros(9, np.int64)
        _check(lib().mss_rom_export_io(self._h, _ptr(n), *([None] * 10)))
        sf, si, sv = np.zeros(n[1], np.int32), np.zeros(n[1], np.int32), np.zeros(n[2])
        rf, ri, rv = np.zeros(n[4], np.int32), np.zeros(n[4], np.int32), np.zeros(n[5])
        gp, mf, mr, mw = np.zeros(n[6] + 1, np.int32), np.zeros(n[7], np.int32), np.zeros(n[8]), np.zeros(n[7])
        _check(lib().mss_rom_export_io(self._h, _ptr(n), _ptr(sf), _ptr(si), _ptr(sv), _ptr(rf), _ptr(ri), _ptr(rv),
                                       _ptr(gp), _ptr(mf), _ptr(mr), _ptr(mw)))
        fM = self.export()[3]

        def entries(face, idx, vals):
            out, o = [], 0
            for f, j in zip(face, idx):
                out.append((int(f), int(j), vals[o:o + fM[f]].copy()))
                o += int(fM[f])
            return out

        groups, o = [], 0
        for g in range(int(n[6])):
            grp = []
            for e in range(int(gp[g]), int(gp[g + 1])):
                f = int(mf[e])
                grp.append((f, mr[o:o + fM[f]].copy(), float(mw[e])))
                o += int(fM[f])
            groups.append(grp)
        return entries(sf, si, sv), entries(rf, ri, rv), groups

    def set_corners(self, groups):
        """groups: list of lists of (face, row values[M_f], weight)."""
        ptr = _arr(np.concatenate([[0], np.cumsum([len(g) for g in groups])]), np.int32)
        face = _arr([m[0] for g in groups for m in g], np.int32)
        rows = _arr(np.concatenate([np.asarray(m[1], np.float64) for g in groups for m in g]) if groups
                    else np.zeros(0), np.float64)
        wt = _arr([m[2] for g in groups for m in g], np.float64)
        _check(lib().mss_rom_set_corners(self._h, len(groups), _ptr(ptr), _ptr(face), _ptr(rows), _ptr(wt)))


class Sim(_Handle):
    """On-line stepping of the coupled ROM (mss_sim)."""

    _destroy = "mss_sim_destroy"

    def __init__(self, rom: Rom, precision: int, tau: float, corner_correction: bool = False,
                 factor_last: bool = False):
        super().__init__()
        flags = (SIM_CORNERS if corner_correction else 0) | (SIM_FACTOR_LAST if factor_last else 0)
        _check(lib().mss_sim_create(rom._h, int(precision), C.c_double(tau), flags, C.byref(self._h)))
        self.precision = precision
        i = self.info()
        self.n_src, self.n_rcv, self.state_size = int(i[0]), int(i[1]), int(i[4])

    def info(self) -> np.ndarray:
        info = np.zeros(8, np.int64)
        _check(lib().mss_sim_info(self._h, _ptr(info)))
        return info

    def reset(self, stream=None):
        _check(lib().mss_sim_reset(self._h, _stream(stream)))

    def step(self, n_steps: int, waveform, traces, use_graph: bool = True, stream=None):
        """waveform, traces: CUDA tensors (float64 / float64 or float32 per precision)."""
        _check(lib().mss_step(self._h, int(n_steps), _devptr(waveform), _devptr(traces), int(bool(use_graph)),
                              _stream(stream)))

    def step_profile(self, n_steps: int, waveform, traces, stream=None) -> np.ndarray:
        """Eager steps with per-kernel CUDA events: mean ms of [cell, face, corner] kernels."""
        ms = np.zeros(3)
        _check(lib().mss_step_profile(self._h, int(n_steps), _devptr(waveform), _devptr(traces), _ptr(ms),
                                      _stream(stream)))
        return ms

    def run_host(self, waveform: np.ndarray, stream=None) -> np.ndarray:
        w = _arr(waveform, np.float64)
        dt = np.float64 if self.precision == FP64 else np.float32
        out = np.zeros((len(w), self.n_rcv, self.n_src), dt)
        _check(lib().mss_run_host(self._h, len(w), _ptr(w), _ptr(out), _stream(stream)))
        return out

    def save_state(self):
        now = np.zeros(self.state_size)
        old = np.zeros(self.state_size)
        st = np.zeros(1, np.int64)
        _check(lib().mss_sim_save_state(self._h, _ptr(now), _ptr(old), _ptr(st)))
        return now, old, int(st[0])

    def load_state(self, now, old, steps: int):
        a, b = _arr(now, np.float64), _arr(old, np.float64)
        _check(lib().mss_sim_load_state(self._h, _ptr(a), _ptr(b), int(steps)))

    def set_schedule(self, sched: int):
        _check(lib().mss_sim_set_schedule(self._h, int(sched)))

    def schedule(self):
        """(current schedule, availability mask [SCHED_COUNT])."""
        cur = np.zeros(1, np.int32)
        av = np.zeros(SCHED_COUNT, np.int32)
        _check(lib().mss_sim_get_schedule(self._h, _ptr(cur), _ptr(av), None))
        return int(cur[0]), av

    def check_stability(self, n_steps: int = 200, seed: int = 0, max_growth: float = 1e3, stream=None) -> float:
        """Growth of the state norm over source-free steps; raises MssError (CFL) above max_growth."""
        g = np.zeros(1)
        _check(lib().mss_sim_check_stability(self._h, int(n_steps), C.c_uint64(seed), C.c_double(max_growth), _ptr(g),
                                             _stream(stream)))
        return float(g[0])

    def debug(self, knob: int, value: int):
        """Failure-path test hooks (make a bounded device wait run out; see mss_sim_debug)."""
        _check(lib().mss_sim_debug(self._h, int(knob), int(value)))

    def clear_error(self, stream=None):
        _check(lib().mss_sim_clear_error(self._h, _stream(stream)))

    def set_tile(self, source_tile: int = 0, tc_sources: int = 0, groups: int = 0):
        _check(lib().mss_sim_set_tile(self._h, int(source_tile), int(tc_sources), int(groups)))

    def tile(self):
        """(CUDA-core source tile, split tensor-core sources per CTA, streamed-kernel groups)."""
        t = np.zeros(3, np.int32)
        cur = np.zeros(1, np.int32)
        _check(lib().mss_sim_get_schedule(self._h, _ptr(cur), None, _ptr(t)))
        return tuple(int(x) for x in t)

    def autotune(self, n_steps: int = 32, stream=None):
        """Time every available schedule, keep the fastest; returns (chosen, ms per step)."""
        ms = np.zeros(SCHED_COUNT)
        ch = np.zeros(1, np.int32)
        _check(lib().mss_sim_autotune(self._h, int(n_steps), _stream(stream), _ptr(ms), _ptr(ch)))
        return int(ch[0]), ms


class Surrogate(_Handle):
    """Learned surrogate network (mss_surrogate): hand-written CUDA forward, backward, Adam."""

    _destroy = "mss_surrogate_destroy"

    def __init__(self, cell: int, n_feat: int, n_out: int, channels: int = 32, hidden: int = 256, seed: int = 0):
        super().__init__()
        _check(lib().mss_surrogate_create(int(cell), int(n_feat), int(n_out), int(channels), int(hidden),
                                          C.c_uint64(seed), C.byref(self._h)))
        info = np.zeros(4, np.int64)
        _check(lib().mss_surrogate_info(self._h, _ptr(info)))
        self.n_params, self.n_in, self.n_feat, self.n_out = (int(v) for v in info)
        self.cell, self.channels, self.hidden = cell, channels, hidden

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        _check(lib().mss_surrogate_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, p):
        a = _arr(p, np.float32)
        _check(lib().mss_surrogate_set_params(self._h, _ptr(a)))

    def forward(self, x, feat, y, stream=None):
        _check(lib().mss_surrogate_forward(self._h, int(x.shape[0]), _devptr(x), None if feat is None else _devptr(feat),
                                           _devptr(y), _stream(stream)))

    def backward(self, x, feat, dy, grad, stream=None):
        _check(lib().mss_surrogate_backward(self._h, int(x.shape[0]), _devptr(x),
                                            None if feat is None else _devptr(feat), _devptr(dy), _devptr(grad),
                                            _stream(stream)))

    def train_step(self, x, feat, target, lr: float, loss=None, mask=None, stream=None):
        _check(lib().mss_surrogate_train_step(self._h, int(x.shape[0]), _devptr(x),
                                              None if feat is None else _devptr(feat), _devptr(target),
                                              None if mask is None else _devptr(mask), C.c_float(lr),
                                              None if loss is None else _devptr(loss), _stream(stream)))

    def set_output_transform(self, mean=None, scale=None):
        if mean is None:
            _check(lib().mss_surrogate_set_output_transform(self._h, None, None))
            return
        m, s = _arr(mean, np.float32), _arr(scale, np.float32)
        _check(lib().mss_surrogate_set_output_transform(self._h, _ptr(m), _ptr(s)))

    def fit_output_transform(self, targets, mask=None):
        t = _arr(targets, np.float64)
        mk = None if mask is None else _arr(mask, np.float32)
        _check(lib().mss_surrogate_fit_output_transform(self._h, int(t.shape[0]), _ptr(t),
                                                        None if mk is None else _ptr(mk)))

    def predict(self, x, feat, y, stream=None):
        _check(lib().mss_surrogate_predict(self._h, int(x.shape[0]), _devptr(x), None if feat is None else _devptr(feat),
                                           _devptr(y), _stream(stream)))

    def infer(self, rom: "Rom", cells, slot_modes: int, io_slots: int, tol: float, stream=None):
        """Predict the listed cells into rom, screen them, rebuild the rejected ones exactly.

        Returns (err, fallback): per-cell transfer-function error before the fallback, and 1 where
        the cell was rebuilt."""
        c = _arr(cells, np.int32)
        err = np.zeros(len(c))
        fb = np.zeros(len(c), np.int32)
        _check(lib().mss_surrogate_infer(self._h, rom._h, rom.part._h, len(c), _ptr(c), int(slot_modes), int(io_slots),
                                         C.c_double(tol), _ptr(err), _ptr(fb), _stream(stream)))
        return err, fb


def step_noalloc(buffers: StepBuffers, n_steps: int, waveform, traces, stream=None):
    """mss_step_noalloc: n_steps with caller-owned buffers; advances ``buffers.cur``."""
    _check(lib().mss_step_noalloc(C.byref(buffers), int(n_steps), _devptr(waveform), _devptr(traces),
                                  _stream(stream)))


class FineSim(_Handle):
    """Fine-grid leapfrog on the GPU (mss_fine)."""

    _destroy = "mss_fine_destroy"

    def __init__(self, op: Operator, precision: int, tau: float, src_nodes, rcv_nodes):
        super().__init__()
        s = _arr(src_nodes, np.int32)
        r = _arr(rcv_nodes, np.int32)
        _check(lib().mss_fine_create(op._h, int(precision), C.c_double(tau), int(s.shape[0]), _ptr(s),
                                     int(r.shape[0]), _ptr(r), C.byref(self._h)))
        self.precision = precision
        self.n_src, self.n_rcv = int(s.shape[0]), int(r.shape[0])

    @classmethod
    def at_unknowns(cls, op: Operator, precision: int, tau: float, src_unknowns, rcv_unknowns) -> "FineSim":
        """mss_fine_create_unknowns: the CSR leapfrog, sources and receivers given as unknowns."""
        self = cls.__new__(cls)
        _Handle.__init__(self)
        s = _arr(src_unknowns, np.int64)
        r = _arr(rcv_unknowns, np.int64)
        _check(lib().mss_fine_create_unknowns(op._h, int(precision), C.c_double(tau), int(s.shape[0]), _ptr(s),
                                              int(r.shape[0]), _ptr(r), C.byref(self._h)))
        self.precision = precision
        self.n_src, self.n_rcv = int(s.shape[0]), int(r.shape[0])
        return self

    def reset(self, stream=None):
        _check(lib().mss_fine_reset(self._h, _stream(stream)))

    def step(self, n_steps: int, waveform, traces, use_graph: bool = True, stream=None):
        _check(lib().mss_fine_step(self._h, int(n_steps), _devptr(waveform), _devptr(traces), int(bool(use_graph)),
                                   _stream(stream)))
