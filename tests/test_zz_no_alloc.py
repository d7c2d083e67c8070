"""The allocation-free step (mss_step_noalloc) against the ordinary one (mss_step).

Some callers cannot let a library allocate device memory -- a solver embedded in a host
application that hands out every device buffer from its own pool and budget, or a latency-
critical loop where cudaMalloc/cudaFree would synchronise the device.  For them the library
offers one step entry point that only launches kernels: the caller lays out every input and
output (here with torch, following the layout documented in include/mss.h) and the flux
exchange uses the library's fixed scratch array.  These tests lay the buffers out themselves,
run two calls in a row, and check the traces against mss_step on the same coefficients: in
FP64 within the tolerance of the other FP64 on-line tests (1e-10 relative L2), and in FP32
(16 sources, so the 16-source tile and its four-wide vector loads run) within 1e-6 of the
FP32 sim.  They sit in a file of their own, collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    import paper_1604_06750_gb300 as pkg
    from paper_1604_06750_gb300 import build
    build.build()
    pkg.lib()
    return pkg


def _layout(topo, co, src, rcv, n_src, n_rcv, dev, fdt=None):
    """Device buffers in the mss_step_buffers layout (values of dtype ``fdt``, FP64 by default)."""
    fdt = torch.float64 if fdt is None else fdt
    K = topo.cell_K()
    fM = [int(x) for x in topo.face_M]
    face_row = np.concatenate([[0], np.cumsum(fM)]).astype(np.int64)
    coef, cell_coef, cell_ghat, cell_state, cell_row = [], [], [], [], []
    row_face_row, row_side = [], []
    o = srow = 0
    for c in range(topo.n_cells):
        m, k = int(topo.cell_m[c]), int(K[c])
        cell_coef.append(o)
        for g in co.gamma[c]:
            coef.append(np.asarray(g).ravel())
            o += k * k
        cell_ghat.append(o)
        for h in co.gamma_hat[c][1:]:
            coef.append(np.asarray(h).ravel())
            o += k * k
        cell_state.append(srow)
        srow += (m - 1) * k
        cell_row.append(len(row_face_row))
        for f in topo.cell_faces[c]:
            side = 0 if topo.face_cells[f][0] == c else 1
            for r in range(fM[f]):
                row_face_row.append(face_row[f] + r)
                row_side.append(side)
    minv, face_minv = [], []
    o = 0
    for f in range(topo.n_faces):
        face_minv.append(o)
        minv.append(np.linalg.inv(co.face_mass[f]).ravel())
        o += fM[f] * fM[f]
    fsrc_ptr, fsrc_index, fsrc_val, sval = [0], [], [], []
    o = 0
    for f in range(topo.n_faces):
        for (ff, j, v) in src:
            if ff == f:
                fsrc_index.append(j)
                fsrc_val.append(o)
                sval.append(np.asarray(v))
                o += len(v)
        fsrc_ptr.append(len(fsrc_index))
    rcv_ptr, rcv_face, rcv_off, rval = [0], [], [], []
    o = 0
    for r in range(n_rcv):
        for (f, j, v) in rcv:
            if j == r:
                rcv_face.append(f)
                rcv_off.append(o)
                rval.append(np.asarray(v))
                o += len(v)
        rcv_ptr.append(len(rcv_face))

    def t(a, dt):
        return torch.tensor(np.asarray(a), dtype=dt, device=dev)

    keep = dict(
        cell_K=t(K, torch.int32), cell_m=t(topo.cell_m, torch.int32), cell_coef=t(cell_coef, torch.int64),
        cell_ghat=t(cell_ghat, torch.int64), cell_state=t(cell_state, torch.int64), cell_row=t(cell_row, torch.int64),
        row_face_row=t(row_face_row, torch.int64), row_side=t(row_side, torch.int8), face_M=t(fM, torch.int32),
        face_two=t([1 if len(cs) == 2 else 0 for cs in topo.face_cells], torch.int32),
        face_row=t(face_row[:-1], torch.int64), face_minv=t(face_minv, torch.int64),
        fsrc_ptr=t(fsrc_ptr, torch.int32), fsrc_index=t(fsrc_index or [0], torch.int32),
        fsrc_val=t(fsrc_val or [0], torch.int64), rcv_ptr=t(rcv_ptr, torch.int32), rcv_face=t(rcv_face or [0], torch.int32),
        rcv_off=t(rcv_off or [0], torch.int64), coef=t(np.concatenate(coef), fdt),
        minv=t(np.concatenate(minv), fdt), src_val=t(np.concatenate(sval), fdt),
        rcv_val=t(np.concatenate(rval), fdt),
        fs0=torch.zeros((int(face_row[-1]), n_src), dtype=fdt, device=dev),
        fs1=torch.zeros((int(face_row[-1]), n_src), dtype=fdt, device=dev),
        cs0=torch.zeros((max(1, srow), n_src), dtype=fdt, device=dev),
        cs1=torch.zeros((max(1, srow), n_src), dtype=fdt, device=dev))
    return keep, int(face_row[-1]), int(max(K)), int(max(topo.cell_m)), int(max(fM))


def _run_pair(P, prec, n_src, tol):
    """Two allocation-free calls in a row against one mss_step run of the same length."""
    dev = torch.device("cuda", 0)
    fdt = torch.float64 if prec == P.FP64 else torch.float32
    topo = synth.box_topology((3, 2, 2), modes=5, m=[2, 3, 4] * 4, io_cells=[(0, 2), (7, 3)], seed=31,
                              ragged_modes=True)
    co = synth.random_coefficients(topo, seed=31)
    n_rcv = 4
    src, rcv = synth.random_io(topo, n_src, n_rcv, seed=31)
    tau, n1, n2 = 0.08, 70, 50
    w = synth.ricker(np.arange(n1 + n2) * tau, 0.6)
    wd = torch.tensor(w, device=dev)
    # reference: the ordinary (allocating) path
    R = P.Rom.import_(topo, co)
    R.set_io(n_src, src, n_rcv, rcv)
    sim = P.Sim(R, prec, tau)
    ref = torch.zeros((n1 + n2, n_rcv, n_src), dtype=fdt, device=dev)
    sim.step(n1 + n2, wd, ref, use_graph=False)
    # allocation-free path, two calls in a row
    keep, face_rows, max_K, max_m, max_M = _layout(topo, co, src, rcv, n_src, n_rcv, dev, fdt)
    b = P.StepBuffers()
    b.precision, b.n_cells, b.n_faces, b.n_src, b.n_rcv = prec, topo.n_cells, topo.n_faces, n_src, n_rcv
    b.max_K, b.max_m, b.max_M, b.cur, b.face_rows, b.tau = max_K, max_m, max_M, 0, face_rows, tau
    for name in ("cell_K", "cell_m", "cell_coef", "cell_ghat", "cell_state", "cell_row", "row_face_row", "row_side",
                 "face_M", "face_two", "face_row", "face_minv", "fsrc_ptr", "fsrc_index", "fsrc_val", "rcv_ptr",
                 "rcv_face", "rcv_off", "coef", "minv", "src_val", "rcv_val"):
        setattr(b, name, keep[name].data_ptr())
    b.face_state[0], b.face_state[1] = keep["fs0"].data_ptr(), keep["fs1"].data_ptr()
    b.cell_state_buf[0], b.cell_state_buf[1] = keep["cs0"].data_ptr(), keep["cs1"].data_ptr()
    out = torch.zeros((n1 + n2, n_rcv, n_src), dtype=fdt, device=dev)
    P.step_noalloc(b, n1, wd, out)
    assert b.cur == n1 % 2
    P.step_noalloc(b, n2, wd[n1:], out[n1:])
    torch.cuda.synchronize()
    a, r = out.double().cpu().numpy(), ref.double().cpu().numpy()
    assert np.linalg.norm(r) > 0
    assert np.linalg.norm(a - r) <= tol * np.linalg.norm(r)
    return b, wd, out


def test_noalloc_step_matches_sim(P):
    b, wd, out = _run_pair(P, P.FP64, 5, 1e-10)
    # sizes beyond the fixed scratch are refused before any launch
    b.face_rows = 1 << 30
    with pytest.raises(P.MssError) as e:
        P.step_noalloc(b, 1, wd, out)
    assert e.value.status == 1 and "scratch" in str(e.value)
    # a face-row count whose byte size would wrap around 64 bits is refused too
    b.face_rows = (1 << 62) + 1
    with pytest.raises(P.MssError) as e:
        P.step_noalloc(b, 1, wd, out)
    assert e.value.status == 1 and "scratch" in str(e.value)


def test_noalloc_step_matches_sim_fp32(P):
    _run_pair(P, P.FP32, 16, 1e-6)
