#!/usr/bin/env python
"""Benchmark of the on-line stage: ROM source·cell-steps per second on one GPU, at the accuracy
the metric asks for (receiver traces within 1e-3 of the fine grid).

Workload: the 3D layered acoustic medium of 128^3 voxels (Neumann top, Dirichlet elsewhere,
4 layers, lognormal perturbations), 512 coarse cells of 16^3 voxels, m = 4 S-fraction layers,
16 surface sources, 128 surface receivers, 4000 leapfrog steps at half the fine-grid CFL limit,
at the operating point of the paper's experiments (Section 7): a band whose minimum wavelength
is one cell edge, and 45 modes per interior face (K up to 270).  One bench step = one whole
on-line simulation of that batch (512 cells x 16 sources x 4000 time steps), state reset at
its start.

Headline: FP32 stepping with the last S-fraction coefficient applied as its Cholesky factor
and the Appendix D corner correction.  Reported beside it: the receiver error against the same
GPU's FP64 fine-grid leapfrog on the original graph (the accuracy target), the FP32 fine grid's
rate at the same tau and steps (the comparison at equal accuracy), FP64 ROM stepping, the
off-line build time, the cell kernel's roofline, and the oracle timed on the host cores on this
ROM's own coefficients.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --profile N [--sched K]   # same workload, N eager time steps, for ncu captures
    python bench.py --band nyquist --modes 15 # the 1/10-Nyquist band at 15 modes (not at 1e-3)
    python bench.py --accuracy                # ROM vs fine grid over face-mode counts
    python bench.py --many-sources            # 4096 cells x 256 sources, every precision
    python bench.py --surrogate               # learned off-line stage vs the exact one

The step schedule is picked by the library's autotuner before the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# The headline workload: the 128^3 layered medium at the operating point of the paper's
# experiments (Section 7: cells about one minimum wavelength across, m = 4, K~ = 180-294), where
# the ROM reaches the 1e-3 receiver level against the fine grid.
WORKLOAD = dict(n=128, cell=16, m=4, n_modes=45, n_src=16, n_steps=4000, band="cell", cellwl=1.0)
# The learned-surrogate mode keeps the 1/10-Nyquist band and 15 modes (its network predicts a
# (2m-1) Kp (Kp+1)/2 vector per cell, which stays small only at few modes).
SURROGATE_WORKLOAD = dict(n=128, cell=16, m=4, n_modes=15, n_src=16, n_steps=4000, band="nyquist", cellwl=1.0)
METRIC = "online ROM source·cell-steps/s vs fine-grid stencil at ≤1e-3 receiver error"
UNIT = "source·cell-steps/s"
ACCURACY_TARGET = 1e-3


def _workload(spec=None, **over):
    p = dict(WORKLOAD if spec is None else spec)
    p.update({k: v for k, v in over.items() if v is not None})
    wl = synth.workload_3d_layers(p["n"], p["cell"], m=p["m"], n_modes=p["n_modes"], n_src=p["n_src"],
                                  n_steps=p["n_steps"], band=p["band"], cell_wavelengths=p["cellwl"])
    wl.band = p["band"]
    wl.cellwl = p["cellwl"]
    return wl


def _config(wl, extra=None):
    nc = int(np.prod([wl.grid.n[a] // wl.cell[a] for a in range(3)]))
    band = {"cell": "%g minimum wavelengths per cell" % wl.cellwl,
            "nyquist": "Ricker peak at 1/10 grid Nyquist"}[wl.band]
    c = {"workload": "3d_layers_%d: %d^3 voxels, %d cells of 16^3, band %s, m=%d, %d modes/face, %d sources, "
                     "%d receivers, %d steps" % (wl.grid.n[0], wl.grid.n[0], nc, band, wl.m, wl.n_modes,
                                                  len(wl.src_nodes), len(wl.rcv_nodes), wl.n_steps),
         "cells": nc, "sources": int(len(wl.src_nodes)), "receivers": int(len(wl.rcv_nodes)),
         "time_steps": int(wl.n_steps), "layers": wl.m, "face_modes": wl.n_modes, "band": wl.band,
         "cell_wavelengths": wl.cellwl if wl.band == "cell" else None}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing
def _oracle_stepper(topo, co, gt, qt):
    """The oracle's ROM leapfrog for host timing, prepared for one topology: the plain C loops
    (OpenMP, all host threads; coefficients marshalled before the clock starts) when gcc could
    build them, else the NumPy restatement.  Returns (run(w, tau, n_steps), label, threads)."""
    try:
        from oracle import c_leapfrog
        lf = c_leapfrog.RomLeapfrog(topo, co, gt, qt)
        return lf.run, "C, OpenMP", c_leapfrog.threads()
    except (OSError, RuntimeError):
        from oracle import online
        return (lambda w, tau, n: online.rom_leapfrog(topo, co, gt, qt, w, tau, n)), "NumPy", os.cpu_count()


def _box_io(wl):
    """(cell, I/O node count) of every cell holding sources or receivers: the distinct nodes inside
    a cell form its one-sided I/O face (the partition's rule), so these are the workload's I/O
    face sizes."""
    nodes = {tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)}
    nc = [wl.grid.n[a] // wl.cell[a] for a in range(3)]
    count = {}
    for p in nodes:
        c = [min(p[a] // wl.cell[a], nc[a] - 1) for a in range(3)]
        lin = (c[0] * nc[1] + c[1]) * nc[2] + c[2]
        count[lin] = count.get(lin, 0) + 1
    return sorted(count.items())


def _io_entries(topo, n_src: int, n_rcv: int):
    """Sources and receivers spread over the one-sided (I/O) faces of a topology, unit vectors of
    the face's modes: the face-level structure of the workload's I/O (the timing does not depend
    on the values)."""
    io = [f for f in range(topo.n_faces) if len(topo.face_cells[f]) == 1]
    src, rcv = [], []
    for j in range(n_src):
        f = io[j % len(io)]
        src.append((f, j, np.full(int(topo.face_M[f]), 1.0 / math.sqrt(topo.face_M[f]))))
    for j in range(n_rcv):
        f = io[(7 * j) % len(io)]
        rcv.append((f, j, np.full(int(topo.face_M[f]), 1.0 / math.sqrt(topo.face_M[f]))))
    return src, rcv


def _exported_rom(LR):
    """The library ROM's topology and FP64 coefficients as the oracle's containers."""
    cm, cfp, cf, fM, fc, g, gh, fm = LR.export()
    faces = [list(map(int, cf[cfp[c]:cfp[c + 1]])) for c in range(len(cm))]
    topo = synth.RomTopology(np.asarray(cm, np.int64), faces, np.asarray(fM, np.int64),
                             [[int(x) for x in row if x >= 0] for row in fc])
    gam, ghat, o = [], [], 0
    for c in range(len(cm)):
        K, m = int(sum(fM[faces[c]])), int(cm[c])
        gam.append([g[o + k * K * K:o + (k + 1) * K * K].reshape(K, K) for k in range(m)])
        ghat.append([gh[o + k * K * K:o + (k + 1) * K * K].reshape(K, K) for k in range(m)])
        o += m * K * K
    fmass, o = [], 0
    for M in fM:
        fmass.append(fm[o:o + M * M].reshape(M, M))
        o += M * M
    return topo, synth.RomCoefficients(gam, ghat, fmass)


def oracle_rate(topo, co, n_src: int, n_rcv: int, n_steps_sample: int, tau: float, prepared=None):
    """The oracle's ROM leapfrog on a given topology and coefficient set, all cells and sources,
    a bounded number of time steps.  Returns (rate in source·cell-steps/s, seconds, label, threads,
    prepared stepper for reuse)."""
    from oracle import online
    if prepared is None:
        src, rcv = _io_entries(topo, n_src, n_rcv)
        gt = online.dense_io(topo, src, n_src, "src")
        qt = online.dense_io(topo, rcv, n_rcv, "rcv")
        prepared = _oracle_stepper(topo, co, gt, qt)
    step, label, threads = prepared
    w = synth.ricker(np.arange(n_steps_sample) * tau, 0.25 / tau)
    t0 = time.perf_counter()
    step(w, tau, n_steps_sample)
    dt = time.perf_counter() - t0
    return topo.n_cells * n_src * n_steps_sample / dt, dt, label, threads, prepared


def oracle_baseline(topo, co, n_src: int, n_rcv: int, tau: float, what: str, target_s: float = 15.0):
    """cpu_baseline entry: a 2-step probe, then a sample sized to about ``target_s`` seconds."""
    rate, dt, label, threads, prep = oracle_rate(topo, co, n_src, n_rcv, 2, tau)
    steps = int(min(2000, max(2, target_s / max(dt / 2, 1e-9))))
    rate, dt, label, threads, _ = oracle_rate(topo, co, n_src, n_rcv, steps, tau, prep)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "seconds": dt,
            "sample": "all %d cells x %d sources x %d time steps of the oracle's ROM leapfrog (%s loops) on %s"
                      % (topo.n_cells, n_src, steps, label, what)}


def run_reference(args):
    """The oracle on the host cores, on the workload's ROM shape: the 512 cells with the K_i and
    m_i the library builds for it (45 modes on every interior face, the I/O faces of the top
    cells with their node counts), random SPD coefficients of those sizes (the host's time does
    not depend on the values), the workload's sources and receivers."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = _workload(band=args.band, n_modes=args.modes, cellwl=args.cellwl)
    n_src, n_rcv = len(wl.src_nodes), len(wl.rcv_nodes)
    nc = tuple(wl.grid.n[a] // wl.cell[a] for a in range(3))
    topo = synth.box_topology(nc, modes=wl.n_modes, m=wl.m, io_cells=_box_io(wl), seed=7)
    co = synth.random_coefficients(topo, seed=7)
    tau = 1e-3
    sample = args.ref_sample
    prep = None
    for _ in range(args.warmup):
        _, _, _, _, prep = oracle_rate(topo, co, n_src, n_rcv, 1, tau, prep)
    times = []
    for _ in range(args.steps):
        rate, dt, label, cores, prep = oracle_rate(topo, co, n_src, n_rcv, sample, tau, prep)
        times.append(dt)
    units = topo.n_cells * n_src * sample
    value = units / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(wl, {"precision": "fp64 (oracle, %s)" % label,
                                   "K_max": int(max(topo.cell_K()))}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "all %d cells x %d sources x %d time steps per bench step (%s oracle loops, "
                                       "the workload's ROM block sizes, random SPD values)"
                                       % (topo.n_cells, n_src, sample, label)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- ranks
def whole_job_rate(units_per_rank: float, seconds: float, world: int, dist=None, device=None):
    """Throughput of the whole job: the units all ranks processed over the slowest rank's time.

    Every rank runs its own replica (no data-path collective); the only exchange is this max over
    ranks of the timed seconds (an all-reduce on ``device``: the GPU under NCCL, the CPU under
    gloo).  Collective: all ranks must call it.  Returns (rate, slowest seconds)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return world * units_per_rank / seconds, seconds


# ----------------------------------------------------------------------------- native
def _kernel_model(rom_info, topo_K, topo_m, n_src, es):
    """Algorithmic bytes and flops of one cell-kernel launch (one time step, all cells)."""
    byts = flops = 0.0
    for K, m in zip(topo_K, topo_m):
        coef = (2 * m - 1) * K * K * es                         # Gamma^1..m, Gamma-hat^2..m, read once
        state = (K + 3 * (m - 1) * K + K) * n_src * es           # U^1 gather, U^k, U^k_old, U^k_new, F^1 out
        byts += coef + state
        flops += 2.0 * (2 * m - 1) * K * K * n_src
    return byts, flops


SCHED_NAMES = ["graph", "graph_stream", "persistent", "persistent_stream", "graph_split"]

def _traffic_record(kernel: str, sources):
    """ncu DRAM bytes per launch of a cell kernel, if recorded for these exact kernel sources."""
    path = os.path.join(ROOT, "profiles", "cell_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get("kernels", {}).get(kernel)
    if not rec:
        return None
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_1604_06750_gb300", "csrc", f), "rb").read())
    return rec.get("bytes_per_launch") if rec.get("source_sha256") == h.hexdigest() else None


def _timed_runs(obj, n_steps, wd, tr, reps, stream, flush=None):
    """``reps`` whole simulations (state reset, n_steps) timed with CUDA events on ``stream``."""
    import torch
    times = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)                                # L2 flush between bench steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj.reset()
        obj.step(n_steps, wd, tr, use_graph=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _per_receiver(a, b):
    """Largest relative L2 over receivers (each receiver's trace over steps and sources)."""
    nb = np.linalg.norm(b)
    worst = 0.0
    for r in range(b.shape[1]):
        d = np.linalg.norm(b[:, r, :])
        if d > 1e-12 * nb:
            worst = max(worst, float(np.linalg.norm(a[:, r, :] - b[:, r, :]) / d))
    return worst


def run_native(args):
    import torch
    import paper_1604_06750_gb300 as P
    from paper_1604_06750_gb300 import build as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    P.lib()
    wl = _workload(band=args.band, n_modes=args.modes, cellwl=args.cellwl)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # ---- off-line (not timed in the metric)
    t0 = time.perf_counter()
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    io = np.concatenate([wl.src_nodes, wl.rcv_nodes]).astype(np.int32)
    LP = P.Partition(L, wl.cell, io)
    lam = L.lambda_max(1e-7)
    tau = wl.cfl_fraction * 2.0 / math.sqrt(lam)
    s = -(2 * math.pi * wl.f_max) ** 2
    t1 = time.perf_counter()
    LR = P.Rom.build(LP, wl.m, wl.n_modes, s, cg_tol=1e-12)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
    cm, cfp, cf, fM, fc, _, _, _ = LR.export()
    Ks = [int(sum(fM[cf[cfp[c]:cfp[c + 1]]])) for c in range(len(cm))]
    nst, S, R = wl.n_steps, len(wl.src_nodes), len(wl.rcv_nodes)
    ncell = len(cm)
    units = ncell * S * nst
    w = synth.ricker(np.arange(nst) * tau, wl.f_peak)
    wd = torch.tensor(w, device=dev)
    factor = not args.plain_fp32
    if args.profile:
        if args.prec_profile == "tf32_tc":
            sim = P.Sim(LR, P.TF32_TC, tau, corner_correction=True)
        else:
            sim = P.Sim(LR, P.FP32, tau, corner_correction=True, factor_last=factor)
            sim.set_schedule(args.sched)
        if args.wide_var:
            sim.set_tile(groups=args.wide_var)
        tr = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
        sim.step(args.profile, wd, tr, use_graph=False)
        torch.cuda.synchronize()
        sim.info()
        print(json.dumps({"profile_steps": args.profile, "precision": args.prec_profile, "factor_last": factor,
                          "schedule": SCHED_NAMES[sim.schedule()[0]],
                          "tile": sim.tile(), "K_max": max(Ks)}))
        return
    # ---- candidate headline arms: FP32 on the CUDA cores (autotuned schedule and tile, the last
    # coefficient applied as its Cholesky factor), and FP32-class products on the tensor cores
    # (TF32 split hi + lo, the wide tcgen05 kernel); each timed the same way, the faster one whose
    # traces stay within the FP32 class of the FP64 ROM is the headline
    flush = torch.empty(int(512e6) // 4, device=dev, dtype=torch.float32)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12            # FP32 FMA lanes x 2 flops x clock (TFLOP/s)
    algo_bytes, algo_flops = _kernel_model(None, Ks, cm, S, 4)

    def measure(sim, sched, kname, ksrc):
        tr = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
        _timed_runs(sim, nst, wd, tr, args.warmup, stream)       # warm-up (captures the CUDA graph)
        torch.cuda.synchronize()
        clocks = Clocks(torch.cuda.current_device())
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        times = _timed_runs(sim, nst, wd, tr, args.steps, stream, flush)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ck = clocks.stop()
        value, t_step = whole_job_rate(units, statistics.mean(times), world, dist, dev)
        sim.info()                                              # raises if a bounded device wait gave up
        trn = tr.double().cpu().numpy()
        # per-kernel timing (eager, CUDA events on the launching stream): the cell kernel of the
        # chosen schedule (the persistent schedule runs the plain cell body inside one kernel, so
        # the graph schedule stands in for it)
        prof_sched = {P.SCHED_PERSIST: P.SCHED_GRAPH, P.SCHED_PERSIST_STREAM: P.SCHED_GRAPH_STREAM}.get(sched, sched)
        sim.set_schedule(prof_sched)
        sim.reset()
        ms = sim.step_profile(200, wd, tr)
        sim.set_schedule(sched)
        cell_s = ms[0] / 1e3
        achieved_gbs = algo_bytes / cell_s / 1e9
        achieved_tf = algo_flops / cell_s / 1e12
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                "traffic": _traffic_record(kname, ksrc)}
        if algo_flops / algo_bytes >= alu_peak * 1e12 / (hbm * 1e9) and "tensor" not in kname:
            roof = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved_tf / alu_peak, "traffic": roof["traffic"]}
        roof.update({"kernel": kname, "algorithmic_bytes_per_launch": algo_bytes,
                     "algorithmic_flops_per_launch": algo_flops, "intensity_flop_per_byte": algo_flops / algo_bytes,
                     "ms_per_launch": ms[0], "tile": sim.tile(), "fp32_alu_frac": achieved_tf / alu_peak,
                     "fp32_alu_peak_tflops": alu_peak,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback",
                     "other_kernels_ms": {"k_face": ms[1], "k_corner": ms[2]}})
        return {"sim": sim, "sched": sched, "value": value, "t_step": t_step, "clocks": ck, "tr": trn, "roof": roof,
                "kper": int(sim.info()[6])}

    arms = {}
    sim = P.Sim(LR, P.FP32, tau, corner_correction=True, factor_last=factor)
    sched, sched_ms = sim.autotune(100)
    wide = max(Ks) > 128 or factor
    if sched in (P.SCHED_GRAPH_STREAM, P.SCHED_PERSIST_STREAM):
        kname = "k_cell_w (wide TMA-streamed)" if wide else "k_cell_s"
    elif sched == P.SCHED_GRAPH_SPLIT:
        kname = "k_flux+k_accel"
    else:
        kname = "k_cell<float,16> (factored last coefficient)" if factor else "k_cell<float,16>"
    ksrc = {"k_cell_w (wide TMA-streamed)": ["cell_wide.cuh", "cell_stream.cuh"],
            "k_cell_s": ["cell_stream.cuh", "online.cu"], "k_flux+k_accel": ["cell_split.cuh", "online.cu"]}.get(
        kname, ["online.cu"])
    arms["fp32"] = measure(sim, sched, kname, ksrc)
    arms["fp32"]["autotune"] = {SCHED_NAMES[k]: (float(sched_ms[k]) if sched_ms[k] >= 0 else None)
                                for k in range(len(SCHED_NAMES))}
    tw_note = None
    if factor and args.arm in ("auto", "tf32_tc"):
        try:
            simtw = P.Sim(LR, P.TF32_TC, tau, corner_correction=True)
        except P.MssError as ex:
            tw_note = str(ex)
        else:
            simtw.autotune(100)                                 # copy-ring depth of its cell kernel
            arms["tf32_tc"] = measure(simtw, P.SCHED_GRAPH, "k_cell_tw (tensor-core TF32 split)",
                                      ["cell_tw.cuh", "cell_tc.cuh"])
    # ---- FP64 ROM stepping (same coefficients), one run
    sim64 = P.Sim(LR, P.FP64, tau, corner_correction=True)
    tr64 = torch.zeros((nst, R, S), device=dev, dtype=torch.float64)
    _timed_runs(sim64, nst, wd, tr64, 1, stream)
    t64 = _timed_runs(sim64, nst, wd, tr64, 1, stream, flush)[0]
    rom64 = tr64.cpu().numpy()
    del sim64, tr64
    # ---- fine grid on the same GPU, original graph, same tau and steps: FP64 is the reference
    # of the accuracy target; FP32 is the comparison path at equal accuracy, timed
    fine64 = P.FineSim(L, P.FP64, tau, wl.src_nodes, wl.rcv_nodes)
    trf64 = torch.zeros((nst, R, S), device=dev, dtype=torch.float64)
    _timed_runs(fine64, nst, wd, trf64, 1, stream)
    ref = trf64.cpu().numpy()
    del fine64, trf64
    fine = P.FineSim(L, P.FP32, tau, wl.src_nodes, wl.rcv_nodes)
    trf = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
    _timed_runs(fine, nst, wd, trf, 1, stream)
    fine_times = _timed_runs(fine, nst, wd, trf, max(1, args.steps), stream, flush)
    tfine = statistics.mean(fine_times)
    fine32 = trf.double().cpu().numpy()
    del fine, trf
    # ---- the headline arm: the fastest whose traces stay within FP32 class (1e-3) of the FP64 ROM
    for k, arm in arms.items():
        arm["vs_rom_fp64"] = _rel(arm["tr"], rom64)
    ok = [k for k, arm in arms.items() if arm["vs_rom_fp64"] <= 1e-3] or ["fp32"]
    head = min(ok, key=lambda k: arms[k]["t_step"])
    if args.arm != "auto" and args.arm in arms:
        head = args.arm
    H = arms[head]
    sim, sched, value, t_step, ck, roof = H["sim"], H["sched"], H["value"], H["t_step"], H["clocks"], H["roof"]
    tr32, kper = H["tr"], H["kper"]
    err = _rel(tr32, ref)
    acc = {"target": ACCURACY_TARGET, "reference": "same GPU's FP64 fine-grid leapfrog on the original graph",
           "rom_fp32_vs_fine_fp64": err, "rom_fp32_vs_fine_fp64_max_per_receiver": _per_receiver(tr32, ref),
           "rom_fp64_vs_fine_fp64": _rel(rom64, ref), "rom_fp32_vs_rom_fp64": _rel(tr32, rom64),
           "fine_fp32_vs_fine_fp64": _rel(fine32, ref), "met": bool(err <= ACCURACY_TARGET)}
    other = {}
    for k, arm in arms.items():
        if k != head:
            other[k] = {"value": arm["value"], "unit": UNIT, "ms_per_step": 1e3 * arm["t_step"],
                        "schedule": SCHED_NAMES[arm["sched"]], "rom_vs_rom_fp64": arm["vs_rom_fp64"],
                        "rom_vs_fine_fp64": _rel(arm["tr"], ref), "cell_kernel": arm["roof"]["kernel"],
                        "cell_kernel_ms": arm["roof"]["ms_per_launch"], "cell_kernel_hbm_frac": arm["roof"]["frac"]}
    if tw_note:
        other["tf32_tc"] = {"unavailable": tw_note}
    # ---- end to end through the C ABI with host buffers (H2D waveform, D2H traces)
    e2e_times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        a = time.perf_counter()
        host_tr = sim.run_host(w)
        e2e_times.append(time.perf_counter() - a)
    e2e = {"value": whole_job_rate(units, statistics.mean(e2e_times), world, dist, dev)[0], "unit": UNIT,
           "h2d_bytes_per_step": int(w.nbytes), "d2h_bytes_per_step": int(host_tr.nbytes)}
    # ---- oracle on the host cores on this ROM's own coefficients, bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        topo, co = _exported_rom(LR)
        cpu = oracle_baseline(topo, co, S, R, tau, "the workload's own ROM coefficients (exported from the GPU "
                                                   "build; sources and receivers on its I/O faces)")
        del topo, co
    # ---- CFL check of the bench's tau through the sim's own kernels (not timed; state restored)
    try:
        stability = {"growth_over_300_source_free_steps": sim.check_stability(300, seed=1), "tau": tau}
    except P.MssError as ex:
        stability = {"error": str(ex), "tau": tau}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    launches = {P.SCHED_GRAPH: nst * kper, P.SCHED_GRAPH_STREAM: nst * kper,
                P.SCHED_GRAPH_SPLIT: nst * (kper + 1)}.get(sched, -(-nst // 512))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "tf32x3+f32" if head == "tf32_tc" else "f32", "data": "synthetic",
            "config": _config(wl, {"precision": ("fp32 state and coefficients, cell products on the tensor cores "
                                                 "as TF32 with both operands split hi + lo (three products), last "
                                                 "coefficient as its Cholesky factor") if head == "tf32_tc" else
                                                ("fp32 state and coefficients, last coefficient as its Cholesky "
                                                 "factor" if factor else "fp32 state and coefficients"),
                                   "corner_correction": True, "K_max": max(Ks), "tau": tau,
                                   "l2": "flushed between steps (512 MB write)",
                                   "parallelism": "independent source batches per GPU" if world > 1 else "single GPU"}),
            "clocks": ck, "gpu_launches": int(args.steps * launches),
            "schedule": {"chosen": SCHED_NAMES[sched], "arm": head,
                         "fp32_autotune_ms_per_time_step": arms["fp32"]["autotune"]},
            "other_arms": other,
            "receiver_rel_l2": acc,
            "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
            "fine_grid": {"value": units / tfine, "unit": UNIT, "ms": 1e3 * tfine,
                          "receiver_rel_l2_vs_fine_fp64": acc["fine_fp32_vs_fine_fp64"],
                          "note": "FP32 7-point leapfrog on the same grid, same tau and steps (the accuracy "
                                  "reference's own method, at equal or better accuracy); cells counted on the "
                                  "same partition"},
            "speedup_vs_fine_grid": tfine / t_step,
            "fp64_rom": {"value": units / t64, "unit": UNIT, "ms": 1e3 * t64},
            "fp32_tc": {"unavailable": "split-BF16 tensor-core cell kernels need K_i <= 128; this workload has K "
                                      "up to %d (the TF32 tensor-core arm covers it)" % max(Ks)} if max(Ks) > 128 else None,
            "offline_s": {"assemble_partition_cfl": t1 - t0, "gpu_rom_build": t2 - t1},
            "stability": stability}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_c3(args):
    """The 256^3 dipping-layer workload end to end on one GPU: GPU off-line build of all 4096 cell
    ROMs (m = 4 in every cell, or with --c3-rule m_i in 3..6 per cell by the library's layer-count
    rule, mss_layer_rule), 256 sources on
    face centres of the skeleton plane one cell below the top, 128 receivers on a line in that
    plane, 6000 steps; FP32 with split-BF16 tensor-core products (the many-source path), BF16
    products and CUDA-core FP32 timed; receiver error against the same GPU's FP64 fine-grid
    leapfrog on the original graph; FP64 parity against the oracle's ROM leapfrog on the exported
    coefficients for three sampled sources over a short window.  One JSON line."""
    import torch
    import paper_1604_06750_gb300 as P
    from paper_1604_06750_gb300 import build as B
    from oracle import online
    B.build()
    P.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    wl = synth.workload_3d_dipping(args.c3_n, 16, m=4, n_modes=args.c3_modes, n_steps=args.c3_steps)
    t0 = time.perf_counter()
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    io = np.concatenate([wl.src_nodes, wl.rcv_nodes]).astype(np.int32)
    LP = P.Partition(L, wl.cell, io)
    lam = L.lambda_max(1e-7)
    tau = wl.cfl_fraction * 2.0 / math.sqrt(lam)
    s = -(2 * math.pi * wl.f_max) ** 2
    t1 = time.perf_counter()
    rule = None
    t_build0 = t1
    if args.c3_rule:
        w_max = 2 * math.pi * wl.f_max
        cm_rule, err_rule = P.Rom.layer_rule(LP, wl.n_modes, s, w_max, (3, 6), 1e-4, cg_tol=1e-12)
        t_build0 = time.perf_counter()
        rule = {"m_counts": {str(k): int(np.sum(cm_rule == k)) for k in range(3, 7)}, "tol": 1e-4,
                "largest_error_kept": float(np.max(err_rule)), "seconds": t_build0 - t1}
        LR = P.Rom.build(LP, 6, wl.n_modes, s, cg_tol=1e-12, cell_m=cm_rule)
    else:
        LR = P.Rom.build(LP, wl.m, wl.n_modes, s, cg_tol=1e-12)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
    cm, cfp, cf, fM, fc, _, _, _ = LR.export()
    Ks = [int(sum(fM[cf[cfp[c]:cfp[c + 1]]])) for c in range(len(cm))]
    nst, S, R = wl.n_steps, len(wl.src_nodes), len(wl.rcv_nodes)
    units = len(cm) * S * nst
    w = synth.ricker(np.arange(nst) * tau, wl.f_peak)
    wd = torch.tensor(w, device=dev)
    flush = torch.empty(int(512e6) // 4, device=dev, dtype=torch.float32)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    out = {"mode": "c3", "config": {"workload": "3d_dipping_%d: %d^3 voxels, %d cells of 16^3 (uneven K_i %d..%d), "
                                                "m=%s, %d modes/face, %d sources, %d receivers, %d steps"
                                                % (args.c3_n, args.c3_n, len(cm), min(Ks), max(Ks),
                                                   "3..6" if rule else "4", wl.n_modes, S, R, nst),
                                    "band": "Ricker peak at 1/10 grid Nyquist",
                                    "layers": ("m_i per cell by the layer-count rule (3..6, tol 1e-4)" if rule
                                               else "m = 4 in every cell")},
           "layer_rule": rule,
           "unit": UNIT, "offline_s": {"assemble_partition_cfl": t1 - t0, "gpu_rom_build": t2 - t_build0},
           "tau": tau, "precisions": {}}
    clocks = Clocks(0)
    clocks.start()
    traces = {}
    for name, prec in (("fp32_tc", P.FP32_TC), ("bf16_tc", P.BF16_TC), ("fp32", P.FP32), ("tf32_tc", P.TF32_TC)):
        try:
            sim = P.Sim(LR, prec, tau, corner_correction=True)
        except P.MssError as ex:
            out["precisions"][name] = {"unavailable": str(ex)}
            continue
        k, msk = sim.autotune(20)
        tr = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
        _timed_runs(sim, nst, wd, tr, 1, stream)
        t = _timed_runs(sim, nst, wd, tr, 1, stream, flush)[0]
        sim.info()
        traces[name] = tr.double().cpu().numpy()
        out["precisions"][name] = {"value": units / t, "ms_per_time_step": 1e3 * t / nst,
                                   "schedule": SCHED_NAMES[k]}
        del sim, tr
        torch.cuda.empty_cache()
    # the accuracy reference: FP64 fine grid on the original graph, same tau and steps
    fine64 = P.FineSim(L, P.FP64, tau, wl.src_nodes, wl.rcv_nodes)
    trf = torch.zeros((nst, R, S), device=dev, dtype=torch.float64)
    fine64.step(nst, wd, trf)
    torch.cuda.synchronize()
    ref = trf.cpu().numpy()
    del fine64, trf
    torch.cuda.empty_cache()
    fine = P.FineSim(L, P.FP32, tau, wl.src_nodes, wl.rcv_nodes)
    trf = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
    _timed_runs(fine, nst, wd, trf, 1, stream)
    tf = _timed_runs(fine, nst, wd, trf, 1, stream, flush)[0]
    fine32 = trf.double().cpu().numpy()
    del fine, trf
    torch.cuda.empty_cache()
    out["clocks"] = clocks.stop()
    out["fine_grid_fp32"] = {"value": units / tf, "ms_per_time_step": 1e3 * tf / nst,
                             "receiver_rel_l2_vs_fine_fp64": rel(fine32, ref)}
    for name in traces:
        out["precisions"][name]["receiver_rel_l2_vs_fine_fp64"] = rel(traces[name], ref)
        out["precisions"][name]["receiver_rel_l2_vs_fp32_tc"] = rel(traces[name], traces["fp32_tc"])
    # FP64 parity against the oracle on the exported coefficients: three sampled sources, no
    # corner correction (the oracle's C loops restate the leapfrog without it), a short window
    npar = args.c3_parity_steps
    pick = [0, S // 2, S - 1]
    topo, co = _exported_rom(LR)
    src_e, rcv_e, _ = LR.export_io()
    src3 = [(f, pick.index(j), v) for (f, j, v) in src_e if j in pick]
    gt = online.dense_io(topo, src3, len(pick), "src")
    qt = online.dense_io(topo, rcv_e, R, "rcv")
    step, label, threads = _oracle_stepper(topo, co, gt, qt)
    t3 = time.perf_counter()
    oref = step(w[:npar], tau, npar)
    t_or = time.perf_counter() - t3
    sim64 = P.Sim(LR, P.FP64, tau, corner_correction=False)
    tr64 = torch.zeros((npar, R, S), device=dev, dtype=torch.float64)
    sim64.step(npar, wd[:npar], tr64)
    torch.cuda.synchronize()
    g64 = tr64.cpu().numpy()[:, :, pick]
    simtc = P.Sim(LR, P.FP32_TC, tau, corner_correction=False)
    trtc = torch.zeros((npar, R, S), device=dev, dtype=torch.float32)
    simtc.step(npar, wd[:npar], trtc)
    torch.cuda.synchronize()
    gtc = trtc.double().cpu().numpy()[:, :, pick]
    out["parity_vs_oracle"] = {"sources": pick, "steps": npar, "fp64_rel_l2": rel(g64, oref),
                               "fp32_tc_rel_l2": rel(gtc, oref), "oracle": "%s, %d threads, %.1f s"
                               % (label, threads, t_or)}
    print(json.dumps(out))


def run_many_sources(args):
    """The 4096-cell, 256-source on-line shape of the 256^3 dipping-layer workload (synthetic SPD
    coefficients, m_i in 3..6, uneven K_i): throughput of every precision, the CUDA-core FP32
    schedule picked by the autotuner, per-kernel roofline of the cell phase.  One JSON line."""
    import torch
    import paper_1604_06750_gb300 as P
    from paper_1604_06750_gb300 import build as B
    B.build()
    P.lib()
    dev = torch.device("cuda", 0)
    topo, co, src, rcv = synth.many_source_case(n_cells=(args.box,) * 3)
    R = P.Rom.import_(topo, co)
    R.set_io(256, src, 128, rcv)
    del co
    if args.profile:
        prec = {"fp32": P.FP32, "fp32_tc": P.FP32_TC, "bf16_tc": P.BF16_TC}[args.prec]
        sim = P.Sim(R, prec, 0.05)
        sim.set_schedule(args.sched)
        w = torch.tensor(synth.ricker(np.arange(args.profile) * 0.05, 4.0), device=dev)
        tr = torch.zeros((args.profile, 128, 256), device=dev, dtype=torch.float32)
        sim.step(args.profile, w, tr, use_graph=False)
        torch.cuda.synchronize()
        sim.info()
        print(json.dumps({"profile_steps": args.profile, "precision": args.prec, "box": args.box}))
        return
    Ks, ms = topo.cell_K(), topo.cell_m
    nst, tau = args.many_steps, 0.05
    w = torch.tensor(synth.ricker(np.arange(nst) * tau, 4.0), device=dev)
    units = topo.n_cells * 256 * nst
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    algo_bytes, algo_flops = _kernel_model(None, Ks, ms, 256, 4)
    flush = torch.empty(int(512e6) // 4, device=dev, dtype=torch.float32)
    out = {"config": {"workload": "many_sources: %d cells (%d^3 box with walls, K_i 45..90), m_i 3..6, "
                                  "256 sources, 128 receivers, synthetic SPD coefficients" % (topo.n_cells, args.box),
                      "time_steps": nst},
           "unit": UNIT, "precisions": {}}
    clocks = Clocks(0)
    clocks.start()
    for name, prec in (("fp32", P.FP32), ("fp32_tc", P.FP32_TC), ("bf16_tc", P.BF16_TC), ("fp64", P.FP64)):
        sim = P.Sim(R, prec, tau)
        rec = {}
        if True:
            k, msk = sim.autotune(20)
            rec["schedule"] = SCHED_NAMES[k]
            rec["autotune_ms_per_time_step"] = {SCHED_NAMES[i]: (float(msk[i]) if msk[i] >= 0 else None)
                                                for i in range(len(SCHED_NAMES))}
        tr = torch.zeros((nst, 128, 256), device=dev, dtype=torch.float64 if prec == P.FP64 else torch.float32)
        sim.step(nst, w, tr)
        times = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            sim.reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sim.step(nst, w, tr)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        sim.info()
        t = statistics.mean(times)
        rec.update({"value": units / t, "ms_per_time_step": 1e3 * t / nst})
        cur, _ = sim.schedule()
        if cur in (2, 3):
            sim.set_schedule({2: 0, 3: 1}[cur])
        rec["profiled_schedule"] = SCHED_NAMES[sim.schedule()[0]]
        sim.reset()
        kms = sim.step_profile(min(nst, 50), w, tr)
        es = 8 if prec == P.FP64 else 4
        ab = _kernel_model(None, Ks, ms, 256, es)[0]
        rec["cell_kernel_ms"] = kms[0]
        rec["face_kernel_ms"] = kms[1]
        rec["roofline"] = {"bound": "hbm", "achieved": ab / (kms[0] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": ab / (kms[0] / 1e3) / 1e9 / hbm, "algorithmic_bytes_per_launch": ab,
                           "algorithmic_flops_per_launch": algo_flops}
        out["precisions"][name] = rec
        del sim, tr
        torch.cuda.empty_cache()
    out["clocks"] = clocks.stop()
    print(json.dumps(out))


def run_surrogate(args):
    """Learned-surrogate off-line stage beside the exact one on the 3D layered workload.

    Training cells: 16^3 cells of 64^3 media from the same layered recipe (other random-field
    seeds), labelled by the exact off-line stage; the network (4 stride/plain 3x3x3 conv layers
    of 32 channels, dense head) is trained by the library's own kernels.  The 512-cell 128^3
    workload's ROM is then built from a skeleton by inference + transfer-function screen +
    exact fallback at several screen tolerances and stepped (FP32, corners) against the exact
    ROM and the fine grid.  One JSON line."""
    import torch
    import paper_1604_06750_gb300 as P
    from paper_1604_06750_gb300 import build as B
    B.build()
    P.lib()
    dev = torch.device("cuda", 0)
    wl = _workload(SURROGATE_WORKLOAD)
    m, nm = wl.m, wl.n_modes
    s = -(2 * math.pi * wl.f_max) ** 2
    io_slots = 8
    Kp = 6 * nm + io_slots
    D = (2 * m - 1) * Kp * (Kp + 1) // 2
    # ---- training data: exact ROMs of the training media
    t0 = time.perf_counter()
    xs, fs, ts, ms_ = [], [], [], []
    build_s = 0.0
    for k in range(args.train_media):
        tw = synth.workload_3d_layers(64, 16, m=m, n_modes=nm, n_src=4, n_steps=10, seed_index=100 + k)
        L = P.Operator(tw.grid, tw.sigma, tw.rho)
        LP = P.Partition(L, tw.cell, np.concatenate([tw.src_nodes, tw.rcv_nodes]).astype(np.int32))
        cells = np.arange(int(LP.info()[0]))
        tb = time.perf_counter()
        LR = P.Rom.build(LP, m, nm, s, cg_tol=1e-12)
        torch.cuda.synchronize()
        build_s += time.perf_counter() - tb
        t, mk = LR.pack(cells, nm, io_slots, m)
        x, f = LP.cell_inputs(cells, nm, io_slots)
        xs.append(x)
        fs.append(f)
        ts.append(t)
        ms_.append(mk)
    T = np.concatenate(ts)
    MK = np.concatenate(ms_)
    X = torch.from_numpy(np.concatenate(xs)).to(dev)
    Fe = torch.from_numpy(np.concatenate(fs)).to(dev)
    Td = torch.from_numpy(T.astype(np.float32)).to(dev)
    Md = torch.from_numpy(MK).to(dev)
    t_data = time.perf_counter() - t0
    sur = P.Surrogate(16, 7, D, channels=32, hidden=128, seed=1)
    sur.fit_output_transform(T, MK)
    loss = torch.zeros(1, device=dev)
    g = torch.Generator().manual_seed(0)
    n = X.shape[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = None
    for it in range(args.train_iters):
        idx = torch.randint(0, n, (args.batch,), generator=g).to(dev)
        lr = 2e-3 if it < args.train_iters * 2 // 3 else 5e-4
        sur.train_step(X[idx].contiguous(), Fe[idx].contiguous(), Td[idx].contiguous(), lr, loss=loss,
                       mask=Md[idx].contiguous())
        if it == 0:
            torch.cuda.synchronize()
            first = float(loss.item())
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    last = float(loss.item())
    # ---- the workload: exact ROM, fine grid
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, np.concatenate([wl.src_nodes, wl.rcv_nodes]).astype(np.int32))
    lam = L.lambda_max(1e-7)
    tau = wl.cfl_fraction * 2.0 / math.sqrt(lam)
    cells = np.arange(int(LP.info()[0]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    LR = P.Rom.build(LP, m, nm, s, cg_tol=1e-12)
    torch.cuda.synchronize()
    t_exact = time.perf_counter() - t0
    LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
    nst, S, R = wl.n_steps, len(wl.src_nodes), len(wl.rcv_nodes)
    w = torch.tensor(synth.ricker(np.arange(nst) * tau, wl.f_peak), device=dev)

    def traces(rom):
        sim = P.Sim(rom, P.FP32, tau, corner_correction=True)
        tr = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
        sim.step(nst, w, tr)
        torch.cuda.synchronize()
        sim.info()
        return tr.double().cpu().numpy()

    ref = traces(LR)
    fine = P.FineSim(L, P.FP32, tau, wl.src_nodes, wl.rcv_nodes)
    trf = torch.zeros((nst, R, S), device=dev, dtype=torch.float32)
    fine.step(nst, w, trf)
    torch.cuda.synchronize()
    fine_tr = trf.double().cpu().numpy()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    runs = []
    for tol in (1e-3, 1e-2, 5e-2, 1e300):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        SK = P.Rom.skeleton(LP, m, nm, s, cg_tol=1e-12)
        err, fb = sur.infer(SK, cells, nm, io_slots, tol)
        torch.cuda.synchronize()
        t_sur = time.perf_counter() - t0
        SK.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
        try:
            tr = traces(SK)
            e_rom, e_fine = rel(tr, ref), rel(tr, fine_tr)
        except P.MssError as ex:          # a surrogate ROM may fail the sim's checks
            e_rom = e_fine = None
            tr = None
        runs.append({"screen_tol": None if tol > 1 else tol, "offline_s": t_sur, "fallback_cells": int(fb.sum()),
                     "screen_err_median": float(np.median(err)), "screen_err_p10": float(np.percentile(err, 10)),
                     "screen_err_p90": float(np.percentile(err, 90)),
                     "receiver_rel_l2_vs_exact_rom": e_rom, "receiver_rel_l2_vs_fine": e_fine})
    out = {"mode": "surrogate", "workload": wl.name, "cells": int(len(cells)),
           "network": {"conv_layers": 4, "channels": 32, "hidden": 128, "outputs": D, "params": sur.n_params,
                       "weights": "bf16 (fp32 masters)"},
           "training": {"media": args.train_media, "cells": int(n), "iterations": args.train_iters,
                        "batch": args.batch, "loss_first": first, "loss_last": last, "train_s": t_train,
                        "label_build_s": build_s, "data_s": t_data},
           "exact_offline_s": t_exact, "exact_rom_vs_fine": rel(ref, fine_tr), "runs": runs}
    print(json.dumps(out))


def run_accuracy(args):
    """ROM against the fine grid at equal receiver accuracy, by default at the operating point of
    the paper's experiments (Section 7: cells about one minimum wavelength across, m = 4);
    ``--acc-band nyquist --acc-m 6`` measures the 1/10-Nyquist band with more layers.

    The 3D layered recipe on an n^3 grid of 16^3-voxel cells, band limit with a minimum wavelength
    of one cell edge, 8 surface sources, fine-grid CFL step for both.  For each face-mode count:
    GPU off-line build, FP32 and FP64 ROM stepping (Appendix D corners, graph schedule), receiver
    rel-L2 against the same GPU's FP64 fine-grid leapfrog, and ms per time step of the FP32 ROM
    beside the FP32 fine grid.  One JSON line."""
    import torch
    import paper_1604_06750_gb300 as P
    from paper_1604_06750_gb300 import build as B
    B.build()
    P.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    modes = [int(x) for x in args.acc_modes.split(",")]
    wl = synth.workload_3d_layers(args.acc_n, 16, m=args.acc_m, n_modes=modes[0], n_src=args.acc_src,
                                  n_steps=args.acc_steps, band=args.acc_band, cell_wavelengths=args.acc_cellwl)
    if args.acc_src_centre:          # sources at the cell centres of their line (8 voxels from the faces)
        wl.src_nodes = np.array([[args.acc_n, wl.src_nodes[0][1], 8 + 16 * j] for j in range(args.acc_n // 16)])
    L = P.Operator(wl.grid, wl.sigma, wl.rho)
    LP = P.Partition(L, wl.cell, np.concatenate([wl.src_nodes, wl.rcv_nodes]).astype(np.int32))
    lam = L.lambda_max(1e-7)
    tau = wl.cfl_fraction * 2.0 / math.sqrt(lam)
    s = -args.acc_shift * (2 * math.pi * wl.f_max) ** 2
    nst, S, R = wl.n_steps, len(wl.src_nodes), len(wl.rcv_nodes)
    wd = torch.tensor(synth.ricker(np.arange(nst) * tau, wl.f_peak), device=dev)

    def run(obj, dtype, reps):
        tr = torch.zeros((nst, R, S), device=dev, dtype=dtype)
        obj.reset()
        obj.step(nst, wd, tr, use_graph=True)              # warm-up, captures the graph
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            obj.reset()
            obj.step(nst, wd, tr, use_graph=True)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return tr.double().cpu().numpy(), statistics.mean(ts)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    ref, t_f64 = run(P.FineSim(L, P.FP64, tau, wl.src_nodes, wl.rcv_nodes), torch.float64, 1)
    f32, t_f32 = run(P.FineSim(L, P.FP32, tau, wl.src_nodes, wl.rcv_nodes), torch.float32, 3)
    rows = []
    for nm in modes:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            LR = P.Rom.build(LP, args.acc_m, nm, s, cg_tol=1e-13)
        except P.MssError as ex:        # e.g. a coefficient block that is not SPD: reported, not fatal
            rows.append({"face_modes": nm, "error": str(ex)})
            continue
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        LR.set_io_nodes(LP, wl.src_nodes, wl.rcv_nodes)
        cm, cfp, cf, fM, _, _, _, _ = LR.export()
        Ks = [int(sum(fM[cf[cfp[c]:cfp[c + 1]]])) for c in range(len(cm))]
        cc = not args.acc_no_corners
        r32, t32 = run(P.Sim(LR, P.FP32, tau, corner_correction=cc), torch.float32, 3)
        simf = P.Sim(LR, P.FP32, tau, corner_correction=cc, factor_last=True)
        fsched, _ = simf.autotune(100)
        rf, tf = run(simf, torch.float32, 3)
        r64, t64 = run(P.Sim(LR, P.FP64, tau, corner_correction=cc), torch.float64, 1)
        rows.append({"face_modes": nm, "K_max": max(Ks), "offline_s": t_build,
                     "rel_l2_rom_fp64_vs_fine_fp64": rel(r64, ref), "rel_l2_rom_fp32_vs_fine_fp64": rel(r32, ref),
                     "rel_l2_rom_fp32_factored_vs_fine_fp64": rel(rf, ref),
                     "rel_l2_rom_fp32_factored_vs_rom_fp64": rel(rf, r64),
                     "rom_fp32_ms_per_time_step": 1e3 * t32 / nst, "rom_fp64_ms_per_time_step": 1e3 * t64 / nst,
                     "rom_fp32_factored_ms_per_time_step": 1e3 * tf / nst,
                     "rom_fp32_factored_schedule": SCHED_NAMES[fsched],
                     "fine_fp32_over_rom_fp32_time": t_f32 / t32, "fine_fp32_over_rom_fp32_factored_time": t_f32 / tf})
        print(json.dumps(rows[-1]), file=sys.stderr)
        del LR
    ncells = int(LP.info()[0])
    out = {"mode": "accuracy", "workload": "3d_layers_%d band=%s: %d^3 voxels, %d cells of 16^3, m=%d, %d sources, "
                                          "%d receivers, %d steps" % (args.acc_n, args.acc_band, args.acc_n, ncells,
                                                                      args.acc_m, S, R, nst),
           "f_peak": wl.f_peak, "f_max": wl.f_max, "tau": tau,
           "fine_fp32_ms_per_time_step": 1e3 * t_f32 / nst, "fine_fp64_ms_per_time_step": 1e3 * t_f64 / nst,
           "rel_l2_fine_fp32_vs_fine_fp64": rel(f32, ref), "roms": rows}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--profile", type=int, default=0, help="run N eager time steps after setup and exit")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp32_tc", "bf16_tc"], help="precision of the --profile run")
    ap.add_argument("--sched", type=int, default=0, choices=[0, 1, 2, 3, 4], help="schedule of the --profile run")
    ap.add_argument("--arm", default="auto", choices=["auto", "fp32", "tf32_tc"],
                    help="headline arm (auto: the faster FP32-class one)")
    ap.add_argument("--prec-profile", default="fp32", choices=["fp32", "tf32_tc"],
                    help="precision of the default workload's --profile run")
    ap.add_argument("--wide-var", type=int, default=0, choices=range(0, 9),
                    help="wide cell kernel variant 1..8 of the --profile run (0: the default)")
    ap.add_argument("--many-sources", action="store_true",
                    help="measure the 4096-cell, 256-source launch shape instead (separate JSON line)")
    ap.add_argument("--many-steps", type=int, default=200, help="time steps per timed run of --many-sources")
    ap.add_argument("--box", type=int, default=16, help="cells per box edge of --many-sources")
    ap.add_argument("--surrogate", action="store_true",
                    help="train the learned surrogate and compare surrogate ROMs with the exact one (JSON line)")
    ap.add_argument("--train-media", type=int, default=24)
    ap.add_argument("--train-iters", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--band", default=None, choices=["cell", "nyquist"],
                    help="band of the headline workload (default: one minimum wavelength per cell)")
    ap.add_argument("--modes", type=int, default=None, help="face modes of the headline workload (default 45)")
    ap.add_argument("--cellwl", type=float, default=None,
                    help="minimum wavelengths per cell of the headline workload's band (default 1)")
    ap.add_argument("--plain-fp32", action="store_true", help="headline FP32 without the factored last coefficient")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle's host timing")
    ap.add_argument("--ref-sample", type=int, default=10, help="time steps per bench step of --impl reference")
    ap.add_argument("--config", default=None, choices=["c3"],
                    help="c3: the 256^3 dipping-layer workload end to end (separate JSON line)")
    ap.add_argument("--c3-n", type=int, default=256)
    ap.add_argument("--c3-modes", type=int, default=15)
    ap.add_argument("--c3-rule", action="store_true",
                    help="--config c3: per-cell layer counts (3..6) by the library's layer-count rule")
    ap.add_argument("--c3-steps", type=int, default=6000)
    ap.add_argument("--c3-parity-steps", type=int, default=200)
    ap.add_argument("--accuracy", action="store_true",
                    help="ROM vs fine grid at equal receiver accuracy over face-mode counts (JSON line)")
    ap.add_argument("--acc-n", type=int, default=64, help="voxels per edge of --accuracy")
    ap.add_argument("--acc-modes", default="15,28,45", help="face-mode counts of --accuracy")
    ap.add_argument("--acc-steps", type=int, default=3000)
    ap.add_argument("--acc-src", type=int, default=8, help="sources of --accuracy")
    ap.add_argument("--acc-no-corners", action="store_true", help="--accuracy without the Appendix D correction")
    ap.add_argument("--acc-src-centre", action="store_true", help="--accuracy with sources at cell centres")
    ap.add_argument("--acc-shift", type=float, default=1.0, help="--accuracy shift as a multiple of -omega_max^2")
    ap.add_argument("--acc-cellwl", type=float, default=1.0, help="--accuracy: minimum wavelengths per cell (band cell)")
    ap.add_argument("--acc-m", type=int, default=4, help="S-fraction layers of --accuracy")
    ap.add_argument("--acc-band", default="cell", choices=["cell", "nyquist"],
                    help="band of --accuracy: one minimum wavelength per cell, or peak at 1/10 grid Nyquist")
    args = ap.parse_args()
    if args.config == "c3":
        run_c3(args)
        return
    if args.accuracy:
        run_accuracy(args)
        return
    if args.surrogate:
        run_surrogate(args)
        return
    if args.many_sources:
        run_many_sources(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
