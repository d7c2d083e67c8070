"""Host logic of the bench's oracle timing (CPU): the ROM shape it times must be the workload's.

The reference arm times the oracle's ROM leapfrog on a box topology with the workload's I/O face
sizes (``bench._box_io``) and random SPD values; the native line's CPU baseline times it on the
library ROM's own coefficients (``bench._exported_rom``).  Both are checked against the oracle's
own partition and ROM of a small layered workload, and the I/O entries the timing uses sit on
one-sided faces.
"""
import numpy as np

import bench
import synth
from oracle import fine, partition, rom


def _case():
    wl = synth.workload_3d_layers(32, 16, m=3, n_modes=4, n_src=4, n_steps=10, band="cell")
    op = fine.FineOperator(wl.grid, wl.sigma, wl.rho)
    io = [tuple(int(x) for x in p) for p in list(wl.src_nodes) + list(wl.rcv_nodes)]
    part = partition.Partition(op, wl.sigma, wl.rho, wl.cell, io_nodes=io)
    return wl, part


def test_box_io_matches_the_partitions_io_faces():
    wl, part = _case()
    io_sizes = sorted(len(f.nodes) for f in part.faces if f.kind == "io")
    assert sorted(n for _, n in bench._box_io(wl)) == io_sizes
    nc = tuple(wl.grid.n[a] // wl.cell[a] for a in range(3))
    topo = synth.box_topology(nc, modes=wl.n_modes, m=wl.m, io_cells=bench._box_io(wl), seed=1)
    # interior faces carry the workload's mode count, I/O faces their node counts
    ref = rom.build_rom(part, wl.m, wl.n_modes, -1.0e3).topology
    assert sorted(int(k) for k in topo.cell_K()) == sorted(int(k) for k in ref.cell_K())


def test_io_entries_sit_on_one_sided_faces():
    topo = synth.box_topology((2, 2, 2), modes=3, m=2, io_cells=[(0, 2), (5, 3)], seed=3)
    src, rcv = bench._io_entries(topo, 5, 4)
    assert {j for _, j, _ in src} == set(range(5)) and {j for _, j, _ in rcv} == set(range(4))
    for f, _, v in src + rcv:
        assert len(topo.face_cells[f]) == 1 and len(v) == topo.face_M[f]
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12


def test_exported_rom_round_trips_the_coefficients():
    import paper_1604_06750_gb300 as P
    from paper_1604_06750_gb300 import build
    build.build()
    P.lib()
    topo = synth.box_topology((2, 2, 1), modes=3, m=[1, 2, 3, 2], io_cells=[(1, 2)], seed=4, ragged_modes=True)
    co = synth.random_coefficients(topo, seed=4)
    R = P.Rom.import_(topo, co)
    t2, c2 = bench._exported_rom(R)
    assert [list(x) for x in t2.cell_faces] == [list(x) for x in topo.cell_faces]
    assert list(t2.face_M) == list(topo.face_M) and list(t2.cell_m) == list(topo.cell_m)
    assert [sorted(x) for x in t2.face_cells] == [sorted(x) for x in topo.face_cells]
    for i in range(topo.n_cells):
        for k in range(int(topo.cell_m[i])):
            assert np.array_equal(c2.gamma[i][k], co.gamma[i][k])
            assert np.array_equal(c2.gamma_hat[i][k], co.gamma_hat[i][k])
    for f in range(topo.n_faces):
        assert np.array_equal(c2.face_mass[f], co.face_mass[f])
