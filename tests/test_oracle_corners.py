"""Exact pin of the oracle's ROM-level Appendix D correction (``online.corner_correct`` with the
S_f rows of ``online.corner_rows``).

Appendix D corrects the face unknowns of a corner-removed graph: every copy k_f of a corner-set
node k takes the mass-weighted mean sum_f (b_{k_f}/b_k) u_{k_f} of the copies.  At the fine level
(S_f = I) that step is ``fine.fine_leapfrog(..., groups=...)``, pinned exactly by
``test_oracle_rom.py::test_appendix_d_correction_exact_at_fine_level`` (it turns the corner-removed
leapfrog into the original one to rounding).  At the ROM level the face unknowns are u~_f, the
hanging values are read through the S_f rows (u^_l = s_l . u~_f) and the correction adds
s_l^T (mean - u^_l).  Since S_f^T S_f = I, that is exactly the fine-level step seen through the
face bases:

    corner_correct(u~)_f  =  S_f^T [ C_fine( lift(u~) ) ]|_f,   lift(u~)|_f = S_f u~_f,

for any orthonormal S_f.  The test checks this identity to rounding on a 2 x 2 cell partition in
2D (one corner node, four copies) and a 2 x 2 x 2 partition in 3D (edge lines with four copies, a
vertex with twelve), with S_f = I and with DCT bases of a few modes, C_fine taken from the
fine-level leapfrog itself (one step at tau = 0 applies only its correction).

Planted mistakes in the oracle's correction data (on the CPU) must fail it: the unweighted mean
in place of the b_{k_f}/b_k weights, weights that do not sum to one (b_k taken as half the node's
mass), and a group that skips one face.
"""
import numpy as np
import pytest

import synth
from oracle import fine, online, partition, rom


def _case(n3d: bool):
    if n3d:
        n, cell = (6, 6, 6), (3, 3, 3)
        g = synth.Grid(n=n, h=0.1, bc=(("D", "N"), ("D", "D"), ("D", "D")))
    else:
        n, cell = (8, 8), (4, 4)
        g = synth.Grid(n=n, h=0.1, bc=(("D", "D"), ("D", "D")))
    rng = np.random.default_rng(1604 + int(n3d))
    s, r = rng.uniform(0.5, 3.0, n), rng.uniform(0.5, 2.5, n)
    op = fine.FineOperator(g, s, r)
    return partition.Partition(op, s, r, cell)


def _fine_correction(part, v):
    """C_fine(v): the fine-level leapfrog's Appendix D step alone (tau = 0, u^0 = u^{-1} = v)."""
    Ap, Bp = part.modified_operator()
    N = Ap.shape[0]
    groups = [[(part.faces[f].nodes[rr], wt) for (f, rr, wt) in grp] for grp in part.corner_groups()]
    out = fine.fine_leapfrog(Ap, Bp, np.zeros((N, v.shape[1])), np.eye(N), np.zeros(2), 0.0, 2,
                             u0=v, um1=v, groups=groups)
    return out[1]


def _check(part, bases, tamper=None, seed=0):
    """Largest relative difference between corner_correct and the projected fine-level step."""
    rng = np.random.default_rng(seed)
    S = 3
    faces_u = [rng.standard_normal((b.shape[1], S)) for b in bases]
    N = part.modified_operator()[0].shape[0]
    v = np.zeros((N, S))
    for f in part.faces:
        v[np.asarray(f.nodes)] = bases[f.id] @ faces_u[f.id]
    ref = _fine_correction(part, v)
    corners = online.corner_rows(part.corner_groups(), bases)
    if tamper is not None:
        corners = tamper(corners)
    got = [x.copy() for x in faces_u]
    online.corner_correct(got, corners)
    err = 0.0
    for f in part.faces:
        want = bases[f.id].T @ ref[np.asarray(f.nodes)]
        err = max(err, float(np.linalg.norm(got[f.id] - want) / np.linalg.norm(want)))
    moved = max(float(np.linalg.norm(a - b)) for a, b in zip(got, faces_u))
    return err, moved


@pytest.mark.parametrize("n3d", [False, True])
@pytest.mark.parametrize("modes", [None, 2, 4])
def test_rom_corner_correction_is_fine_step_through_face_bases(n3d, modes):
    part = _case(n3d)
    groups = part.corner_groups()
    assert len(groups) >= 1
    if n3d:
        assert sorted({len(gr) for gr in groups}) == [4, 12]   # edge lines and the vertex
    if modes is None:
        bases = [np.eye(len(f.nodes)) for f in part.faces]
    else:
        bases = [rom.face_basis(f, modes) for f in part.faces]
    err, moved = _check(part, bases)
    assert err <= 1e-12
    assert moved > 1e-3          # the correction did something on these random states


def _unweighted(corners):
    return [[(f, s, 1.0 / len(gr)) for (f, s, _) in gr] for gr in corners]


def _unnormalised(corners):
    return [[(f, s, 2.0 * wt) for (f, s, wt) in gr] for gr in corners]


def _skip_one_face(corners):
    out = []
    for gr in corners:
        wsum = sum(wt for (_, _, wt) in gr[1:])
        out.append([(f, s, wt / wsum) for (f, s, wt) in gr[1:]])
    return out


@pytest.mark.parametrize("n3d", [False, True])
@pytest.mark.parametrize("plant", [_unweighted, _unnormalised, _skip_one_face])
def test_planted_corner_mistakes_fail(n3d, plant):
    part = _case(n3d)
    bases = [rom.face_basis(f, 3) for f in part.faces]
    err, _ = _check(part, bases, tamper=plant)
    assert err > 1e-6


def test_planted_sequential_correction_fails(monkeypatch):
    """All corrections of a level are taken from its uncorrected values (reading R13); a variant
    that applies the groups one after another, each reading values already corrected by the
    groups before it, breaks the identity wherever groups share a face and S_f != I."""

    def sequential(faces_u, corners):
        for grp in corners:
            uh = [s @ faces_u[f] for (f, s, _) in grp]
            mean = sum(wt * x for (_, _, wt), x in zip(grp, uh))
            for (f, s, _), x in zip(grp, uh):
                faces_u[f] += np.outer(s, mean - x)

    part = _case(True)
    bases = [rom.face_basis(f, 3) for f in part.faces]
    assert _check(part, bases)[0] <= 1e-12
    monkeypatch.setattr(online, "corner_correct", sequential)
    assert _check(part, bases)[0] > 1e-6
