"""CPU pin: the strict crossing of a segment and a triangle (Sec. 3.2, read
strictly: the open segment crosses the open triangle transversally) implies
that their boxes overlap in the open sense on every axis, so the streaming
kernel's crossing traversal may prune with strict box tests.

Argument: if on some axis the segment's interval and the triangle's only
touch at a value c (one's maximum is the other's minimum), a common point
has that coordinate c; the open segment and the open triangle reach c at a
relative-interior point, where a linear function is extreme only if it is
constant, so both lie in the plane at c -- coplanar, which the strict test
rejects.  Node boxes contain the boxes below them, so the same holds for
node pairs.  This test checks the implication with the oracle's own strict
predicate on configurations full of exact contacts (hand-built solids,
lattice placements of unit solids, urban buildings sharing walls, edges and
corners), and that the open test does prune pairs the closed test keeps.
"""
import numpy as np

import oracle
from cases import HAND, lattice_case_sets
from paper_2609_24513_gb300 import synth


def _edges_and_tris(ds, k):
    v, t = ds.mesh(k)
    v = np.asarray(v, np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return v, e, np.asarray(t)


def _check_pair(dsA, i, dsB, j):
    """(crossings found, closed-overlap pairs, of those pruned by the open test)"""
    va, ea, ta = _edges_and_tris(dsA, i)
    vb, eb, tb = _edges_and_tris(dsB, j)
    found = closed = pruned = 0
    for (v_s, e_s, v_t, t_t) in ((va, ea, vb, tb), (vb, eb, va, ta)):
        slo = np.minimum(v_s[e_s[:, 0]], v_s[e_s[:, 1]])
        shi = np.maximum(v_s[e_s[:, 0]], v_s[e_s[:, 1]])
        tlo = np.minimum(np.minimum(v_t[t_t[:, 0]], v_t[t_t[:, 1]]), v_t[t_t[:, 2]])
        thi = np.maximum(np.maximum(v_t[t_t[:, 0]], v_t[t_t[:, 1]]), v_t[t_t[:, 2]])
        cl = np.all((slo[:, None, :] <= thi[None]) & (tlo[None] <= shi[:, None, :]), axis=2)
        op = np.all((slo[:, None, :] < thi[None]) & (tlo[None] < shi[:, None, :]), axis=2)
        closed += int(cl.sum())
        pruned += int((cl & ~op).sum())
        for a, b in zip(*np.nonzero(cl)):
            p, q = v_s[e_s[a, 0]], v_s[e_s[a, 1]]
            x, y, z = v_t[t_t[b, 0]], v_t[t_t[b, 1]], v_t[t_t[b, 2]]
            if oracle.segtri_strict(p, q, x, y, z):
                found += 1
                assert op[a, b], "a strict crossing with boxes that only touch"
    return found, closed, pruned


def test_hand_built_contacts():
    total_pruned = 0
    for name, (ma, mb, _) in HAND.items():
        A, B = synth.concat([ma]), synth.concat([mb])
        _, _, pr = _check_pair(A, 0, B, 0)
        total_pruned += pr
    assert total_pruned > 0


def test_lattice_placements():
    A, B, cand, _ = lattice_case_sets()
    found = pruned = 0
    for i, j in cand[::3]:
        f, _, pr = _check_pair(A, int(i), B, int(j))
        found += f
        pruned += pr
    assert found > 0 and pruned > 0


def test_urban_touching_buildings():
    U = synth.urban(5001, n_buildings=300, n_parts=30)
    cand = oracle.mbb_candidates(U, U, self_join=True)
    found = pruned = 0
    for i, j in cand[:50]:
        f, _, pr = _check_pair(U, int(i), U, int(j))
        found += f
        pruned += pr
    assert found > 0 and pruned > 0
