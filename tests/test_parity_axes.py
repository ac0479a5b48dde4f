"""Containment parity along any axis direction, checked on the CPU.

The paper casts the parity ray along +z (Alg. 2, Sec. 3.3); the oracle does
the same with a symbolic perturbation of the origin.  The GPU casts it along
whichever of the six axis directions leaves the target mesh's box soonest,
with the perturbation v + e u_hat + e^2 w_hat for the cyclic triple
(u, w, axis): a triangle counts when the perturbed origin lies strictly
inside its projection along the axis and the triangle's plane is met on the
ray's side.  For a closed surface and a point off it the parity is the
point's mod-2 winding number, whatever the direction.

These tests evaluate that per-direction rule with exact integers and check it
against the oracle's +z parity for every direction, on solids whose vertices,
edges and faces are aligned with the query points' coordinates (so that the
perturbation decides many projections) and on curved meshes.
"""
import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import synth

from cases import lattice_case_sets


def _o2(a, b, c):
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])


def _side_eps(a, b, v):
    """sign of orient2d(a, b, v + (e, e^2)) in the projected (u, w) plane."""
    o = _o2(a, b, np.broadcast_to(v, a.shape))
    first = np.where(a[:, 1] != b[:, 1], np.where(a[:, 1] > b[:, 1], 1, -1),
                     np.sign(b[:, 0] - a[:, 0]))
    return np.where(o != 0, np.sign(o), first)


def axis_parity(v, tri_xyz, ax, direction):
    """Parity of the perturbed ray from v along axis `ax`, sign `direction`,
    over triangles tri_xyz (T x 3 x 3 int64)."""
    u, w = (ax + 1) % 3, (ax + 2) % 3
    a, b, c = tri_xyz[:, 0], tri_xyz[:, 1], tri_xyz[:, 2]
    pa, pb, pc = a[:, [u, w]], b[:, [u, w]], c[:, [u, w]]
    pv = np.asarray(v, np.int64)[[u, w]]
    s2 = _o2(pa, pb, pc)
    s = np.sign(s2)
    inside = (_side_eps(pa, pb, pv) == s) & (_side_eps(pb, pc, pv) == s) & (_side_eps(pc, pa, pv) == s)
    d = np.asarray(v, np.int64) - a
    n = np.cross(b - a, c - a)
    o = (d * n).sum(axis=1)
    hit = (s2 != 0) & inside & (o != 0) & (np.sign(o) == -direction * s)
    return int(hit.sum()) & 1


def _mesh_tris(ds, k):
    v, t = ds.mesh(k)
    return v.astype(np.int64)[t]


def _query_points(rng, tris, n):
    """Points around the mesh: random ones, and ones built from the mesh's own
    vertex coordinates (+-1) so that projections pass exactly through
    vertices and along edges."""
    V = tris.reshape(-1, 3)
    lo, hi = V.min(axis=0) - 2, V.max(axis=0) + 2
    pts = [rng.integers(lo, hi + 1, size=(n, 3))]
    idx = rng.integers(0, len(V), size=(n, 3))
    aligned = np.stack([V[idx[:, k], k] for k in range(3)], axis=1)
    pts.append(aligned + rng.integers(-1, 2, size=(n, 3)) * (rng.random((n, 3)) < 0.3))
    return np.clip(np.concatenate(pts), 0, (1 << 18) - 1)


def _check_mesh(ds, k, rng, n):
    tris = _mesh_tris(ds, k)
    checked = 0
    for v in _query_points(rng, tris, n):
        ref, on = oracle.point_query([int(x) for x in v], ds, k)
        if on:
            continue
        for ax in range(3):
            for d in (1, -1):
                assert axis_parity(v, tris, ax, d) == int(ref), (k, v.tolist(), ax, d)
        checked += 1
    return checked


def test_axis_parity_on_aligned_solids():
    """Boxes, tetrahedra and octahedra of the exhaustive lattice cases."""
    rng = np.random.default_rng(8100)
    A, B, _, _ = lattice_case_sets()
    total = 0
    for ds in (A, B):
        for k in rng.choice(ds.nmesh, size=min(8, ds.nmesh), replace=False):
            total += _check_mesh(ds, int(k), rng, 60)
    assert total > 300


def test_axis_parity_on_boxes_sharing_planes():
    """Nested and adjacent boxes: many points share a face plane or an edge
    line with the query mesh."""
    rng = np.random.default_rng(8200)
    meshes = [synth.box((10, 10, 10), (30, 30, 30)), synth.box((0, 5, 10), (40, 25, 30)),
              synth.box((20, 20, 20), (21, 60, 21))]
    ds = synth.concat(meshes)
    total = sum(_check_mesh(ds, k, rng, 150) for k in range(ds.nmesh))
    assert total > 300


@pytest.mark.parametrize("seed", [1001])
def test_axis_parity_on_spheres(seed):
    rng = np.random.default_rng(8300)
    A, _ = synth.tiny_spheres(seed)
    total = sum(_check_mesh(A, k, rng, 25) for k in range(3))
    assert total > 100


def test_outside_the_box_parity_is_even():
    """The containment prefilter: a point outside a closed mesh's closed box
    has even parity (the ray leaves the box without meeting the surface an
    odd number of times), so the kernels skip its traversal."""
    rng = np.random.default_rng(8400)
    A, _ = synth.tiny_spheres(1002)
    for k in range(4):
        tris = _mesh_tris(A, k)
        V = tris.reshape(-1, 3)
        lo, hi = V.min(axis=0), V.max(axis=0)
        pts = rng.integers(lo - 50, hi + 51, size=(400, 3))
        out = ((pts < lo) | (pts > hi)).any(axis=1)
        for v in pts[out]:
            ref, on = oracle.point_query([int(x) for x in v], A, k)
            assert not on and not ref
            for ax in range(3):
                for d in (1, -1):
                    assert axis_parity(v, tris, ax, d) == 0
