"""Shared hand-built inputs for the oracle pins and the GPU parity tests."""
import itertools

import numpy as np

from paper_2609_24513_gb300 import synth

HAND = {
    "disjoint boxes": (synth.box((100, 100, 100), (110, 110, 110)),
                       synth.box((120, 100, 100), (130, 110, 110)), False),
    "face to face": (synth.box((100, 100, 100), (110, 110, 110)),
                     synth.box((110, 102, 103), (120, 108, 113)), False),
    "shared edge": (synth.box((100, 100, 100), (110, 110, 110)),
                    synth.box((110, 110, 100), (120, 120, 110)), False),
    "shared vertex": (synth.box((100, 100, 100), (110, 110, 110)),
                      synth.box((110, 110, 110), (120, 120, 120)), False),
    "interpenetrating boxes": (synth.box((100, 100, 100), (110, 110, 110)),
                               synth.box((105, 103, 96), (117, 108, 104)), True),
    "nested boxes": (synth.box((100, 100, 100), (130, 130, 130)),
                     synth.box((107, 111, 113), (117, 119, 121)), True),
    "nested boxes sharing a face": (synth.box((100, 100, 100), (120, 120, 120)),
                                    synth.box((100, 105, 105), (110, 115, 115)), True),
    "vertex on a face, outside": (synth.box((100, 100, 100), (120, 120, 120)),
                                  synth.tetra((110, 110, 120), (105, 105, 130),
                                              (118, 106, 131), (108, 117, 129)), False),
    "identical meshes": (synth.box((100, 100, 100), (110, 110, 110)),
                         synth.box((100, 100, 100), (110, 110, 110)), False),
}




def lattice_shapes():
    return {
        "cube": synth.box((0, 0, 0), (2, 2, 2)),
        "tetra": synth.tetra((0, 0, 0), (2, 0, 0), (0, 2, 0), (0, 0, 2)),
        "octa": synth.octahedron((1, 1, 1), 1),
    }


def lattice_case_sets():
    """Every ordered pair of the three unit shapes, B shifted by every offset in
    [-3, 3]^3.  Returns (A, B, candidates, labels)."""
    shapes = lattice_shapes()
    base = np.array([20, 20, 20])
    offs = list(itertools.product(range(-3, 4), repeat=3))
    names = list(shapes)
    meshes_a = [synth.translate(shapes[na], base) for na in names]
    meshes_b, cand, meta = [], [], []
    for na in names:
        for nb in names:
            for o in offs:
                meshes_b.append(synth.translate(shapes[nb], base + np.array(o)))
                cand.append((names.index(na), len(meshes_b) - 1))
                meta.append((na, nb, o))
    return (synth.concat(meshes_a), synth.concat(meshes_b),
            np.array(cand, dtype=np.int32), meta)


def sat_overlap(va, ta, vb, tb):
    """Exact: interiors of two convex polytopes intersect iff no candidate axis
    (face normals, edge x edge) weakly separates them."""
    def normals(v, t):
        a = v[t[:, 0]]
        return np.cross(v[t[:, 1]] - a, v[t[:, 2]] - a)

    def edges(v, t):
        e = np.concatenate([v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 1]], v[t[:, 0]] - v[t[:, 2]]])
        return e
    axes = [normals(va, ta), normals(vb, tb)]
    ea, eb = edges(va, ta), edges(vb, tb)
    axes.append(np.cross(ea[:, None, :], eb[None, :, :]).reshape(-1, 3))
    ax = np.concatenate(axes)
    ax = ax[np.any(ax != 0, axis=1)]
    pa, pb = va @ ax.T, vb @ ax.T
    sep = (pa.max(axis=0) <= pb.min(axis=0)) | (pb.max(axis=0) <= pa.min(axis=0))
    return not bool(sep.any())
