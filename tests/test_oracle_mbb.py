"""Pin of the oracle's bounding-box filter join (``oracle.mbb_candidates``,
the filter step of Sec. 3.1 that yields the candidate pairs the refinement
tests).

The reference here is independent of the C code: each mesh's closed box is
taken from its own vertex rows with Python integers, and every (i, j) is
tested by brute force with ``lo <= hi`` comparisons on all three axes.  The
hand-built cases fix the expected answers by reasoning: boxes that touch on a
face, an edge or a single corner meet (closed boxes), boxes one grid unit
apart do not; a self join lists i < j only and never (i, i).  Meshes of
different vertex counts and datasets of different sizes make a wrong offset
or a swapped loop bound visible.
"""
import numpy as np
import pytest

import oracle
from paper_2609_24513_gb300 import synth


def _boxes(ds):
    out = []
    for k in range(ds.nmesh):
        rows = ds.xyz[int(ds.voff[k]):int(ds.voff[k + 1])].tolist()
        lo = [min(int(r[d]) for r in rows) for d in range(3)]
        hi = [max(int(r[d]) for r in rows) for d in range(3)]
        out.append((lo, hi))
    return out


def _brute(dsA, dsB, self_join=False):
    ba, bb = _boxes(dsA), _boxes(dsB)
    pairs = []
    for i, (alo, ahi) in enumerate(ba):
        for j, (blo, bhi) in enumerate(bb):
            if self_join and j <= i:
                continue
            if all(alo[d] <= bhi[d] and blo[d] <= ahi[d] for d in range(3)):
                pairs.append((i, j))
    return np.array(pairs, dtype=np.int32).reshape(-1, 2)


def _cube(lo, hi):
    return synth.box(lo, hi)


# B meshes placed around the A cube [100, 200]^3, with the expected verdict
AROUND = [
    ("face", (200, 120, 120), (300, 180, 180), True),
    ("face_low", (0, 120, 120), (100, 180, 180), True),
    ("edge", (200, 200, 120), (300, 300, 180), True),
    ("corner", (200, 200, 200), (300, 300, 300), True),
    ("corner_low", (0, 0, 0), (100, 100, 100), True),
    ("gap_x", (201, 120, 120), (300, 180, 180), False),
    ("gap_low_z", (120, 120, 0), (180, 180, 99), False),
    ("gap_edge", (201, 201, 120), (300, 300, 180), False),
    ("gap_corner", (201, 200, 200), (300, 300, 300), False),
    ("overlap_1", (199, 120, 120), (300, 180, 180), True),
    ("contains", (50, 50, 50), (250, 250, 250), True),
    ("inside", (120, 130, 140), (150, 160, 170), True),
    ("flat_touch", (120, 120, 200), (180, 180, 260), True),
    ("far", (1000, 1000, 1000), (1100, 1100, 1100), False),
]


def test_touching_boxes_meet_and_separated_ones_do_not():
    A = synth.concat([_cube((100, 100, 100), (200, 200, 200))])
    B = synth.concat([_cube(lo, hi) for _, lo, hi, _ in AROUND])
    got = oracle.mbb_candidates(A, B)
    want = np.array([(0, j) for j, c in enumerate(AROUND) if c[3]], np.int32)
    assert np.array_equal(got, want), [AROUND[j][0] for j in got[:, 1]]
    assert np.array_equal(got, _brute(A, B))
    # swapping the datasets transposes the pairs
    back = oracle.mbb_candidates(B, A)
    assert np.array_equal(back, want[:, ::-1])


def test_self_join_lists_each_unordered_pair_once():
    # a row of cubes that touch their neighbours on a face, plus one cube
    # identical to the first and one isolated cube
    row = [_cube((100 * k, 0, 0), (100 * k + 100, 100, 100)) for k in range(4)]
    ds = synth.concat(row + [_cube((0, 0, 0), (100, 100, 100)),
                             _cube((1000, 1000, 1000), (1050, 1050, 1050))])
    got = oracle.mbb_candidates(ds, ds, self_join=True)
    want = np.array([(0, 1), (0, 4), (1, 2), (1, 4), (2, 3)], np.int32)
    assert np.array_equal(got, want)
    assert np.array_equal(got, _brute(ds, ds, self_join=True))
    # without the self-join rule every ordered pair appears, (i, i) included
    full = oracle.mbb_candidates(ds, ds)
    assert np.array_equal(full, _brute(ds, ds))
    assert {(i, i) for i in range(6)} <= {tuple(p) for p in full.tolist()}
    assert len(full) == 2 * len(want) + 6


def _random_solids(rng, n, step):
    """Boxes, tetrahedra and octahedra (different vertex counts) whose
    coordinates are multiples of `step`, so that exact contacts are common."""
    meshes = []
    for _ in range(n):
        kind = rng.integers(3)
        c = rng.integers(3, 14, size=3) * step  # every corner stays >= 0
        r = int(rng.integers(1, 3)) * step
        if kind == 0:
            lo = c - rng.integers(0, 3, size=3) * step
            meshes.append(_cube(lo, lo + rng.integers(1, 4, size=3) * step))
        elif kind == 1:
            meshes.append(synth.octahedron(c, r))
        else:
            for _ in range(100):  # redraw all four corners until the volume is nonzero
                p = [c + rng.integers(-2, 3, size=3) * step for _ in range(4)]
                if abs(np.linalg.det(np.array([p[1] - p[0], p[2] - p[0], p[3] - p[0]], float))) >= 1:
                    break
            else:
                raise AssertionError("no tetrahedron of nonzero volume drawn")
            meshes.append(synth.tetra(*p))
    return synth.concat(meshes)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_solids_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    A = _random_solids(rng, 37, 1000)
    B = _random_solids(rng, 23, 1000)
    got = oracle.mbb_candidates(A, B)
    assert np.array_equal(got, _brute(A, B))
    assert 0 < len(got) < 37 * 23
    s = oracle.mbb_candidates(A, A, self_join=True)
    assert np.array_equal(s, _brute(A, A, self_join=True))
    assert np.all(s[:, 0] < s[:, 1])
