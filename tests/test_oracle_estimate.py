"""Pins of the selectivity-estimate oracle (paper Sec. 3.5).

The estimator is a heuristic, so the pins fix what is exact around it: mesh
volumes (exact box volumes, a library convex hull, the closed form of an
extruded prism with a pyramid roof), the per-cell object counts (brute force
over the cells), the capped regime where every cell's probability is 1 (the
estimate is then the brute-force count of co-occupying object pairs), the
identities the formula implies (symmetry, doubling, translation) and the
estimate's intent: for uniformly placed cubes it approximates the number of
box-overlapping pairs.
"""
import numpy as np
import pytest

import oracle
from oracle import estimate as est
from paper_2609_24513_gb300 import synth


def _cubes(rng, n, side, lo=20000, hi=240000):
    out = []
    for _ in range(n):
        c = rng.integers(lo, hi - side, size=3)
        out.append(synth.box(tuple(c), tuple(c + side)))
    return synth.concat(out)


def test_mesh_volume_of_boxes_is_exact():
    rng = np.random.default_rng(9000)
    for _ in range(50):
        lo = rng.integers(0, 200000, size=3)
        ext = rng.integers(1, 50000, size=3)
        v, t = synth.box(tuple(lo), tuple(lo + ext))
        assert est.mesh_volume(v, t) == float(np.prod(ext))


def test_mesh_volume_matches_convex_hull():
    spatial = pytest.importorskip("scipy.spatial")
    A, _ = synth.tiny_spheres(1001)
    for k in range(A.nmesh):
        v, t = A.mesh(k)
        hull = spatial.ConvexHull(np.asarray(v, np.float64)).volume
        assert abs(est.mesh_volume(v, t) - hull) <= 1e-9 * hull


def test_mesh_volume_of_a_non_convex_building():
    """Prism over a star-shaped footprint plus a pyramid roof over its centre:
    volume = footprint area x (height + roof / 3)."""
    rng = np.random.default_rng(9100)
    for _ in range(20):
        n = int(rng.integers(6, 40))
        th = np.sort(2 * np.pi * (np.arange(n) + rng.uniform(-0.3, 0.3, size=n)) / n)
        rr = rng.uniform(300, 1000, size=n)
        fp = np.rint(np.stack([rr * np.cos(th), rr * np.sin(th)], 1) + 5000)
        fp[:, :] = fp - np.rint(fp.mean(axis=0)) + 5000     # centre on an integer point
        height, roof, bands = int(rng.integers(100, 3000)), int(rng.integers(10, 500)), 3
        v, t = synth.building(fp, 1000, height, roof, bands)
        x, y = fp[:, 0], fp[:, 1]
        area = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
        assert abs(est.mesh_volume(v, t) - area * (height + roof / 3.0)) <= 1e-6 * area * height


def test_cell_counts_match_brute_force():
    rng = np.random.default_rng(9200)
    A = _cubes(rng, 60, 9000)
    B = _cubes(rng, 40, 23000)
    G = 5
    sa, sb = est.object_stats(A), est.object_stats(B)
    g0, cw = est.grid_of(sa, sb, G)
    N, S, R = est.cell_stats(sa, g0, cw, G)
    lo, hi, side, ratio = sa
    for i in range(G):
        for j in range(G):
            for k in range(G):
                clo = g0 + cw * np.array([i, j, k])
                chi = clo + cw
                touch = np.all((lo <= chi) & (hi >= clo), axis=1)
                assert N[i, j, k] == touch.sum()
                assert np.isclose(S[i, j, k], side[touch].sum())
                assert np.isclose(R[i, j, k], ratio[touch].sum())
    assert np.allclose(ratio, 1.0)                      # boxes fill their boxes


def test_capped_regime_counts_co_occupying_pairs():
    """Objects much larger than the cells: every occupied cell has P = 1, so the
    estimate is the sum over cells of N_1 N_2, counted here by brute force."""
    rng = np.random.default_rng(9300)
    A = _cubes(rng, 12, 60000)
    B = _cubes(rng, 9, 80000)
    G = 8
    E, cells, slots = est.estimate(A, B, G=G)
    sa, sb = est.object_stats(A), est.object_stats(B)
    g0, cw = est.grid_of(sa, sb, G)
    total = 0
    for idx in np.ndindex(G, G, G):
        clo = g0 + cw * np.array(idx)
        chi = clo + cw
        na = np.all((sa[0] <= chi) & (sa[1] >= clo), axis=1).sum()
        nb = np.all((sb[0] <= chi) & (sb[1] >= clo), axis=1).sum()
        total += na * nb
    assert E == pytest.approx(total) and slots == pytest.approx(2 * total)


def test_identities():
    rng = np.random.default_rng(9400)
    A, B = synth.tiny_spheres(1002)
    E, _, _ = est.estimate(A, B, G=6)
    assert E > 0
    assert est.estimate(B, A, G=6)[0] == pytest.approx(E)           # symmetric
    AA = synth.concat([A.mesh(k) for k in range(A.nmesh)] * 2)      # every object twice
    assert est.estimate(AA, B, G=6)[0] == pytest.approx(2 * E)
    d = np.array([1234, -567, 890], np.float32)                      # translation
    At = synth.concat([(v + d, t) for v, t in (A.mesh(k) for k in range(A.nmesh))])
    Bt = synth.concat([(v + d, t) for v, t in (B.mesh(k) for k in range(B.nmesh))])
    assert est.estimate(At, Bt, G=6)[0] == pytest.approx(E, rel=1e-9)
    # one coarse cell keeps P below its cap: sparser objects (volume ratio
    # < 1) weigh less with a larger gamma, and the eps bias only adds
    E1 = est.estimate(A, B, G=1)[0]
    assert 0 < E1 < A.nmesh * B.nmesh
    assert est.estimate(A, B, G=1, gamma=2.0)[0] < E1
    assert est.estimate(A, B, G=1, eps=0.0)[0] < E1


def test_estimate_approximates_box_overlaps_of_uniform_cubes():
    """Equal cubes placed uniformly, one cell: the estimate is the number of
    pairs whose boxes overlap if centres were uniform in a periodic cell, so
    it should land near the brute-force count (boundary effects and the eps
    bias keep it within about 20 %)."""
    rng = np.random.default_rng(9500)
    A = _cubes(rng, 400, 20000)
    B = _cubes(rng, 400, 30000)
    E, _, _ = est.estimate(A, B, G=1)
    K = len(oracle.mbb_candidates(A, B))
    assert K > 1000
    assert 0.8 < E / K < 1.25
