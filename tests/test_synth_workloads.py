"""Generators of the batching and urban workloads: closed meshes, the face
counts and shapes they promise, and (with the oracle) the intended mix of
pair classes."""
import collections

import numpy as np

import oracle
from paper_2609_24513_gb300 import synth


def test_latlong_sphere_counts_and_closure():
    rng = np.random.default_rng(0)
    for F in (200, 1000, 5000):
        v, t = synth.latlong_sphere(F, 0.02, np.full(3, 0.5), rng)
        ds = synth.concat([(v, t)])
        assert oracle.is_closed_manifold(ds, 0)
        assert 0.7 * F < len(t) < 1.3 * F


def test_batching_workload():
    A, B, cand, off, cls = synth.batching(3001, n_pairs=300, n_templates=60)
    for ds in (A, B):
        f = np.diff(ds.toff)
        assert f.min() >= 150 and f.max() <= 60000
        assert all(oracle.is_closed_manifold(ds, k) for k in range(ds.nmesh))
    # translated meshes stay on the grid
    for (i, j), o in zip(cand, off):
        v, _ = B.mesh(int(j))
        assert np.all(v.min(axis=0) + o >= 0) and np.all(v.max(axis=0) + o <= synth.QMAX)
    flags = oracle.join(A, B, cand, tier=2, offsets=off)
    assert flags[cls == 1].all()                 # containment pairs intersect
    assert flags[cls == 2].mean() < 0.05          # box-corner placements rarely touch
    assert 0.5 < flags[cls == 0].mean() <= 1.0    # most crossing placements cross
    assert 0.2 < flags.mean() < 0.5


def test_urban_workload():
    U = synth.urban(5001, n_buildings=400, n_parts=40)
    assert all(oracle.is_closed_manifold(U, k) for k in range(U.nmesh))
    tags = collections.Counter(U.meta["tags"])
    assert tags["building"] > 300 and tags["box"] + tags["cylinder"] == 40
    assert tags["shared_wall"] + tags["shared_edge"] > 0
    cand = oracle.mbb_candidates(U, U, self_join=True)
    flags = oracle.join(U, U, cand, tier=2)
    t = U.meta["tags"]
    # buildings sharing a wall plane or an edge touch but never intersect
    for (i, j), f in zip(cand, flags):
        if t[i] == t[j] and t[i] in ("shared_wall", "shared_edge") and abs(int(i) - int(j)) == 1:
            assert not f
    assert 0 < flags.sum() < len(cand)


def test_tiers_agree_on_workload_samples():
    """Oracle self-consistency (pure brute force against the box-pruned tier)
    on seeded samples of the batching pairs (with their translations) and of
    the urban self join's candidates, including its exactly touching walls.
    The pathology meshes (5k-50k triangles) make a brute-force pair cost
    seconds, so that workload is checked through tier 2 only."""
    rng = np.random.default_rng(3)
    A, B, cand, off, cls = synth.batching(3002, n_pairs=400, n_templates=60)
    fa, fb = np.diff(A.toff), np.diff(B.toff)
    small = np.nonzero((fa[cand[:, 0]] < 1500) & (fb[cand[:, 1]] < 1500))[0]
    pick = rng.choice(small, size=min(60, len(small)), replace=False)
    f1 = oracle.join(A, B, cand[pick], tier=1, offsets=off[pick])
    f2 = oracle.join(A, B, cand[pick], tier=2, offsets=off[pick])
    assert (f1 == f2).all() and 0 < f1.sum() < len(pick)
    U = synth.urban(5002, n_buildings=120, n_parts=12)
    uc = oracle.mbb_candidates(U, U, self_join=True)
    fu = np.diff(U.toff)
    light = np.nonzero((fu[uc[:, 0]] < 800) & (fu[uc[:, 1]] < 800))[0]
    pick = rng.choice(light, size=min(80, len(light)), replace=False)
    g1 = oracle.join(U, U, uc[pick], tier=1)
    g2 = oracle.join(U, U, uc[pick], tier=2)
    assert (g1 == g2).all()
