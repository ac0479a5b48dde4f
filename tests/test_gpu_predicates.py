"""GPU parity of the paper's other join predicates (pj_join_opts.predicate):
overlap, contains and within (Sec. 3.2-3.3, Alg. 2) and the any-vertex
completeness mode, against ``oracle.join(..., predicate=...)`` on every
candidate: hand-built solids (both roles), exhaustive lattice placements,
nested spheres, instanced pairs with translations, and a shard of the full
pathology workload.  Every front end (streaming, breadth-first, per-warp,
one launch per pair), the exact leaves and graph replay are covered.
Results are pair sets, compared exactly.
"""
import numpy as np
import pytest

import oracle
from cases import HAND, lattice_case_sets
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu

PREDS = ("intersects", "overlap", "contains", "within", "any_vertex")
MODES = {
    "stream": dict(wave_levels=pierce.PJ_FRONT_STREAM),
    "stream_graph": dict(wave_levels=pierce.PJ_FRONT_STREAM, use_graph=True),
    "stream_exact": dict(wave_levels=pierce.PJ_FRONT_STREAM, leaf_mode=pierce.PJ_LEAF_EXACT),
    "wave": dict(wave_levels=9),
    "warps": dict(wave_levels=pierce.PJ_FRONT_NONE, warps_per_pair=2),
    "per_pair": dict(launch_mode=pierce.PJ_LAUNCH_PER_PAIR),
}


@pytest.fixture(scope="module")
def ctx():
    c = pierce.Context(0)
    yield c
    c.close()


def _flags(ctx, ha, hb, cand, pred, off=None, **kw):
    res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, cand=cand, cand_offsets=off,
                                       keep_flags=True, out_host=True, predicate=pred, **kw)
    flags = pierce.device_to_numpy(res.flags, int(res.n_candidates), np.uint8)
    pairs = pierce.pairs_to_numpy(res)
    pierce.pj_free_pairs(ctx.h, res)
    return flags, pairs


def _load(ctx, ds, W=4, L=4):
    h = ctx.load(ds)
    ctx.build(h, W, L)
    return h


@pytest.mark.parametrize("mode", sorted(MODES))
def test_hand_built_solids_every_predicate(ctx, mode):
    for name, (ma, mb, _) in sorted(HAND.items()):
        for A, B in ((synth.concat([ma]), synth.concat([mb])),
                     (synth.concat([mb]), synth.concat([ma]))):
            ha, hb = _load(ctx, A), _load(ctx, B)
            one = np.zeros((1, 2), np.int32)
            for p in PREDS:
                exp = oracle.join(A, B, one, predicate=p)
                got, pairs = _flags(ctx, ha, hb, one, p, **MODES[mode])
                assert np.array_equal(got, exp), (name, p, mode)
                assert np.array_equal(pairs, one[exp.astype(bool)])
            pierce.pj_free_dataset(ctx.h, ha)
            pierce.pj_free_dataset(ctx.h, hb)


def test_lattice_placements_every_predicate(ctx):
    A, B, cand, _ = lattice_case_sets()
    ha, hb = _load(ctx, A, 4, 2), _load(ctx, B, 4, 2)
    exp = {p: oracle.join(A, B, cand, predicate=p) for p in PREDS}
    # the any-vertex mode recovers contacts the strict rule misses
    assert exp["any_vertex"].sum() > exp["intersects"].sum()
    for mode in ("stream", "wave", "warps"):
        for p in PREDS:
            got, _ = _flags(ctx, ha, hb, cand, p, width=4, leaf_size=2, **MODES[mode])
            assert np.array_equal(got, exp[p]), (p, mode)


def test_nested_spheres_contain_and_within(ctx):
    # a large sphere holding a small one, a crossing pair and a disjoint pair
    big = synth._placed_sphere(3, np.array([0.5, 0.5, 0.5]), 0.2, np.eye(3))
    small = synth._placed_sphere(2, np.array([0.52, 0.48, 0.5]), 0.05, np.eye(3))
    cross = synth._placed_sphere(2, np.array([0.69, 0.5, 0.5]), 0.05, np.eye(3))
    far = synth._placed_sphere(2, np.array([0.9, 0.9, 0.9]), 0.05, np.eye(3))
    A = synth.concat([big, small])
    B = synth.concat([small, cross, far, big])
    cand = np.array([(i, j) for i in range(2) for j in range(4)], np.int32)
    ha, hb = _load(ctx, A), _load(ctx, B)
    for p in PREDS:
        exp = oracle.join(A, B, cand, predicate=p)
        for mode in ("stream", "stream_graph", "warps"):
            got, _ = _flags(ctx, ha, hb, cand, p, **MODES[mode])
            assert np.array_equal(got, exp), (p, mode)
    c = oracle.join(A, B, cand, predicate="contains")
    w = oracle.join(A, B, cand, predicate="within")
    assert c[0] == 1 and w[7] == 1           # big holds small; small within big


@pytest.mark.parametrize("W,L", [(4, 4), (8, 2), (2, 1)])
def test_tiny_spheres_every_predicate(ctx, W, L):
    for seed in (1001, 1002):
        A, B = synth.tiny_spheres(seed)
        cand = oracle.mbb_candidates(A, B)
        ha, hb = _load(ctx, A, W, L), _load(ctx, B, W, L)
        for p in PREDS:
            exp = oracle.join(A, B, cand, predicate=p)
            for mode in ("stream", "stream_exact", "warps"):
                got, pairs = _flags(ctx, ha, hb, cand, p, width=W, leaf_size=L, **MODES[mode])
                assert np.array_equal(got, exp), (seed, p, mode)
                assert np.array_equal(pairs, cand[exp.astype(bool)])


def test_instanced_pairs_with_translations(ctx):
    A, B, cand, off, _ = synth.batching(3001, n_pairs=1200, n_templates=120)
    ha, hb = _load(ctx, A), _load(ctx, B)
    for p in ("overlap", "contains", "within"):
        exp = oracle.join(A, B, cand, offsets=off, predicate=p, threads=None)
        for mode in ("stream_graph", "wave"):
            got, _ = _flags(ctx, ha, hb, cand, p, off=off, **MODES[mode])
            assert np.array_equal(got, exp), (p, mode)
    assert oracle.join(A, B, cand, offsets=off, predicate="contains", threads=None).sum() > 0


def test_pathology_shard_every_predicate_but_any_vertex(ctx, pathology_truth):
    A, B, cand, inter = pathology_truth
    rng = np.random.default_rng(17)
    # every intersecting candidate and as many others, in candidate order
    pick = np.sort(np.concatenate([np.flatnonzero(inter),
                                   rng.choice(np.flatnonzero(inter == 0), 20000, replace=False)]))
    shard = np.ascontiguousarray(cand[pick])
    ha, hb = _load(ctx, A, 4, 2), _load(ctx, B, 4, 2)
    for p in ("overlap", "contains", "within"):
        exp = oracle.join(A, B, shard, predicate=p, threads=None)
        got, _ = _flags(ctx, ha, hb, shard, p, width=4, leaf_size=2, use_graph=True)
        assert np.array_equal(got, exp), p
    got, _ = _flags(ctx, ha, hb, shard, "intersects", width=4, leaf_size=2)
    assert np.array_equal(got, inter[pick])
