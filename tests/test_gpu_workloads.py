"""GPU parity on the batching workload (instanced candidate pairs of very
uneven size) and the urban precision-stress self join (shared walls, edges
and corners; FP32 filter against all-int64 leaves).  At full size the oracle
refines every candidate (sharded over the host cores), so the whole pair set
is compared."""
import numpy as np
import pytest

import oracle
from conftest import oracle_flags
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = pierce.Context(0)
    yield c
    c.close()


def _join_flags(ctx, ha, hb, cand, off=None, **kw):
    res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, cand=cand, cand_offsets=off,
                                       keep_flags=True, out_host=True, **kw)
    flags = pierce.device_to_numpy(res.flags, int(res.n_candidates), np.uint8)
    pairs = pierce.pairs_to_numpy(res)
    pierce.pj_free_pairs(ctx.h, res)
    return flags, pairs


def test_batching_small_all_pairs(ctx):
    A, B, cand, off, cls = synth.batching(3001, n_pairs=1500, n_templates=150)
    exp = oracle.join(A, B, cand, tier=2, offsets=off)
    ha, hb = ctx.load(A), ctx.load(B)
    for W, L in ((4, 4), (8, 2)):
        ctx.build(ha, W, L)
        ctx.build(hb, W, L)
        for kw in (dict(use_graph=True), dict(launch_mode=pierce.PJ_LAUNCH_PER_PAIR),
                   dict(leaf_mode=pierce.PJ_LEAF_EXACT, wave_levels=-1, warps_per_pair=2),
                   dict(wave_levels=pierce.PJ_FRONT_STREAM, use_graph=True)):
            flags, _ = _join_flags(ctx, ha, hb, cand, off, width=W, leaf_size=L, **kw)
            assert np.array_equal(flags, exp), (W, L, kw)


def test_batching_full_size_all_pairs(ctx):
    A, B, cand, off, cls = synth.batching(3001)
    exp = oracle_flags("batching 100,000 instanced pairs", A, B, cand, offsets=off)
    ha, hb = ctx.load(A), ctx.load(B)
    ctx.build(ha, 4, 4)
    ctx.build(hb, 4, 4)
    flags, pairs = _join_flags(ctx, ha, hb, cand, off, use_graph=True)
    assert len(flags) == 100000
    assert 0.2 < exp.mean() < 0.5
    assert np.array_equal(flags, exp)               # every candidate
    assert np.array_equal(pairs, cand[exp.astype(bool)])
    again, _ = _join_flags(ctx, ha, hb, cand, off, use_graph=True)   # graph replay
    assert np.array_equal(again, exp)


def test_urban_small_self_join(ctx):
    U = synth.urban(5001, n_buildings=2000, n_parts=200)
    exp = oracle.join_all(U, U, self_join=True)
    h = ctx.load(U)
    ctx.build(h, 4, 4)
    ctx.reset_counters()
    got, _ = ctx.join(h, h, self_join=True)
    assert np.array_equal(got, exp)
    assert ctx.counters()["exact_fallbacks"] > 0      # near-degenerate contacts reach int64
    got_exact, _ = ctx.join(h, h, self_join=True, leaf_mode=pierce.PJ_LEAF_EXACT)
    assert np.array_equal(got_exact, exp)


def test_urban_full_size(ctx):
    U = synth.urban(5001)
    cand = oracle.mbb_candidates(U, U, self_join=True)
    exp = oracle_flags("urban self join 55,000 meshes", U, U, cand)
    want = cand[exp.astype(bool)]
    h = ctx.load(U)
    ctx.build(h, 4, 4)
    got, info = ctx.join(h, h, self_join=True, use_graph=True)
    assert info["n_candidates"] == len(cand)
    assert np.array_equal(got, want)                # every candidate
    got_exact, _ = ctx.join(h, h, self_join=True, leaf_mode=pierce.PJ_LEAF_EXACT)
    assert np.array_equal(got_exact, want)
