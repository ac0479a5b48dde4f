"""The dataset-level join (pj_dataset_join: one BVH per dataset, every owned
edge traced both ways with all of its crossings, one parity ray per object,
pairs deduplicated by a hashmap sized by the estimate, by counting two-pass
or by a fixed hashmap; paper Sec. 3.1-3.5) against the oracle, for the
intersects and overlap predicates: tiny spheres at three BVH shapes,
hand-built solids in both roles, exhaustive lattice placements (many parity
vertices on the other surface: the per-pair recheck), a self join of urban
buildings and the full pathology workload.  Pair sets compared exactly."""
import numpy as np
import pytest

import oracle
from cases import HAND, lattice_case_sets
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu

MATS = ("estimated", "two_pass", "fixed")


@pytest.fixture(scope="module")
def ctx():
    c = pierce.Context(0)
    yield c
    c.close()


def _truth(A, B, pred, self_join=False):
    cand = oracle.mbb_candidates(A, B, self_join)
    return cand[oracle.join(A, B, cand, predicate=pred, threads=None).astype(bool)]


@pytest.mark.parametrize("W,L", [(4, 2), (8, 4), (2, 1)])
def test_tiny_spheres(ctx, W, L):
    for seed in (1001, 1002, 1003):
        A, B = synth.tiny_spheres(seed)
        ha, hb = ctx.load(A), ctx.load(B)
        for pred in ("intersects", "overlap"):
            want = _truth(A, B, pred)
            for mat in MATS:
                got, st = pierce.pj_dataset_join(ctx.h, ha, hb, width=W, leaf_size=L,
                                                 predicate=pred, materialize=mat)
                assert np.array_equal(got, want), (seed, pred, mat)
                assert st["hits"] >= 0 and st["edges"] > 0


def test_hand_built_both_roles(ctx):
    for name, (ma, mb, _) in sorted(HAND.items()):
        for X, Y in ((ma, mb), (mb, ma)):
            A, B = synth.concat([X]), synth.concat([Y])
            ha, hb = ctx.load(A), ctx.load(B)
            for pred in ("intersects", "overlap"):
                want = _truth(A, B, pred)
                for mat in MATS:
                    got, _ = pierce.pj_dataset_join(ctx.h, ha, hb, predicate=pred, materialize=mat)
                    assert np.array_equal(got, want), (name, pred, mat)
            pierce.pj_free_dataset(ctx.h, ha)
            pierce.pj_free_dataset(ctx.h, hb)


def test_lattice_placements_recheck(ctx):
    A, B, cand, _ = lattice_case_sets()
    ha, hb = ctx.load(A), ctx.load(B)
    want = _truth(A, B, "intersects")
    for mat in MATS:
        got, st = pierce.pj_dataset_join(ctx.h, ha, hb, materialize=mat)
        assert np.array_equal(got, want), mat
    assert st["recheck_pairs"] > 0          # vertices on the other surface were rechecked


def test_urban_self_join(ctx):
    U = synth.urban(5001, n_buildings=2000, n_parts=200)
    h = ctx.load(U)
    want = _truth(U, U, "intersects", self_join=True)
    for mat in MATS:
        got, _ = pierce.pj_dataset_join(ctx.h, h, h, self_join=True, materialize=mat)
        assert np.array_equal(got, want), mat
        assert np.all(got[:, 0] < got[:, 1])


def test_overflowing_fixed_hashmap_relaunches(ctx):
    A, B = synth.tiny_spheres(1002)
    ha, hb = ctx.load(A), ctx.load(B)
    want = _truth(A, B, "intersects")
    got, st = pierce.pj_dataset_join(ctx.h, ha, hb, materialize="fixed", fixed_slots=16)
    assert np.array_equal(got, want)
    assert st["relaunches"] > 0 and st["slots"] > 16


def test_pathology_full(ctx, pathology_truth):
    A, B, cand, flags = pathology_truth
    want = cand[flags.astype(bool)]
    ha, hb = ctx.load(A), ctx.load(B)
    for mat in MATS:
        got, st = pierce.pj_dataset_join(ctx.h, ha, hb, materialize=mat)
        assert np.array_equal(got, want), mat
        print("dataset join %s: %d pairs, %.2f ms (trace %.2f, materialise %.2f), %d edges, "
              "%d crossings, %d slots, %d relaunches, %d rechecked"
              % (mat, len(got), st["ms_total"], st["ms_trace"], st["ms_materialize"],
                 st["edges"], st["hits"], st["slots"], st["relaunches"], st["recheck_pairs"]))
