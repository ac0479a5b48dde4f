"""The device selectivity estimate (pj_estimate_join, paper Sec. 3.5)
against the oracle's statement of it (oracle/estimate.py): the total and
every cell's expected pair count, on uniform cubes, tiny spheres, the urban
buildings and the full pathology datasets, at several grid sizes.  Floating
point: both sides sum in float64 in different orders, so the comparison is
relative, 1e-9 (the terms are products and sums of a few thousand doubles;
their rounding is about 1e-13 relative)."""
import numpy as np
import pytest

import oracle
from oracle import estimate as orc_est
from paper_2609_24513_gb300 import pierce, synth

pytestmark = pytest.mark.gpu

REL = 1e-9


def _cubes(rng, n, side, lo=20000, hi=240000):
    c = rng.integers(lo, hi - side, size=(n, 3))
    return synth.concat([synth.box(tuple(p), tuple(p + side)) for p in c])


def _check(ctx, A, B, G):
    ha, hb = ctx.load(A), ctx.load(B)
    got = pierce.pj_estimate_join(ctx.h, ha, hb, G, cells=True)
    e, E, slots = orc_est.estimate(A, B, G)
    assert got["grid"] == G
    assert abs(got["e_final"] - e) <= REL * max(e, 1e-300)
    assert abs(got["slots"] - slots) <= REL * max(slots, 1e-300)
    np.testing.assert_allclose(got["cells"].reshape(G, G, G), E, rtol=REL, atol=1e-300)
    assert got["cells_occupied"] >= int((E > 0).sum())
    pierce.pj_free_dataset(ctx.h, ha)
    pierce.pj_free_dataset(ctx.h, hb)
    return got


@pytest.fixture(scope="module")
def ctx():
    c = pierce.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("G", [1, 4, 16, 37])
def test_uniform_cubes(ctx, G):
    rng = np.random.default_rng(G)
    A, B = _cubes(rng, 300, 4000), _cubes(rng, 200, 9000)
    got = _check(ctx, A, B, G)
    assert got["e_final"] > 0


@pytest.mark.parametrize("G", [2, 16])
def test_tiny_spheres_and_urban(ctx, G):
    A, B = synth.tiny_spheres(1001)
    _check(ctx, A, B, G)
    U = synth.urban(5001, n_buildings=1500, n_parts=150)
    _check(ctx, U, U, G)


def test_pathology_full(ctx, pathology_truth):
    A, B, cand, flags = pathology_truth
    got = _check(ctx, A, B, 16)
    # context, not a pin: the estimate against the true number of pairs
    print("pathology estimate %.1f pairs (true %d), %.3f ms" % (got["e_final"], int(flags.sum()),
                                                                 got["ms"]))


def test_bad_grid_is_refused(ctx):
    A, B = synth.tiny_spheres(5, n_a=2, n_b=2)
    ha, hb = ctx.load(A), ctx.load(B)
    with pytest.raises(pierce.PierceError):
        pierce.pj_estimate_join(ctx.h, ha, hb, 257)
