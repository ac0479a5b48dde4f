"""The bounding-box filter join by sort and sweep (Sec. 3.1, the filter step),
taken when the all-pairs count passes 2^24: the device candidate list must be
the oracle's, in the oracle's order (checked through the per-candidate flags,
which line up with the device list), and the refined pair set the oracle's,
for a self join and for a join of two different datasets."""
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


def _check(ctx, name, A, B, self_join):
    ma, mb = A.nmesh, B.nmesh
    assert (ma * (ma - 1) // 2 if self_join else ma * mb) > (1 << 24)  # the sweep path
    cand = oracle.mbb_candidates(A, B, self_join=self_join)
    flags = oracle_flags(name, A, B, cand)
    ha = ctx.load(A)
    hb = ha if self_join else ctx.load(B)
    ctx.build(ha, 4, 2)
    if not self_join:
        ctx.build(hb, 4, 2)
    res = pierce.pj_join_intersects_ex(ctx.h, ha, hb, self_join=self_join, width=4, leaf_size=2,
                                       out_host=True, keep_flags=True)
    n = int(res.n_candidates)
    got_flags = pierce.device_to_numpy(res.flags, n, np.uint8)
    got = pierce.pairs_to_numpy(res)
    pierce.pj_free_pairs(ctx.h, res)
    assert n == len(cand)
    assert np.array_equal(got_flags, flags)     # the same list, in the same order
    assert np.array_equal(got, cand[flags.astype(bool)])
    again, info = ctx.join(ha, hb, self_join=self_join, use_graph=True)
    assert info["n_candidates"] == len(cand) and np.array_equal(again, got)
    return len(cand), len(got)


def test_self_join(ctx):
    U = synth.urban(5003, n_buildings=5600, n_parts=600)
    c, k = _check(ctx, "urban self join 6,200 meshes", U, U, True)
    assert c > 1000 and k > 100


def test_two_datasets(ctx):
    A = synth.urban(5004, n_buildings=3900, n_parts=400)
    B = synth.urban(5005, n_buildings=3900, n_parts=400)
    c, k = _check(ctx, "urban x urban 4,300 x 4,300 meshes", A, B, False)
    assert c > 1000 and k > 100
